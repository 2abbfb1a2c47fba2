"""Pins for the oracle's shape-complementarity score (Sec. 4.2, Eq. (score)).

Each check ties the score to something other than its own code: the exact
zero mode (products of ball volumes), the reduction to the already pinned
correlation when the offset is zero, the exact lens-volume score (layer (a))
that the band-limited score must approach as the mode box grows, and the
one-ball-each case against the four closed-form lens volumes.  A dropped
term, a flipped sign or an offset applied to one shape only fails one of
them.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1711_05075_gb300 import synth


def vol(r):
    return 4.0 / 3.0 * math.pi * np.asarray(r, dtype=np.float64) ** 3


def _pair(n=40, seed=9):
    return synth.ellipsoid_shape(n, seed), synth.torus_shape(n, seed + 1)


@pytest.mark.parametrize("r0,lam", [(0.03, 2.0), (0.05, 0.7)])
def test_score_zero_mode_is_a_product_of_volumes(r0, lam):
    A, B = _pair(30, 2)
    q = synth.shoemake_quaternions(synth.SplitMix64(1), 1)[0]
    G = O.score_spectrum(A, B, q, 8, r0, lam)
    wa = (vol(A.r() + r0) - lam * vol(A.r())).sum()
    wb = (vol(B.r() + r0) - lam * vol(B.r())).sum()
    assert G[0, 0, 0].real == pytest.approx(-wa * wb, rel=1e-13)
    assert abs(G[0, 0, 0].imag) < 1e-14 * abs(wa * wb)


def test_score_without_offset_is_the_negated_correlation():
    # r0 = 0: F_S = i (1 - lambda) f_S, so G = -(1 - lambda)^2 g
    A, B = _pair(30, 4)
    q = synth.shoemake_quaternions(synth.SplitMix64(2), 1)[0]
    lam = 2.5
    G = O.band_limited_score(A, B, q, 16, 0.0, lam)
    g = O.band_limited_corr(A, B, q, 16)
    np.testing.assert_allclose(G, -(1 - lam) ** 2 * g, rtol=1e-12, atol=1e-12 * np.abs(g).max())


def test_band_limited_score_converges_to_exact_score():
    # The four terms nearly cancel (|G| is about a tenth of the terms' sizes), so the
    # gap is measured against the sum of the terms' norms, the scale of the truncation
    # error of each; it must fall with N like that of the correlation.
    A, B = _pair()
    q = synth.shoemake_quaternions(synth.SplitMix64(4), 1)[0]
    r0, lam = 0.03, 2.0
    errs = []
    for N in (8, 16, 32, 48):
        t = O.grid_points(N)
        gb = O.band_limited_score(A, B, q, N, r0, lam).reshape(-1)
        ga = O.exact_score(A.xyz, A.r(), B.xyz, B.r(), t, r0, lam, q=q)
        scale = sum(abs(c) * np.linalg.norm(O.exact_corr(A.xyz, A.r() + da, B.xyz, B.r() + db, t, q))
                    for da, db, c in ((0, 0, lam ** 2), (r0, 0, lam), (0, r0, lam), (r0, r0, 1.0)))
        errs.append(np.linalg.norm(gb - ga) / scale)
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:])), errs
    assert errs[3] < errs[1] / 4 and errs[-1] < 6e-3, errs


def test_one_ball_each_matches_the_four_lens_volumes():
    # G(t) = -lam^2 V(r1, r2, d) + lam V(r1 + r0, r2, d) + lam V(r1, r2 + r0, d) - V(r1 + r0, r2 + r0, d),
    # d = |c1 - c2 - t| (nearest image); the band-limited score approaches it.
    r1, r2, r0, lam = 0.3, 0.2, 0.1, 1.5  # balls several grid cells wide at N = 48
    A = synth.Shape(np.array([[0.1, -0.05, 0.02]]), np.array([0], np.int32), (r1,))
    B = synth.Shape(np.array([[-0.2, 0.1, 0.0]]), np.array([0], np.int32), (r2,))
    N = 48
    t = O.grid_points(N)
    d = A.xyz[0] - B.xyz[0] - t
    d -= 2.0 * np.round(d / 2.0)
    d = np.linalg.norm(d, axis=1)
    V = O.lens_volume
    ref = -lam ** 2 * V(r1, r2, d) + lam * V(r1 + r0, r2, d) + lam * V(r1, r2 + r0, d) - V(r1 + r0, r2 + r0, d)
    got = O.band_limited_score(A, B, synth.IDENTITY_QUAT[0], N, r0, lam).reshape(-1)
    scale = sum(abs(c) * np.linalg.norm(V(a, b, d)) for a, b, c in
                ((r1, r2, lam ** 2), (r1 + r0, r2, lam), (r1, r2 + r0, lam), (r1 + r0, r2 + r0, 1.0)))
    assert np.linalg.norm(got - ref) / scale < 5e-3
    # and the exact layer gives the closed form itself
    ex = O.exact_score(A.xyz, A.r(), B.xyz, B.r(), t, r0, lam)
    np.testing.assert_allclose(ex, ref, rtol=1e-12, atol=1e-15)
