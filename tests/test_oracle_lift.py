"""Pins for the oracle's lifted (4D) nonequiradius correlation (Sec. 3.2).

The cone transform against closed forms and scipy's adaptive quadrature; the
closed-form pair volume against special cases and against scipy quadrature
of the lens volume along the lifted axis; the exact layer's support against
Lemma 2 (positive exactly where two balls intersect); the exact zero mode;
single-knot phases with the rotation and the mirror; and convergence of the
band-limited layer to the exact one in the r = 0 and an offset section.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1711_05075_gb300 import synth

scipy_integrate = pytest.importorskip("scipy.integrate")

L, P, PR = 0.1, 2.0, 0.4


def test_cone_ft_closed_forms_and_quadrature():
    assert O.cone_ft(0.0, 0.0, L) == pytest.approx(math.pi * L ** 4 / 3, rel=1e-14)
    for k in (3.0, 30.0, 120.0):
        ref = 4 * math.pi / k ** 3 * (2 * (1 - math.cos(k * L)) / k - L * math.sin(k * L))
        assert O.cone_ft(k, 0.0, L).real == pytest.approx(ref, rel=1e-12, abs=1e-18)
    for k, a in ((0.0, 40.0), (25.0, -60.0), (90.0, 150.0)):
        def h(s):
            return float(O.ball_ft(s, k))
        re = scipy_integrate.quad(lambda s: h(s) * math.cos(a * s), 0, L, epsabs=1e-16, epsrel=1e-13, limit=200)[0]
        im = scipy_integrate.quad(lambda s: h(s) * math.sin(a * s), 0, L, epsabs=1e-16, epsrel=1e-13, limit=200)[0]
        got = complex(O.cone_ft(k, a, L))
        assert abs(got - complex(re, im)) <= 1e-11 * abs(complex(re, im)) + 1e-19


def _pair_quad(ri, rj, rs, d, LL):
    lo, hi = max(ri - LL, rs - rj), min(ri, rs - rj + LL)
    if hi <= lo:
        return 0.0
    f = lambda s: float(O.lens_volume(ri - s, s + rj - rs, d))
    c = ri - rj + rs
    pts = [p for p in (0.5 * (c - d), 0.5 * (c + d)) if lo < p < hi]
    return scipy_integrate.quad(f, lo, hi, points=pts or None, epsabs=1e-18, epsrel=1e-12, limit=200)[0]


def test_lifted_pair_special_cases_and_quadrature():
    rho = 0.05
    assert O.lifted_pair(rho, rho, 0.0, 0.0, 1.0) == pytest.approx(2 / 3 * math.pi * rho ** 4, rel=1e-14)
    assert O.lifted_pair(0.05, 0.03, 0.0, 0.08, L) == 0.0  # touching: d = r_i + r_j
    assert O.lifted_pair(0.05, 0.03, 0.01, 0.075, L) == 0.0  # offset section shrinks the sum to 0.07
    rng = np.random.default_rng(3)
    for _ in range(40):
        ri, rj = rng.uniform(0.01, 0.09, 2)
        rs = rng.uniform(-0.05, 0.05)
        d = rng.uniform(0, 0.2)
        ref = _pair_quad(ri, rj, rs, d, L)
        assert O.lifted_pair(ri, rj, rs, d, L) == pytest.approx(ref, rel=1e-9, abs=1e-16)


def _knots(n, seed, lo=0.03, hi=0.09):
    rng = synth.SplitMix64(seed)
    xyz = (rng.uniform(3 * n).reshape(n, 3) - 0.5) * 0.6
    r = lo + (hi - lo) * rng.uniform(n)
    return xyz, r


def test_exact_layer_support_is_lemma_2():
    # g(t, 0) > 0 exactly when some ball of A meets some ball of t + R B
    xa, ra = _knots(12, 1)
    xb, rb = _knots(9, 2)
    q = synth.shoemake_quaternions(synth.SplitMix64(3), 1)[0]
    t = np.random.default_rng(4).uniform(-1, 1, (3000, 3))
    g = O.lifted_exact(xa, ra, xb, rb, t, 0.0, L, q=q)
    yb = O.rotate(xb, q)
    d = xa[:, None, None, :] - yb[None, :, None, :] - t[None, None, :, :]
    d -= P * np.round(d / P)
    gap = np.linalg.norm(d, axis=-1) - (ra[:, None, None] + rb[None, :, None])
    overlap = (gap < 0).any(axis=(0, 1))
    assert overlap.any() and (~overlap).any()
    np.testing.assert_array_equal(g > 0, overlap)


def test_zero_mode_and_single_knot_phases():
    xa, ra = _knots(7, 5)
    xb, rb = _knots(5, 6)
    q = synth.shoemake_quaternions(synth.SplitMix64(7), 1)[0]
    g = O.lifted_corr_spectrum((xa, ra), (xb, rb), q, 8, 8, L, P, PR)
    assert g[0, 0, 0, 0].real == pytest.approx(7 * 5 * (math.pi * L ** 4 / 3) ** 2, rel=1e-13)
    # one knot: rho^(xi, eta) = exp(-2 pi i (xi.x/P + eta r/P_r)); mirrored: r -> -r; rotated: x -> R x
    x, r = np.array([[0.1, -0.2, 0.3]]), np.array([0.07])
    rho = O.lifted_spectrum(x, r, 8, 8, P, PR, q=q, mirror=True)
    y = O.quat_to_matrix(q) @ x[0]
    m = np.array([0, 1, 2, 3, -4, -3, -2, -1], dtype=np.float64)
    for ix, iy, iz, ie in ((1, 2, 3, 1), (7, 5, 1, 6), (0, 0, 2, 3)):
        ref = np.exp(-2j * np.pi * ((m[ix] * y[0] + m[iy] * y[1] + iz * y[2]) / P + m[ie] * (-r[0]) / PR))
        assert abs(rho[ix, iy, iz, ie] - ref) < 1e-13


def test_band_limited_converges_to_exact():
    xa, ra = _knots(6, 8, 0.05, 0.09)
    xb, rb = _knots(6, 9, 0.05, 0.09)
    q = synth.shoemake_quaternions(synth.SplitMix64(10), 1)[0]
    errs = {0.0: [], 0.03: []}
    for N, Nr in ((8, 8), (16, 16), (32, 32)):
        g = O.lifted_corr_spectrum((xa, ra), (xb, rb), q, N, Nr, L, P, PR)
        got = O.lifted_slices(g, list(errs), P, PR)
        for s, rs in enumerate(errs):
            ref = O.lifted_exact(xa, ra, xb, rb, O.grid_points(N, P), rs, L, q=q, period=P).reshape(N, N, N)
            errs[rs].append(np.linalg.norm(got[s] - ref) / np.linalg.norm(ref))
    for rs, e in errs.items():
        assert e[0] > e[1] > e[2], (rs, e)
        assert e[2] < 0.1, (rs, e)
