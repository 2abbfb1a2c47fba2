"""Pins for the FP64 oracle: each check ties it to something other than itself.

Closed forms, textbook special cases, quadrature, Monte Carlo, a library
rotation, exact invariants of the Fourier form, and convergence of the
band-limited layer (b) to the exact layer (a).  A plausible slip in the oracle
(a dropped term, a flipped sign, a wrong index, a transposed operand, a level
mix-up) fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1711_05075_gb300 import synth

P = 2.0


def vol(r):
    return 4.0 / 3.0 * math.pi * np.asarray(r, dtype=np.float64) ** 3


# ------------------------------------------------------------------ lens volume
def test_lens_special_cases():
    r1, r2 = 0.3, 0.2
    assert O.lens_volume(r1, r2, 0.0) == pytest.approx(vol(0.2), rel=1e-15)
    assert O.lens_volume(r1, r2, 0.09) == pytest.approx(vol(0.2), rel=1e-15)  # contained
    assert O.lens_volume(r1, r2, 0.5) == 0.0
    assert O.lens_volume(r1, r2, 0.7) == 0.0
    # continuous at both ends of the cap formula
    for d0 in (abs(r1 - r2), r1 + r2):
        lo = O.lens_volume(r1, r2, d0 - 1e-9)
        hi = O.lens_volume(r1, r2, d0 + 1e-9)
        assert abs(lo - hi) < 1e-7 * vol(0.2)


def test_lens_equal_radii_textbook():
    # Two equal balls: V = pi (4r + d)(2r - d)^2 / 12 (standard lens formula).
    r = 0.25
    d = np.linspace(0.0, 2 * r, 41)[1:-1]
    ref = math.pi * (4 * r + d) * (2 * r - d) ** 2 / 12.0
    np.testing.assert_allclose(O.lens_volume(r, r, d), ref, rtol=1e-13)


@pytest.mark.parametrize("r1,r2,d", [(0.3, 0.2, 0.25), (0.1, 0.08, 0.05), (0.2, 0.2, 0.3)])
def test_lens_monte_carlo(r1, r2, d):
    rng = np.random.default_rng(1234)
    n = 2_000_000
    p = (rng.random((n, 3)) * 2 - 1) * r1  # box around ball 1 centred at 0
    in1 = (p ** 2).sum(1) <= r1 * r1
    in2 = ((p - np.array([d, 0.0, 0.0])) ** 2).sum(1) <= r2 * r2
    frac = np.mean(in1 & in2)
    box = (2 * r1) ** 3
    est = box * frac
    sig = box * math.sqrt(frac * (1 - frac) / n)
    assert abs(O.lens_volume(r1, r2, d) - est) < 4 * sig


# ------------------------------------------------------------------ ball FT
def test_ball_ft_zero_limit_is_volume():
    r = np.array([0.01, 0.04, 0.08, 0.3])
    np.testing.assert_allclose(O.ball_ft(r, 0.0), vol(r), rtol=1e-15)
    np.testing.assert_allclose(O.ball_ft(r, 1e-9), vol(r), rtol=1e-14)


def test_ball_ft_series_branch_vs_high_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    r = 0.08
    for x in [1e-4, 1e-2, 0.1, 0.3, 0.4999, 0.5, 0.5001, 2.0, 7.5]:
        k = x / r
        ref = 4 * mp.pi * (mp.sin(mp.mpf(x)) - x * mp.cos(mp.mpf(x))) / mp.mpf(k) ** 3
        assert float(O.ball_ft(r, k)) == pytest.approx(float(ref), rel=2e-13, abs=1e-18)


def test_ball_ft_vs_radial_quadrature():
    # F{1_ball}(omega) = 4 pi int_0^r s^2 sin(k s)/(k s) ds, k = 2 pi |omega|.
    from scipy.integrate import quad
    for r in (0.04, 0.08):
        for k in (0.0, 3.0, 40.0, 150.0, 400.0):
            f = (lambda s: s * s * math.sin(k * s) / (k * s)) if k > 0 else (lambda s: s * s)
            ref = 4 * math.pi * quad(f, 0.0, r, epsabs=1e-16, epsrel=1e-12, limit=200)[0]
            assert O.ball_ft(r, k) == pytest.approx(ref, rel=1e-10, abs=1e-16)


# ------------------------------------------------------------------ rotations
def test_rotation_matches_scipy():
    from scipy.spatial.transform import Rotation
    q = synth.shoemake_quaternions(synth.SplitMix64(7), 16)
    for qq in q:
        ref = Rotation.from_quat([qq[1], qq[2], qq[3], qq[0]]).as_matrix()
        np.testing.assert_allclose(O.quat_to_matrix(qq), ref, atol=1e-14)
        np.testing.assert_allclose(O.quat_to_matrix(-3.0 * qq), ref, atol=1e-14)


def test_rotation_90_about_z():
    c = math.cos(math.pi / 4)
    q = np.array([c, 0.0, 0.0, c])
    np.testing.assert_allclose(O.rotate(np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.5]]), q),
                               [[0.0, 1.0, 0.0], [-1.0, 0.0, 0.5]], atol=1e-15)
    with pytest.raises(ValueError):
        O.quat_to_matrix(np.zeros(4))


# ------------------------------------------------------------------ layer (a)
def test_exact_two_balls_geometry():
    # B's ball at R c2 + t sits on A's ball at c1 exactly when t = c1 - R c2.
    c1 = np.array([[0.3, 0.0, 0.0]])
    c2 = np.array([[0.0, 0.3, 0.0]])
    c = math.cos(math.pi / 4)
    q = np.array([c, 0.0, 0.0, c])  # R c2 = (-0.3, 0, 0)
    t = np.array([[0.6, 0.0, 0.0], [0.6 + 0.05, 0.0, 0.0], [0.0, 0.0, 0.0], [-0.6, 0.0, 0.0]])
    g = O.exact_corr(c1, [0.08], c2, [0.04], t, q=q)
    assert g[0] == pytest.approx(vol(0.04), rel=1e-14)
    assert g[1] == pytest.approx(O.lens_volume(0.08, 0.04, 0.05), rel=1e-14)
    assert g[2] == 0.0 and g[3] == 0.0


def test_exact_periodic_wrap():
    # Centres 1.9 apart along x touch through the periodic image (P = 2).
    a = np.array([[0.95, 0.0, 0.0]])
    b = np.array([[-0.95, 0.0, 0.0]])
    g = O.exact_corr(a, [0.08], b, [0.08], np.array([[0.0, 0.0, 0.0], [-0.1, 0.0, 0.0]]))
    assert g[0] == pytest.approx(O.lens_volume(0.08, 0.08, 0.1), rel=1e-13)
    assert g[1] == pytest.approx(vol(0.08), rel=1e-13)


# ------------------------------------------------------------------ layer (b)
def _pair(n=48, seed=3):
    A = synth.ellipsoid_shape(n, seed)
    B = synth.torus_shape(n, seed + 1)
    return A, B


def test_spectrum_zero_mode_is_volume():
    A, B = _pair()
    fa = O.shape_spectrum(A.xyz, A.level, A.radii, 8)
    assert fa[0, 0, 0].real == pytest.approx(vol(A.r()).sum(), rel=1e-14)
    assert abs(fa[0, 0, 0].imag) < 1e-15
    g = O.band_limited_spectrum(A, B, synth.IDENTITY_QUAT[0], 8)
    assert g[0, 0, 0].real == pytest.approx(vol(A.r()).sum() * vol(B.r()).sum(), rel=1e-14)


def test_sum_over_translations_is_volume_product():
    A, B = _pair()
    q = synth.shoemake_quaternions(synth.SplitMix64(11), 1)[0]
    for N in (8, 16):
        g = O.band_limited_corr(A, B, q, N)
        assert (P / N) ** 3 * g.sum() == pytest.approx(vol(A.r()).sum() * vol(B.r()).sum(), rel=1e-12)


def test_single_knot_spectrum_is_ball_ft_times_shift():
    # One ball at c: f^(m) = h^(r, 2 pi |m|/P) exp(-2 pi i m.c/P) (shift multiplier, App. C).
    N = 8
    c = np.array([[0.3, -0.2, 0.45]])
    f = O.shape_spectrum(c, [1], (0.02, 0.08), N)
    m = np.fft.fftfreq(N, 1.0 / N)
    mx, my, mz = np.meshgrid(m, m, np.arange(N // 2 + 1), indexing="ij")
    k = 2 * math.pi * np.sqrt(mx ** 2 + my ** 2 + mz ** 2) / P
    # magnitude from the radial ball transform, phase read off at three axis modes
    np.testing.assert_allclose(np.abs(f), np.abs(O.ball_ft(0.08, k)), rtol=1e-12, atol=1e-18)
    for ax, mode in ((0, (1, 0, 0)), (1, (0, 1, 0)), (2, (0, 0, 1))):
        ang = np.angle(f[mode])  # h^ > 0 at k = 2 pi / P for r = 0.08
        assert math.remainder(ang + 2 * math.pi * c[0, ax] / P, 2 * math.pi) == pytest.approx(0.0, abs=1e-12)


def test_levels_are_independent_of_their_order():
    A, _ = _pair()
    f1 = O.shape_spectrum(A.xyz, A.level, A.radii, 8)
    f2 = O.shape_spectrum(A.xyz, 1 - A.level, A.radii[::-1], 8)
    np.testing.assert_allclose(f1, f2, rtol=1e-13, atol=1e-16)
    f3 = O.shape_spectrum(A.xyz, np.zeros_like(A.level), (0.08,), 8)
    f4 = O.shape_spectrum(A.xyz, np.ones_like(A.level), (0.01, 0.08), 8)
    np.testing.assert_allclose(f3, f4, rtol=1e-13, atol=1e-16)
    with pytest.raises(ValueError):
        O.shape_spectrum(A.xyz, A.level + 5, A.radii, 8)


def test_grid_and_pointwise_inverse_agree():
    A, B = _pair()
    N = 16
    g = O.band_limited_spectrum(A, B, synth.IDENTITY_QUAT[0], N)
    full = O.inverse_grid(g)
    idx = synth.translation_sample(N, 200, seed=5)
    pts = O.inverse_at(g, O.grid_points(N, idx=idx))
    np.testing.assert_allclose(pts, full.reshape(-1)[idx], rtol=1e-11, atol=1e-14 * np.abs(full).max())


def test_grid_translation_is_cyclic_shift():
    # Moving B by s = v P/N turns g(t) into g(t + s): a cyclic shift by v on the grid.
    A, B = _pair()
    N = 16
    v = np.array([3, -2, 5])
    s = v * P / N
    B2 = synth.Shape(B.xyz + s, B.level, B.radii)
    q = synth.IDENTITY_QUAT[0]
    g = O.band_limited_corr(A, B, q, N)
    g2 = O.band_limited_corr(A, B2, q, N)
    np.testing.assert_allclose(g2, np.roll(g, shift=tuple(-v), axis=(0, 1, 2)), rtol=1e-10,
                               atol=1e-12 * np.abs(g).max())


def test_off_grid_translation_covariance():
    A, B = _pair()
    N = 16
    s = np.array([0.0371, -0.0213, 0.0517])
    B2 = synth.Shape(B.xyz + s, B.level, B.radii)
    q = synth.IDENTITY_QUAT[0]
    g = O.band_limited_spectrum(A, B, q, N)
    g2 = O.inverse_grid(O.band_limited_spectrum(A, B2, q, N))
    idx = synth.translation_sample(N, 100, seed=2)
    t = O.grid_points(N, idx=idx)
    np.testing.assert_allclose(g2.reshape(-1)[idx], O.inverse_at(g, t + s), rtol=1e-10,
                               atol=1e-12 * np.abs(g2).max())


def test_swap_shapes_reflects_translation():
    A, B = _pair()
    N = 16
    q = synth.IDENTITY_QUAT[0]
    gab = O.band_limited_corr(A, B, q, N)
    gba = O.band_limited_corr(B, A, q, N)
    neg = (-np.arange(N)) % N  # -t_k = t_{N-k} on the periodic grid
    np.testing.assert_allclose(gba, gab[np.ix_(neg, neg, neg)], rtol=1e-10, atol=1e-12 * np.abs(gab).max())


def test_rotation_equals_prerotated_knots():
    A, B = _pair()
    N = 8
    c = math.cos(math.pi / 4)
    q = np.array([c, 0.0, 0.0, c])
    rotated = np.stack([-B.xyz[:, 1], B.xyz[:, 0], B.xyz[:, 2]], axis=1)  # 90 deg about z, by hand
    g1 = O.band_limited_corr(A, B, q, N)
    g2 = O.band_limited_corr(A, synth.Shape(rotated, B.level, B.radii), synth.IDENTITY_QUAT[0], N)
    np.testing.assert_allclose(g1, g2, rtol=1e-11, atol=1e-13 * np.abs(g1).max())


def test_band_limited_converges_to_exact():
    # The periodised exact correlation has Fourier coefficients g^(m)/P^3 (Poisson summation),
    # so layer (b) must approach layer (a) as the mode box grows; the spectrum of the lens
    # volume falls like |m|^-4, so the rel-L2 gap falls roughly like N^-2.5.
    A, B = _pair(n=40, seed=9)
    q = synth.shoemake_quaternions(synth.SplitMix64(4), 1)[0]
    errs = []
    for N in (8, 16, 32, 48):
        gb = O.band_limited_corr(A, B, q, N)
        ga = O.exact_corr(A.xyz, A.r(), B.xyz, B.r(), O.grid_points(N), q=q).reshape(N, N, N)
        errs.append(np.linalg.norm(gb - ga) / np.linalg.norm(ga))
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:])), errs
    assert errs[2] < errs[1] / 4 and errs[-1] < 8e-3, errs
