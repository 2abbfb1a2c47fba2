"""Pins for the oracle's truncated single-configuration query (Sec. 4.1, Eq. (single)).

The mode order is checked by hand on a small case; with every mode the query
must equal numpy's inverse FFT of the full Hermitian spectrum at the grid
points; with one mode it is the product of the shapes' volumes over P^3; and
on the grid the squared error of any truncation equals, by the discrete
Parseval identity, the energy of the dropped modes.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1711_05075_gb300 import synth

P = 2.0


def vol(r):
    return 4.0 / 3.0 * math.pi * np.asarray(r, dtype=np.float64) ** 3


def _spectrum(N, seed=5):
    A, B = synth.ellipsoid_shape(30, seed), synth.torus_shape(30, seed + 1)
    q = synth.shoemake_quaternions(synth.SplitMix64(seed), 1)[0]
    return A, B, O.band_limited_spectrum(A, B, q, N)


def _full(ghat):
    """Full N^3 spectrum in FFT order from the stored half (Hermitian, Nyquist planes zero)."""
    N = ghat.shape[0]
    full = np.zeros((N, N, N), dtype=np.complex128)
    full[:, :, : N // 2] = ghat[:, :, : N // 2]
    j = np.arange(N)
    neg = (-j) % N
    for mz in range(1, N // 2):
        full[:, :, N - mz] = np.conj(ghat[np.ix_(neg, neg)][:, :, mz])
    return full


def test_mode_order_by_hand():
    m, w = O.query_modes(8, 8)
    expect = [(0, 0, 0), (0, 0, 1), (0, 1, 0), (1, 0, 0),           # |m|^2 = 0, 1
              (-1, 0, 1), (-1, 1, 0), (0, -1, 1), (0, 1, 1)]         # |m|^2 = 2, by (m_x, m_y, m_z)
    assert [tuple(x) for x in m] == expect
    np.testing.assert_array_equal(w, [1, 2, 2, 2, 2, 2, 2, 2])
    total = ((8 - 1) ** 3 + 1) // 2
    assert O.query_modes(8, 10 ** 6)[0].shape[0] == total


def test_all_modes_equal_numpy_inverse_fft_on_the_grid():
    N = 16
    _, _, g = _spectrum(N)
    m, w = O.query_modes(N, 10 ** 6)
    got = O.query_at(g, m, w, O.grid_points(N)).reshape(N, N, N)
    j = np.arange(N)
    sgn = np.where(j < N // 2, j, j - N) % 2
    sign = (-1.0) ** (sgn[:, None, None] + sgn[None, :, None] + sgn[None, None, :])  # t_k = -P/2 + k P/N
    ref = np.fft.ifftn(_full(g) * sign).real * N ** 3 / P ** 3
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


def test_one_mode_is_the_volume_product():
    A, B, g = _spectrum(16)
    m, w = O.query_modes(16, 1)
    t = np.random.default_rng(0).uniform(-1, 1, (7, 3))
    np.testing.assert_allclose(O.query_at(g, m, w, t), vol(A.r()).sum() * vol(B.r()).sum() / P ** 3, rtol=1e-12)


@pytest.mark.parametrize("mprime", [1, 10, 123, 800])
def test_truncation_error_is_the_dropped_energy(mprime):
    # sum_k |g(t_k) - g'(t_k)|^2 = N^3 P^-6 sum_{dropped m (both signs)} |g^(m)|^2
    N = 12
    _, _, g = _spectrum(N, 7)
    m_all, w_all = O.query_modes(N, 10 ** 6)
    t = O.grid_points(N)
    full = O.query_at(g, m_all, w_all, t)
    part = O.query_at(g, m_all[:mprime], w_all[:mprime], t)
    dropped = m_all[mprime:]
    energy = (w_all[mprime:] * np.abs(g[dropped[:, 0] % N, dropped[:, 1] % N, dropped[:, 2]]) ** 2).sum()
    assert np.sum((full - part) ** 2) == pytest.approx(N ** 3 * energy / P ** 6, rel=1e-9)
