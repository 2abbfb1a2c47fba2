"""FP64 CPU oracle for the ball-union correlation (ctypes wrapper of oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg may import it; the product path never does.  It shares no
code with the CUDA path.  See oracle.c for the two layers and their citations.

Parity status: every function here is pinned by a CPU test against something
other than itself (closed forms, quadrature, Monte Carlo, library rotations,
invariants, and convergence of layer (b) to layer (a)); none is "parity unpinned".
The complementarity score (Sec. 4.2) is pinned by its exact zero mode, its
reduction to the correlation at r0 = 0 and its convergence to the exact
lens-volume score.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain gcc, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        d, i, vp = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        L.bco_lens_volume.restype = d
        L.bco_lens_volume.argtypes = [d, d, d]
        L.bco_lens_volume_many.argtypes = [i, vp, vp, vp, vp]
        L.bco_ball_ft.restype = d
        L.bco_ball_ft.argtypes = [d, d]
        L.bco_ball_ft_many.argtypes = [i, vp, vp, vp]
        L.bco_quat_to_matrix.restype = i
        L.bco_quat_to_matrix.argtypes = [vp, vp]
        L.bco_rotate.restype = i
        L.bco_rotate.argtypes = [i, vp, vp, vp]
        L.bco_exact_corr.restype = i
        L.bco_exact_corr.argtypes = [i, vp, vp, i, vp, vp, vp, d, i, vp, vp]
        L.bco_shape_spectrum.restype = i
        L.bco_shape_spectrum.argtypes = [i, vp, vp, i, vp, vp, d, i, vp]
        L.bco_corr_spectrum.argtypes = [i, vp, vp, vp]
        L.bco_inverse_at.argtypes = [i, d, vp, i, vp, vp]
        L.bco_inverse_grid.argtypes = [i, d, vp, vp]
        L.bco_lifted_pair.restype = d
        L.bco_lifted_pair.argtypes = [d, d, d, d, d]
        L.bco_lifted_exact.restype = i
        L.bco_lifted_exact.argtypes = [i, vp, vp, i, vp, vp, vp, d, d, d, i, vp, vp]
        _lib = L
    return _lib


def _f64(a):
    return np.require(np.asarray(a, dtype=np.float64), requirements="C")


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------------ primitives
def lens_volume(r1, r2, d):
    """Intersection volume of two balls (radii r1, r2, centre distance d); broadcasts."""
    r1, r2, d = np.broadcast_arrays(_f64(r1), _f64(r2), _f64(d))
    r1, r2, d = _f64(r1), _f64(r2), _f64(d)
    out = np.empty(r1.shape, dtype=np.float64)
    lib().bco_lens_volume_many(int(out.size), _ptr(r1), _ptr(r2), _ptr(d), _ptr(out))
    return out


def ball_ft(r, k):
    """FT of a ball indicator of radius r at angular wavenumber k; broadcasts."""
    r, k = np.broadcast_arrays(_f64(r), _f64(k))
    r, k = _f64(r), _f64(k)
    out = np.empty(r.shape, dtype=np.float64)
    lib().bco_ball_ft_many(int(out.size), _ptr(r), _ptr(k), _ptr(out))
    return out


def quat_to_matrix(q):
    q = _f64(q).reshape(4)
    R = np.empty(9, dtype=np.float64)
    if lib().bco_quat_to_matrix(_ptr(q), _ptr(R)):
        raise ValueError("zero quaternion")
    return R.reshape(3, 3)


def rotate(xyz, q):
    xyz = _f64(xyz).reshape(-1, 3)
    q = _f64(q).reshape(4)
    out = np.empty_like(xyz)
    if lib().bco_rotate(int(xyz.shape[0]), _ptr(xyz), _ptr(q), _ptr(out)):
        raise ValueError("zero quaternion")
    return out


# ------------------------------------------------------------------ layer (a)
def exact_corr(xa, ra, xb, rb, t, q=None, period=2.0):
    """Layer (a): periodised sum of lens volumes at translations t (nt x 3)."""
    xa, ra, xb, rb = _f64(xa).reshape(-1, 3), _f64(ra), _f64(xb).reshape(-1, 3), _f64(rb)
    t = _f64(t).reshape(-1, 3)
    out = np.empty(t.shape[0], dtype=np.float64)
    qa = None if q is None else _f64(q).reshape(4)
    qp = None if qa is None else _ptr(qa)
    rc = lib().bco_exact_corr(int(xa.shape[0]), _ptr(xa), _ptr(ra), int(xb.shape[0]), _ptr(xb),
                              _ptr(rb), qp, float(period), int(t.shape[0]), _ptr(t), _ptr(out))
    if rc == -2:
        raise ValueError("r_i + r_j must stay below P/2 for the nearest-image sum")
    if rc:
        raise ValueError("zero quaternion")
    return out


# ------------------------------------------------------------------ layer (b)
def shape_spectrum(xyz, level, radii, N, q=None, period=2.0):
    """Level-summed spectrum f^(m) on the Hermitian half, complex128 [N, N, N/2+1]."""
    xyz = _f64(xyz).reshape(-1, 3)
    level = np.ascontiguousarray(level, dtype=np.int32)
    radii = _f64(radii)
    out = np.empty((N, N, N // 2 + 1, 2), dtype=np.float64)
    qa = None if q is None else _f64(q).reshape(4)
    rc = lib().bco_shape_spectrum(int(xyz.shape[0]), _ptr(xyz), _ptr(level), int(radii.size),
                                  _ptr(radii), None if qa is None else _ptr(qa), float(period),
                                  int(N), _ptr(out))
    if rc == -3:
        raise ValueError("level id out of range")
    if rc:
        raise ValueError("zero quaternion")
    return out[..., 0] + 1j * out[..., 1]


def corr_spectrum(fa, fb):
    """g^ = f^_A conj(f^_B) with the Nyquist planes zeroed."""
    N = fa.shape[0]
    a = np.ascontiguousarray(np.stack([fa.real, fa.imag], axis=-1))
    b = np.ascontiguousarray(np.stack([fb.real, fb.imag], axis=-1))
    g = np.empty_like(a)
    lib().bco_corr_spectrum(int(N), _ptr(a), _ptr(b), _ptr(g))
    return g[..., 0] + 1j * g[..., 1]


def _pack(g):
    return np.ascontiguousarray(np.stack([g.real, g.imag], axis=-1))


def inverse_at(ghat, t, period=2.0):
    """g(t) = P^-3 sum_m g^(m) exp(2 pi i m.t / P) at arbitrary translations t (nt x 3)."""
    N = ghat.shape[0]
    t = _f64(t).reshape(-1, 3)
    out = np.empty(t.shape[0], dtype=np.float64)
    lib().bco_inverse_at(int(N), float(period), _ptr(_pack(ghat)), int(t.shape[0]), _ptr(t), _ptr(out))
    return out


def inverse_grid(ghat, period=2.0):
    """The same sum on the whole grid t_k = -P/2 + k P/N; returns [N, N, N] (kz fastest)."""
    N = ghat.shape[0]
    out = np.empty((N, N, N), dtype=np.float64)
    lib().bco_inverse_grid(int(N), float(period), _ptr(_pack(ghat)), _ptr(out))
    return out


# ------------------------------------------------------------------ helpers
def grid_points(N, period=2.0, idx=None):
    """Translations t_k = -P/2 + k P/N for linear indices idx (all N^3 when None)."""
    if idx is None:
        idx = np.arange(N ** 3, dtype=np.int64)
    idx = np.asarray(idx, dtype=np.int64)
    kx, ky, kz = idx // (N * N), (idx // N) % N, idx % N
    h = period / N
    return np.stack([-0.5 * period + kx * h, -0.5 * period + ky * h, -0.5 * period + kz * h], axis=1)


def band_limited_spectrum(A, B, q, N, period=2.0):
    """g^ for shapes A, B (synth.Shape) with B rotated by q; Nyquist planes zeroed."""
    fa = shape_spectrum(A.xyz, A.level, A.radii, N, None, period)
    fb = shape_spectrum(B.xyz, B.level, B.radii, N, q, period)
    return corr_spectrum(fa, fb)


def band_limited_corr(A, B, q, N, period=2.0, idx=None):
    """Layer (b) on the full translation grid (idx None) or at sampled linear indices."""
    g = band_limited_spectrum(A, B, q, N, period)
    if idx is None:
        return inverse_grid(g, period)
    return inverse_at(g, grid_points(N, period, idx), period)


# ------------------------------------------------------------------ shape complementarity (Sec. 4.2)
# Reading of Eq. (score): the affinity F_S = i (f_{S+B0} - lambda f_S), the
# offset S + B0 of a union of balls taken as the same knots with every radius
# grown by r0 (Sec. 4.2 observes that the offset raises the radii of the
# primitive balls), and the correlation of F_A with F_RB taken without complex
# conjugation, so that i * i = -1 and
#     G = -lambda^2 g_{A,B} + lambda g_{A+B0,B} + lambda g_{A,B+B0} - g_{A+B0,B+B0},
# which carries the signs the text assigns to the three terms (core-core
# penalty ~ -lambda^2, offset-core reward ~ +lambda, offset-offset penalty ~ -1).
def score_spectrum(A, B, q, N, r0, lam, period=2.0):
    """G^(m) on the Hermitian half: -W_A(m) conj(W_RB(m)), W_X = f^_{X+B0} - lambda f^_X,
    Nyquist planes zeroed."""
    ra, rb = _f64(A.radii), _f64(B.radii)
    wa = shape_spectrum(A.xyz, A.level, ra + r0, N, None, period) - lam * shape_spectrum(A.xyz, A.level, ra, N, None, period)
    wb = shape_spectrum(B.xyz, B.level, rb + r0, N, q, period) - lam * shape_spectrum(B.xyz, B.level, rb, N, q, period)
    return -corr_spectrum(wa, wb)


def band_limited_score(A, B, q, N, r0, lam, period=2.0, idx=None):
    """Layer (b) of the score on the full translation grid (idx None) or at sampled linear indices."""
    g = score_spectrum(A, B, q, N, r0, lam, period)
    if idx is None:
        return inverse_grid(g, period)
    return inverse_at(g, grid_points(N, period, idx), period)


def exact_score(xa, ra, xb, rb, t, r0, lam, q=None, period=2.0):
    """Layer (a) of the score: the four periodised lens-volume sums of Eq. (score)."""
    ra, rb = _f64(ra), _f64(rb)

    def E(a, b):
        return exact_corr(xa, a, xb, b, t, q, period)

    return -lam ** 2 * E(ra, rb) + lam * E(ra + r0, rb) + lam * E(ra, rb + r0) - E(ra + r0, rb + r0)


# ------------------------------------------------------------------ single-configuration queries (Sec. 4.1)
# Reading of the truncation in Eq. (single): the modes are taken outward from
# the origin (where the spectrum's magnitude concentrates), ordered by
# (|m|^2, m_x, m_y, m_z) over the canonical half space m_z > 0, or m_z = 0 and
# (m_y > 0, or m_y = 0 and m_x >= 0); each mode but m = 0 also stands for its
# conjugate -m (weight 2), so the truncated sum stays real.
def query_modes(N, mprime):
    """The first m' canonical modes (m' x 3 ints) and their weights."""
    h = N // 2 - 1
    r = np.arange(-h, h + 1)
    mx, my, mz = (a.ravel() for a in np.meshgrid(r, r, np.arange(0, h + 1), indexing="ij"))
    canon = (mz > 0) | (my > 0) | ((my == 0) & (mx >= 0))
    mx, my, mz = mx[canon], my[canon], mz[canon]
    q = mx * mx + my * my + mz * mz
    sel = np.lexsort((mz, my, mx, q))[:mprime]
    return np.stack([mx[sel], my[sel], mz[sel]], axis=1), np.where(q[sel] == 0, 1.0, 2.0)


def query_at(ghat, modes, w, t, period=2.0, chunk=4096):
    """g'(t) = P^-3 sum_i w_i Re(g^(m_i) exp(2 pi i m_i.t / P)), direct FP64 sum over the listed modes."""
    N = ghat.shape[0]
    t = _f64(t).reshape(-1, 3)
    modes = np.asarray(modes, dtype=np.int64)
    gm = ghat[modes[:, 0] % N, modes[:, 1] % N, modes[:, 2]] * np.asarray(w, dtype=np.float64)
    out = np.zeros(t.shape[0], dtype=np.float64)
    for s in range(0, modes.shape[0], chunk):
        ph = np.exp(2j * np.pi * (t @ modes[s:s + chunk].T.astype(np.float64)) / period)
        out += (ph * gm[s:s + chunk]).real.sum(axis=1)
    return out / period ** 3



# ------------------------------------------------------------------ lifted (4D) correlation (Sec. 3.2)
# Knots carry their own radii: knot (x, r) lifts to the trimmed half-cone
# D(x, r) = {(y, s) : |y - x| <= r - s, r - L <= s <= r} (Eq. (L2cone)), whose
# r = 0 section is the ball of radius r.  B is rotated and mirrored in r
# before the correlation (the pre-reflection of Sec. 3.2), and the lifted
# correlation g(t, r) is the 4D overlap volume of the two cone unions at the
# lifted translation (t, r).  Its r = 0 section is positive exactly where the
# two ball unions intersect (Lemma 2); r != 0 sections are the obstacles of
# offset shapes.  Fourier form (Eqs. (rhoAhat), (fconehat), (ccghat)):
#     rho^_X(xi, eta) = sum_i exp(-2 pi i (xi . x_i / P + eta r_i / P_r))
#     g^(xi, eta)     = rho^_A(xi, eta) conj(rho^_{R B mirrored}(xi, eta)) f^_D0(xi, eta)^2
#     f^_D0(xi, eta)  = int_0^L h^(s, 2 pi |xi| / P) exp(+2 pi i eta s / P_r) ds
#     g(t, r)         = P^-3 P_r^-1 sum g^(xi, eta) exp(2 pi i (xi . t / P + eta r / P_r)),
# xi in [-N/2, N/2)^3, eta in [-N_r/2, N_r/2), every mode with a component at
# the lower edge (-N/2 or -N_r/2) set to zero.
def lifted_pair(ri, rj, rs, d, L):
    """4D overlap volume of one cone pair at lifted offset rs, centre distance d (closed form)."""
    return lib().bco_lifted_pair(float(ri), float(rj), float(rs), float(d), float(L))


def lifted_exact(xa, ra, xb, rb, t, rs, L, q=None, period=2.0):
    """Layer (a): the lifted correlation at translations t (nt x 3) and lifted offset rs."""
    xa, ra, xb, rb = _f64(xa).reshape(-1, 3), _f64(ra), _f64(xb).reshape(-1, 3), _f64(rb)
    t = _f64(t).reshape(-1, 3)
    out = np.empty(t.shape[0], dtype=np.float64)
    qa = None if q is None else _f64(q).reshape(4)
    rc = lib().bco_lifted_exact(int(xa.shape[0]), _ptr(xa), _ptr(ra), int(xb.shape[0]), _ptr(xb), _ptr(rb),
                                None if qa is None else _ptr(qa), float(L), float(period), float(rs),
                                int(t.shape[0]), _ptr(t), _ptr(out))
    if rc == -2:
        raise ValueError("r_i + r_j + |r_s| must stay below P/2")
    if rc:
        raise ValueError("zero quaternion")
    return out


def _fft_modes(n):
    j = np.arange(n)
    return np.where(j < n // 2, j, j - n)


def lifted_spectrum(xyz, r, N, Nr, period=2.0, period_r=0.4, q=None, mirror=False):
    """rho^(xi, eta) as complex128 [N, N, N/2, Nr]: xi_x, xi_y and eta in FFT order, xi_z in [0, N/2)."""
    x = _f64(xyz).reshape(-1, 3)
    if q is not None:
        x = rotate(x, q)
    rr = -_f64(r) if mirror else _f64(r)
    m = _fft_modes(N).astype(np.float64)
    e = _fft_modes(Nr).astype(np.float64)
    Ex = np.exp(-2j * np.pi * np.outer(m, x[:, 0]) / period)
    Ey = np.exp(-2j * np.pi * np.outer(m, x[:, 1]) / period)
    Ez = np.exp(-2j * np.pi * np.outer(np.arange(N // 2), x[:, 2]) / period)
    Er = np.exp(-2j * np.pi * np.outer(e, rr) / period_r)
    E1 = (Ex[:, None, :] * Ey[None, :, :]).reshape(N * N, -1)
    E2 = (Ez[:, None, :] * Er[None, :, :]).reshape((N // 2) * Nr, -1)
    return (E1 @ E2.T).reshape(N, N, N // 2, Nr)


def cone_ft(k, alpha, L, nodes=64):
    """f^_D0 = int_0^L h^(s, k) exp(i alpha s) ds for arrays k (angular wavenumber) and alpha,
    by Gauss-Legendre quadrature (numpy's nodes) in FP64; broadcasts."""
    k, alpha = np.broadcast_arrays(_f64(k), _f64(alpha))
    xg, wg = np.polynomial.legendre.leggauss(nodes)
    s = 0.5 * L * (xg + 1.0)
    w = 0.5 * L * wg
    out = np.zeros(k.shape, dtype=np.complex128)
    for sj, wj in zip(s, w):  # one node at a time (bounded memory at large N)
        out += wj * ball_ft(np.full(k.shape, sj), k) * np.exp(1j * alpha * sj)
    return out


def lifted_corr_spectrum(A, B, q, N, Nr, L, period=2.0, period_r=0.4):
    """g^(xi, eta) [N, N, N/2, Nr]; A and B are (xyz, r) pairs; lower-edge modes zeroed."""
    ra = lifted_spectrum(A[0], A[1], N, Nr, period, period_r)
    rb = lifted_spectrum(B[0], B[1], N, Nr, period, period_r, q=q, mirror=True)
    m = _fft_modes(N).astype(np.float64)
    mz = np.arange(N // 2, dtype=np.float64)
    e = _fft_modes(Nr).astype(np.float64)
    q2 = m[:, None, None] ** 2 + m[None, :, None] ** 2 + mz[None, None, :] ** 2
    k = 2.0 * np.pi * np.sqrt(q2) / period
    f = cone_ft(k[..., None], 2.0 * np.pi * e[None, None, None, :] / period_r, L)
    g = ra * np.conj(rb) * f * f
    g[N // 2, :, :, :] = 0.0
    g[:, N // 2, :, :] = 0.0
    g[:, :, :, Nr // 2] = 0.0
    return g


def lifted_slices(ghat, slices, period=2.0, period_r=0.4):
    """g(t_k, r_s) on the N^3 translation grid for each r_s: [len(slices), N, N, N]."""
    N, Nr = ghat.shape[0], ghat.shape[3]
    e = _fft_modes(Nr).astype(np.float64)
    out = []
    for rs in slices:
        G = np.zeros((N, N, N // 2 + 1), dtype=np.complex128)
        G[:, :, : N // 2] = (ghat * np.exp(2j * np.pi * e * float(rs) / period_r)).sum(axis=-1) / period_r
        out.append(inverse_grid(G, period))
    return np.stack(out)
