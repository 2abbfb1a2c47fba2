"""FP64 CPU oracle for the ball-union correlation (ctypes wrapper of oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg may import it; the product path never does.  It shares no
code with the CUDA path.  See oracle.c for the two layers and their citations.

Parity status: every function here is pinned by a CPU test against something
other than itself (closed forms, quadrature, Monte Carlo, library rotations,
invariants, and convergence of layer (b) to layer (a)); none is "parity unpinned".
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
