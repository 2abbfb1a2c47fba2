"""GB300 (sm_103a) ball-union correlation: Python binding of libballcorr.so.

The binding only marshals arguments: every step of the correlation runs in the
library's CUDA kernels.  PyTorch supplies device memory and streams.  There is
no CPU fallback: if the library is missing or cannot load, `lib()` raises.

Functions named bc_* mirror the C ABI in include/ballcorr.h one to one; the
`Context` / `Shape` classes wrap them for convenience.
"""
from __future__ import annotations

import ctypes
import math
import os
import weakref

import numpy as np

from . import build as _build

_lib = None

BC_STATUS = {0: "BC_OK", 1: "BC_ERR_ARG", 2: "BC_ERR_OOM", 3: "BC_ERR_CUDA", 4: "BC_ERR_TIMEOUT",
             5: "BC_ERR_UNSUPPORTED", 6: "BC_ERR_INTERNAL"}
BC_MAX_LEVELS = 8


BC_NUM_STAGES = 7


class bc_profile(ctypes.Structure):
    _fields_ = [("calls", ctypes.c_int), ("launches", ctypes.c_longlong), ("ms", ctypes.c_double * BC_NUM_STAGES),
                ("bytes", ctypes.c_double * BC_NUM_STAGES)]


class bc_tuning(ctypes.Structure):
    _fields_ = [("spread", ctypes.c_int), ("sweep_batch", ctypes.c_int), ("graphs", ctypes.c_int),
                ("fft_schedule", ctypes.c_int), ("z_transform", ctypes.c_int), ("persistent", ctypes.c_int),
                ("overlap", ctypes.c_int)]


class bc_lift_params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("Nr", ctypes.c_int), ("L", ctypes.c_double), ("period", ctypes.c_double),
                ("period_r", ctypes.c_double), ("contraction", ctypes.c_int)]


class BallCorrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{BC_STATUS.get(status, status)}: {msg}")
        self.status = status


class bc_params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("sigma", ctypes.c_int), ("W", ctypes.c_int), ("beta", ctypes.c_double),
                ("period", ctypes.c_double), ("level_count", ctypes.c_int),
                ("level_radii", ctypes.POINTER(ctypes.c_double)), ("precision", ctypes.c_int)]


def library_path() -> str:
    return _build.LIB


def lib():
    """Loads libballcorr.so (building it first if the sources are newer)."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libballcorr.so not found at {path}")
        L = ctypes.CDLL(path)
        vp, i, st = ctypes.c_void_p, ctypes.c_int, ctypes.c_int
        L.bc_create.argtypes = [ctypes.POINTER(bc_params), vp, ctypes.POINTER(vp)]
        L.bc_destroy.argtypes = [vp]
        L.bc_shape_create.argtypes = [vp, vp, vp, i, i, ctypes.POINTER(vp)]
        L.bc_shapes_create.argtypes = [vp, i, vp, vp, vp, i, vp]
        L.bc_shape_destroy.argtypes = [vp]
        L.bc_correlate.argtypes = [vp, vp, vp, vp, i, vp, i]
        L.bc_sync.argtypes = [vp]
        L.bc_sweep.argtypes = [vp, vp, vp, vp, i, i, vp, vp, i]
        L.bc_sweep.restype = st
        L.bc_pairs.argtypes = [vp, vp, vp, vp, i, vp, vp, vp, i]
        L.bc_pairs.restype = st
        L.bc_shape_moments.argtypes = [vp, vp, vp]
        L.bc_shape_moments_rot.argtypes = [vp, vp, vp, i, vp]
        L.bc_mlp_features_rows.argtypes = [vp, vp, i, vp, vp, vp]
        L.bc_mlp_set_features.argtypes = [vp, i]
        L.bc_mlp_rotated_moments.argtypes = [vp]
        L.bc_mlp_rotated_moments.restype = i
        L.bc_mlp_param_count.argtypes = [i]
        L.bc_mlp_param_count.restype = ctypes.c_longlong
        L.bc_mlp_create.argtypes = [vp, i, vp, ctypes.POINTER(vp)]
        L.bc_mlp_destroy.argtypes = [vp]
        L.bc_mlp_features.argtypes = [vp, vp, i, vp, vp, vp]
        L.bc_mlp_predict.argtypes = [vp, vp, i, vp]
        L.bc_mlp_grads.argtypes = [vp, vp, vp, i, vp, vp]
        L.bc_mlp_train_step.argtypes = [vp, vp, vp, i, ctypes.c_float, vp]
        L.bc_mlp_train.argtypes = [vp, vp, vp, i, i, i, ctypes.c_float, ctypes.c_ulonglong, vp]
        L.bc_mlp_state.argtypes = [vp, vp, vp, vp, ctypes.POINTER(ctypes.c_longlong), i]
        L.bc_learned_sweep.argtypes = [vp, vp, vp, vp, vp, i, i, vp, vp, vp, vp]
        L.bc_learned_sweep_avg.argtypes = [vp, vp, vp, vp, vp, i, i, vp, i, vp, vp, vp, vp]
        L.bc_learned_sweep_cascade.argtypes = [vp, vp, vp, vp, vp, i, i, vp, i, i, vp, vp, vp, vp]
        L.bc_learned_sweep_coarse.argtypes = [vp, vp, vp, vp, vp, i, i, vp, i, i, vp, vp, vp, i, vp, vp, vp, vp]
        L.bc_topk.argtypes = [vp, vp, i, i, vp]
        L.bc_sweep_plan.argtypes = [vp, vp, vp, vp, i, i, vp, vp, ctypes.POINTER(vp)]
        L.bc_plan_run.argtypes = [vp]
        L.bc_plan_destroy.argtypes = [vp]
        for f in ("bc_sweep_plan", "bc_plan_run", "bc_plan_destroy"):
            getattr(L, f).restype = st
        L.bc_topk.restype = st
        for f in ("bc_shape_moments", "bc_shape_moments_rot", "bc_mlp_features_rows", "bc_mlp_set_features",
                  "bc_mlp_create", "bc_mlp_destroy", "bc_mlp_features", "bc_mlp_predict",
                  "bc_mlp_grads", "bc_mlp_train_step", "bc_mlp_train", "bc_mlp_state", "bc_learned_sweep",
                  "bc_learned_sweep_avg", "bc_learned_sweep_cascade", "bc_learned_sweep_coarse"):
            getattr(L, f).restype = st
        L.bc_selftest_wait.argtypes = [vp]
        for f in ("bc_create", "bc_destroy", "bc_shape_create", "bc_shapes_create", "bc_shape_destroy", "bc_correlate",
                  "bc_sync", "bc_selftest_wait"):
            getattr(L, f).restype = st
        L.bc_last_error.restype = ctypes.c_char_p
        L.bc_last_error.argtypes = []
        L.bc_version.restype = ctypes.c_char_p
        L.bc_version.argtypes = []
        L.bc_profile_begin.argtypes = [vp, i]
        L.bc_profile_begin.restype = st
        L.bc_profile_end.argtypes = [vp, ctypes.POINTER(bc_profile)]
        L.bc_profile_end.restype = st
        L.bc_stage_name.argtypes = [i]
        L.bc_stage_name.restype = ctypes.c_char_p
        L.bc_correlate_noalloc.argtypes = [ctypes.POINTER(bc_params), vp, vp, i, vp, vp, i, vp, vp, vp]
        L.bc_correlate_noalloc.restype = st
        L.bc_get_tuning.argtypes = [vp, ctypes.POINTER(bc_tuning)]
        L.bc_set_tuning.argtypes = [vp, ctypes.POINTER(bc_tuning)]
        L.bc_autotune.argtypes = [vp, vp, vp, i, ctypes.POINTER(bc_tuning)]
        for f in ("bc_get_tuning", "bc_set_tuning", "bc_autotune"):
            getattr(L, f).restype = st
        d = ctypes.c_double
        L.bc_score.argtypes = [vp, vp, vp, vp, i, d, d, vp, i]
        L.bc_score_sweep.argtypes = [vp, vp, vp, vp, i, i, d, d, vp, vp, i]
        L.bc_score.restype = st
        L.bc_score_sweep.restype = st
        L.bc_query_create.argtypes = [vp, vp, vp, vp, i, ctypes.POINTER(vp)]
        L.bc_query_eval.argtypes = [vp, vp, i, vp, i]
        L.bc_query_destroy.argtypes = [vp]
        for f in ("bc_query_create", "bc_query_eval", "bc_query_destroy"):
            getattr(L, f).restype = st
        L.bc_lift_create.argtypes = [ctypes.POINTER(bc_lift_params), vp, ctypes.POINTER(vp)]
        L.bc_lift_correlate.argtypes = [vp, vp, i, vp, i, vp, vp, i, vp, i]
        L.bc_lift_destroy.argtypes = [vp]
        for f in ("bc_lift_create", "bc_lift_correlate", "bc_lift_destroy"):
            getattr(L, f).restype = st
        _lib = L
    return _lib


def _check(status):
    if status != 0:
        raise BallCorrError(status, lib().bc_last_error().decode())


def _ptr(x):
    """Raw address of a torch tensor or numpy array (no copies are made here)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    return x.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------- C ABI mirror
def bc_create(N, W, radii, period=2.0, beta=0.0, sigma=2, precision=0, stream=None):
    radii = np.ascontiguousarray(radii, dtype=np.float64)
    p = bc_params(int(N), int(sigma), int(W), float(beta), float(period), int(radii.size),
                  radii.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(precision))
    h = ctypes.c_void_p()
    s = None if stream is None else ctypes.c_void_p(stream)
    _check(lib().bc_create(ctypes.byref(p), s, ctypes.byref(h)))
    return h


def bc_destroy(ctx):
    _check(lib().bc_destroy(ctx))


def bc_shape_create(ctx, xyz, level, n, on_device):
    h = ctypes.c_void_p()
    _check(lib().bc_shape_create(ctx, _ptr(xyz), _ptr(level), int(n), int(on_device), ctypes.byref(h)))
    return h


def bc_shapes_create(ctx, xyzs, levels, ns, on_device):
    """Several shapes with one stream synchronisation; returns their handles."""
    count = len(ns)
    px = (ctypes.c_void_p * max(count, 1))(*[_ptr(x) for x in xyzs])
    pl = (ctypes.c_void_p * max(count, 1))(*[_ptr(l) for l in levels])
    pn = (ctypes.c_int * max(count, 1))(*[int(n) for n in ns])
    hs = (ctypes.c_void_p * max(count, 1))()
    _check(lib().bc_shapes_create(ctx, int(count), px, pl, pn, int(on_device), hs))
    return [ctypes.c_void_p(hs[i]) for i in range(count)]


def bc_shape_destroy(shape):
    _check(lib().bc_shape_destroy(shape))


def bc_correlate(ctx, A, B, quats, k, out, out_on_device):
    _check(lib().bc_correlate(ctx, A, B, _ptr(quats), int(k), _ptr(out), int(out_on_device)))


def bc_sweep(ctx, A, B, quats, k, batch, peak, argmax, out_on_device):
    _check(lib().bc_sweep(ctx, A, B, _ptr(quats), int(k), int(batch), _ptr(peak), _ptr(argmax), int(out_on_device)))


def bc_pairs(ctx, As, Bs, quats, npairs, out, peak, argmax, on_device):
    """As, Bs: sequences of shape handles (marshalled into C arrays of pointers)."""
    arrA = (ctypes.c_void_p * npairs)(*[h.value for h in As])
    arrB = (ctypes.c_void_p * npairs)(*[h.value for h in Bs])
    _check(lib().bc_pairs(ctx, arrA, arrB, _ptr(quats), int(npairs), _ptr(out), _ptr(peak), _ptr(argmax),
                          int(on_device)))


def bc_shape_moments(ctx, shape, out):
    _check(lib().bc_shape_moments(ctx, shape, _ptr(out)))


def bc_shape_moments_rot(ctx, shape, quats, n, out):
    _check(lib().bc_shape_moments_rot(ctx, shape, _ptr(quats), int(n), _ptr(out)))


def bc_mlp_param_count(hidden):
    return int(lib().bc_mlp_param_count(int(hidden)))


def bc_mlp_create(ctx, hidden, init):
    h = ctypes.c_void_p()
    init = np.ascontiguousarray(init, dtype=np.float32)
    _check(lib().bc_mlp_create(ctx, int(hidden), _ptr(init), ctypes.byref(h)))
    return h


def bc_mlp_destroy(net):
    _check(lib().bc_mlp_destroy(net))


def bc_mlp_features(net, quats, n, fa, fb, X):
    _check(lib().bc_mlp_features(net, _ptr(quats), int(n), _ptr(fa), _ptr(fb), _ptr(X)))


def bc_mlp_features_rows(net, quats, n, fa, fb_rows, X):
    _check(lib().bc_mlp_features_rows(net, _ptr(quats), int(n), _ptr(fa), _ptr(fb_rows), _ptr(X)))


def bc_mlp_set_features(net, rotated_moments):
    _check(lib().bc_mlp_set_features(net, int(rotated_moments)))


def bc_mlp_rotated_moments(net):
    return int(lib().bc_mlp_rotated_moments(net))


def bc_mlp_predict(net, X, n, y):
    _check(lib().bc_mlp_predict(net, _ptr(X), int(n), _ptr(y)))


def bc_mlp_grads(net, X, t, n, grads, loss):
    _check(lib().bc_mlp_grads(net, _ptr(X), _ptr(t), int(n), _ptr(grads), _ptr(loss)))


def bc_mlp_train_step(net, X, t, n, lr, loss):
    _check(lib().bc_mlp_train_step(net, _ptr(X), _ptr(t), int(n), float(lr), _ptr(loss)))


def bc_mlp_train(net, X, t, n, batch, epochs, lr, seed, loss):
    _check(lib().bc_mlp_train(net, _ptr(X), _ptr(t), int(n), int(batch), int(epochs), float(lr), int(seed), _ptr(loss)))


def bc_mlp_state(net, params, m, v, step, get):
    """step: a ctypes.c_longlong (read or written in place)."""
    _check(lib().bc_mlp_state(net, _ptr(params), _ptr(m), _ptr(v), ctypes.byref(step), int(get)))


def bc_learned_sweep(ctx, net, A, B, quats, n, topk, idx, peak, argmax, scores):
    _check(lib().bc_learned_sweep(ctx, net, A, B, _ptr(quats), int(n), int(topk), _ptr(idx), _ptr(peak),
                                  _ptr(argmax), _ptr(scores)))


def bc_sweep_plan(ctx, A, B, quats, k, batch, peak, argmax):
    h = ctypes.c_void_p()
    _check(lib().bc_sweep_plan(ctx, A, B, _ptr(quats), int(k), int(batch), _ptr(peak), _ptr(argmax), ctypes.byref(h)))
    return h


def bc_plan_run(plan):
    _check(lib().bc_plan_run(plan))


def bc_plan_destroy(plan):
    _check(lib().bc_plan_destroy(plan))


def bc_topk(ctx, scores, n, k, idx):
    _check(lib().bc_topk(ctx, _ptr(scores), int(n), int(k), _ptr(idx)))


def bc_sync(ctx):
    _check(lib().bc_sync(ctx))


def bc_selftest_wait(ctx):
    """Status of the bounded-wait self-test: BC_ERR_TIMEOUT (4) when the timeout path works."""
    return int(lib().bc_selftest_wait(ctx))


def bc_version() -> str:
    return lib().bc_version().decode()


BC_NOALLOC_MAX_N = 32
BC_NOALLOC_MAX_LEVELS = 2
BC_NOALLOC_MAX_KNOTS = 8192


def bc_correlate_noalloc(N, W, radii, xyzA, levelA, nA, xyzB, levelB, nB, quat, out, period=2.0, beta=0.0,
                         stream=None):
    """The allocation-free correlation (see include/ballcorr.h): device inputs and output,
    scratch in the library's static device array."""
    radii = np.ascontiguousarray(radii, dtype=np.float64)
    p = bc_params(int(N), 2, int(W), float(beta), float(period), int(radii.size),
                  radii.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0)
    q = np.ascontiguousarray(np.asarray(quat, dtype=np.float32).reshape(4))
    s = None if stream is None else ctypes.c_void_p(stream)
    _check(lib().bc_correlate_noalloc(ctypes.byref(p), _ptr(xyzA), _ptr(levelA), int(nA), _ptr(xyzB), _ptr(levelB),
                                      int(nB), _ptr(q), _ptr(out), s))


def bc_profile_begin(ctx, max_calls):
    _check(lib().bc_profile_begin(ctx, int(max_calls)))


def bc_profile_end(ctx):
    """Returns {calls, launches, stages: [{name, ms, bytes}]} for the profiled calls."""
    p = bc_profile()
    _check(lib().bc_profile_end(ctx, ctypes.byref(p)))
    return {"calls": p.calls, "launches": p.launches,
            "stages": [{"name": lib().bc_stage_name(s).decode(), "ms": p.ms[s], "bytes": p.bytes[s]}
                       for s in range(BC_NUM_STAGES)]}


def bc_score(ctx, A, B, quats, k, r0, lam, out, out_on_device):
    _check(lib().bc_score(ctx, A, B, _ptr(quats), int(k), float(r0), float(lam), _ptr(out), int(out_on_device)))


def bc_score_sweep(ctx, A, B, quats, k, batch, r0, lam, peak, argmax, out_on_device):
    _check(lib().bc_score_sweep(ctx, A, B, _ptr(quats), int(k), int(batch), float(r0), float(lam), _ptr(peak),
                                _ptr(argmax), int(out_on_device)))


def bc_query_create(ctx, A, B, quat, mprime):
    q = np.ascontiguousarray(np.asarray(quat, dtype=np.float32).reshape(4))
    h = ctypes.c_void_p()
    _check(lib().bc_query_create(ctx, A, B, _ptr(q), int(mprime), ctypes.byref(h)))
    return h


def bc_query_eval(q, t, npts, g, on_device):
    _check(lib().bc_query_eval(q, _ptr(t), int(npts), _ptr(g), int(on_device)))


def bc_query_destroy(q):
    _check(lib().bc_query_destroy(q))


def _tuning_dict(t):
    return {"spread": t.spread, "sweep_batch": t.sweep_batch, "graphs": t.graphs, "fft_schedule": t.fft_schedule,
            "z_transform": t.z_transform, "persistent": t.persistent, "overlap": t.overlap}


def bc_get_tuning(ctx):
    t = bc_tuning()
    _check(lib().bc_get_tuning(ctx, ctypes.byref(t)))
    return _tuning_dict(t)


def bc_set_tuning(ctx, spread, sweep_batch, graphs=1, fft_schedule=0, z_transform=0, persistent=1, overlap=1):
    t = bc_tuning(int(spread), int(sweep_batch), int(graphs), int(fft_schedule), int(z_transform), int(persistent),
                  int(overlap))
    _check(lib().bc_set_tuning(ctx, ctypes.byref(t)))


def bc_autotune(ctx, A, B, rotations=0):
    t = bc_tuning()
    _check(lib().bc_autotune(ctx, A, B, int(rotations), ctypes.byref(t)))
    return _tuning_dict(t)


# ---------------------------------------------------------------- convenience
def default_beta(W, sigma=2):
    return math.pi * math.sqrt((W / sigma) ** 2 * (sigma - 0.5) ** 2 - 0.8)


class Context:
    """Correlation context on the current CUDA device and a torch stream."""

    def __init__(self, N, W, radii, period=2.0, beta=0.0, stream=None, precision=0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        self.N, self.W, self.period = int(N), int(W), float(period)
        self.radii = tuple(float(r) for r in radii)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle = None
        self.handle = bc_create(N, W, radii, period, beta, precision=precision, stream=self.stream.cuda_stream)
        self._shapes = weakref.WeakSet()
        self._nets = weakref.WeakSet()
        self._queries = weakref.WeakSet()

    def shape(self, xyz, level):
        s = Shape(self, xyz, level)
        self._shapes.add(s)
        return s

    def shapes(self, pairs):
        """Several shapes [(xyz, level), ...], all host or all CUDA arrays, uploaded
        with one stream synchronisation (bc_shapes_create)."""
        arrs = [Shape._arrays(x, l) for x, l in pairs]
        devs = {d for _, _, d in arrs}
        if len(devs) > 1:
            raise ValueError("shapes: mix of host and device arrays")
        hs = bc_shapes_create(self.handle, [a[0] for a in arrs], [a[1] for a in arrs], [a[0].shape[0] for a in arrs],
                              devs.pop() if arrs else 0)
        out = []
        for (x, l, d), h in zip(arrs, hs):
            s = Shape.__new__(Shape)
            s.ctx, s.n, s.handle = self, x.shape[0], h
            self._shapes.add(s)
            out.append(s)
        return out

    def correlate(self, A, B, quats, out=None):
        """g for each rotation: a (k, N, N, N) float32 CUDA tensor (or `out`)."""
        import torch
        q = np.ascontiguousarray(np.asarray(quats, dtype=np.float32).reshape(-1, 4))
        k = q.shape[0]
        if out is None:
            out = torch.empty((k, self.N, self.N, self.N), dtype=torch.float32, device="cuda")
        assert out.is_cuda and out.is_contiguous() and out.dtype == torch.float32 and out.numel() == k * self.N ** 3
        bc_correlate(self.handle, A.handle, B.handle, q, k, out, 1)
        return out

    def sweep(self, A, B, quats, batch=0):
        """Peak value and lowest argmax index over the translation grid per rotation:
        (float32 [k], int32 [k]) CUDA tensors."""
        import torch
        q = np.ascontiguousarray(np.asarray(quats, dtype=np.float32).reshape(-1, 4))
        k = q.shape[0]
        peak = torch.empty(k, dtype=torch.float32, device="cuda")
        arg = torch.empty(k, dtype=torch.int32, device="cuda")
        bc_sweep(self.handle, A.handle, B.handle, q, k, batch, peak, arg, 1)
        return peak, arg

    def score(self, A, B, quats, r0, lam, out=None):
        """Complementarity score G (Sec. 4.2) for each rotation: (k, N, N, N) float32 CUDA tensor."""
        import torch
        q = np.ascontiguousarray(np.asarray(quats, dtype=np.float32).reshape(-1, 4))
        k = q.shape[0]
        if out is None:
            out = torch.empty((k, self.N, self.N, self.N), dtype=torch.float32, device="cuda")
        assert out.is_cuda and out.is_contiguous() and out.dtype == torch.float32 and out.numel() == k * self.N ** 3
        bc_score(self.handle, A.handle, B.handle, q, k, r0, lam, out, 1)
        return out

    def score_sweep(self, A, B, quats, r0, lam, batch=0):
        """Best score over the translation grid and its lowest index per rotation (CUDA tensors)."""
        import torch
        q = np.ascontiguousarray(np.asarray(quats, dtype=np.float32).reshape(-1, 4))
        k = q.shape[0]
        peak = torch.empty(k, dtype=torch.float32, device="cuda")
        arg = torch.empty(k, dtype=torch.int32, device="cuda")
        bc_score_sweep(self.handle, A.handle, B.handle, q, k, batch, r0, lam, peak, arg, 1)
        return peak, arg

    def query(self, A, B, quat, mprime):
        """Truncated single-configuration queries of g for one rotation (see Query)."""
        q = Query(self, A, B, quat, mprime)
        self._queries.add(q)
        return q

    def pairs(self, As, Bs, quats, grids=False, peaks=True):
        """Ragged batch of independent pairs; returns (grids or None, peak or None, argmax or None)."""
        import torch
        q = np.ascontiguousarray(np.asarray(quats, dtype=np.float32).reshape(-1, 4))
        n = q.shape[0]
        out = torch.empty((n, self.N, self.N, self.N), dtype=torch.float32, device="cuda") if grids else None
        peak = torch.empty(n, dtype=torch.float32, device="cuda") if peaks else None
        arg = torch.empty(n, dtype=torch.int32, device="cuda") if peaks else None
        bc_pairs(self.handle, [a.handle for a in As], [b.handle for b in Bs], q, n, out, peak, arg, 1)
        return out, peak, arg

    def correlate_host(self, A, B, quats, out):
        """Same, writing into host memory `out` (numpy array or pinned tensor); synchronous."""
        q = np.ascontiguousarray(np.asarray(quats, dtype=np.float32).reshape(-1, 4))
        bc_correlate(self.handle, A.handle, B.handle, q, q.shape[0], out, 0)
        return out

    def sync(self):
        bc_sync(self.handle)

    def selftest_wait(self):
        """Runs bc_selftest_wait: 4 (BC_ERR_TIMEOUT, after about 2 s) when bounded device waits give up cleanly."""
        return bc_selftest_wait(self.handle)

    @property
    def tuning(self):
        """The context's implementation choices: {"spread", "sweep_batch", "graphs", "fft_schedule", "z_transform",
        "persistent", "overlap"}."""
        return bc_get_tuning(self.handle)

    def set_tuning(self, spread=None, sweep_batch=None, graphs=None, fft_schedule=None, z_transform=None,
                   persistent=None, overlap=None):
        t = self.tuning
        bc_set_tuning(self.handle, t["spread"] if spread is None else spread,
                      t["sweep_batch"] if sweep_batch is None else sweep_batch,
                      t["graphs"] if graphs is None else graphs,
                      t["fft_schedule"] if fft_schedule is None else fft_schedule,
                      t["z_transform"] if z_transform is None else z_transform,
                      t["persistent"] if persistent is None else persistent,
                      t["overlap"] if overlap is None else overlap)

    def autotune(self, A, B, rotations=0):
        """Times the candidates on these shapes and keeps the fastest (see bc_autotune)."""
        return bc_autotune(self.handle, A.handle, B.handle, rotations)

    def close(self):
        if self.handle is not None:
            for s in list(self._shapes):
                s.close()
            for net in list(self._nets):
                net.close()
            for q in list(self._queries):
                q.close()
            bc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MLP:
    """The learned rotation proposal (132 -> H -> H -> 1) on a context's device and stream."""

    def __init__(self, ctx: Context, hidden: int, init, rotated_moments=False):
        self.ctx, self.hidden = ctx, int(hidden)
        self.nparams = bc_mlp_param_count(hidden)
        init = np.ascontiguousarray(init, dtype=np.float32).reshape(-1)
        assert init.size == self.nparams
        self.handle = bc_mlp_create(ctx.handle, hidden, init)
        ctx._nets.add(self)
        if rotated_moments:
            bc_mlp_set_features(self.handle, 1)

    @property
    def rotated_moments(self):
        return bc_mlp_rotated_moments(self.handle) == 1

    def features(self, quats_dev, fa, fb):
        """Feature rows (n x 144): fb is one moment vector (64) for every row, or one per
        row (n x 64, e.g. moments_rot of the ligand)."""
        import torch
        n = quats_dev.shape[0]
        X = torch.empty((n, 144), dtype=torch.float32, device="cuda")
        if fb.dim() == 2:
            assert fb.shape == (n, 64) and fb.is_contiguous()
            bc_mlp_features_rows(self.handle, quats_dev, n, fa, fb, X)
        else:
            bc_mlp_features(self.handle, quats_dev, n, fa, fb, X)
        return X

    def predict(self, X):
        import torch
        y = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
        bc_mlp_predict(self.handle, X, X.shape[0], y)
        return y

    def grads(self, X, t):
        import torch
        g = torch.empty(self.nparams, dtype=torch.float32, device="cuda")
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        bc_mlp_grads(self.handle, X, t, X.shape[0], g, loss)
        return g, loss

    def train_step(self, X, t, lr, loss=None):
        bc_mlp_train_step(self.handle, X, t, X.shape[0], lr, loss)

    def train(self, X, t, epochs, batch, lr, seed=0, loss=None):
        """`epochs` passes of Adam steps over (X, t) in device-shuffled batches (bc_mlp_train)."""
        bc_mlp_train(self.handle, X, t, X.shape[0], batch, epochs, lr, seed, loss)

    def state(self):
        p = np.empty(self.nparams, np.float32)
        m = np.empty_like(p)
        v = np.empty_like(p)
        step = ctypes.c_longlong(0)
        bc_mlp_state(self.handle, p, m, v, step, 1)
        return {"params": p, "adam_m": m, "adam_v": v, "step": step.value}

    def load_state(self, st):
        step = ctypes.c_longlong(int(st["step"]))
        bc_mlp_state(self.handle, np.ascontiguousarray(st["params"], np.float32),
                     np.ascontiguousarray(st["adam_m"], np.float32), np.ascontiguousarray(st["adam_v"], np.float32),
                     step, 0)

    def close(self):
        if self.handle is not None:
            bc_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def moments(ctx: Context, shape) -> "torch.Tensor":
    import torch
    out = torch.empty(64, dtype=torch.float32, device="cuda")
    bc_shape_moments(ctx.handle, shape.handle, out)
    return out


def moments_rot(ctx: Context, shape, quats_dev) -> "torch.Tensor":
    """(n, 64) CUDA tensor: the moments of `shape` turned by each of the n device quaternions."""
    import torch
    q = quats_dev.contiguous().float()
    out = torch.empty((q.shape[0], 64), dtype=torch.float32, device="cuda")
    bc_shape_moments_rot(ctx.handle, shape.handle, q, q.shape[0], out)
    return out


def learned_sweep(ctx: Context, net: MLP, A, B, quats_dev, topk, orientations=None, keep=None, coarse=None):
    """(idx, peak, argmax, scores) CUDA tensors: network scores of all rotations, the topk
    best, and the correlation peaks of those.  With `orientations` (k x 4 host quaternions)
    the scores are averaged over the receptor turned by each of them
    (bc_learned_sweep_avg); with `keep` as well, only the best `keep` rotations of the
    one-view scores are scored again (bc_learned_sweep_cascade; scores are then the
    one-view scores).  With coarse = (cctx, Ac, Bc, coarse_keep) the network's best
    coarse_keep are correlated on the coarse context first and the topk best of those by
    their coarse peaks get full correlations (bc_learned_sweep_coarse; keep defaults to
    all rotations)."""
    import torch
    n = quats_dev.shape[0]
    idx = torch.empty(topk, dtype=torch.int32, device="cuda")
    peak = torch.empty(topk, dtype=torch.float32, device="cuda")
    arg = torch.empty(topk, dtype=torch.int32, device="cuda")
    scores = torch.empty(n, dtype=torch.float32, device="cuda")
    if coarse is not None:
        cctx, Ac, Bc, ckeep = coarse
        o = np.ascontiguousarray(np.asarray(orientations if orientations is not None else np.zeros((0, 4)),
                                            dtype=np.float32).reshape(-1, 4))
        _check(lib().bc_learned_sweep_coarse(ctx.handle, net.handle, A.handle, B.handle, _ptr(quats_dev), int(n),
                                             int(topk), _ptr(o), int(o.shape[0]), int(n if keep is None else keep),
                                             cctx.handle, Ac.handle, Bc.handle, int(ckeep), _ptr(idx), _ptr(peak),
                                             _ptr(arg), _ptr(scores)))
    elif keep is not None:
        o = np.ascontiguousarray(np.asarray(orientations if orientations is not None else np.zeros((0, 4)),
                                            dtype=np.float32).reshape(-1, 4))
        _check(lib().bc_learned_sweep_cascade(ctx.handle, net.handle, A.handle, B.handle, _ptr(quats_dev), int(n),
                                              int(topk), _ptr(o), int(o.shape[0]), int(keep), _ptr(idx), _ptr(peak),
                                              _ptr(arg), _ptr(scores)))
    elif orientations is None:
        bc_learned_sweep(ctx.handle, net.handle, A.handle, B.handle, quats_dev, n, topk, idx, peak, arg, scores)
    else:
        o = np.ascontiguousarray(np.asarray(orientations, dtype=np.float32).reshape(-1, 4))
        _check(lib().bc_learned_sweep_avg(ctx.handle, net.handle, A.handle, B.handle, _ptr(quats_dev), int(n),
                                          int(topk), _ptr(o), int(o.shape[0]), _ptr(idx), _ptr(peak), _ptr(arg),
                                          _ptr(scores)))
    return idx, peak, arg, scores


class Shape:
    """A union of balls uploaded to the device: xyz (n x 3) and level ids (n)."""

    def __init__(self, ctx: Context, xyz, level):
        self.ctx = ctx
        self.handle = None
        x, l, dev = Shape._arrays(xyz, level)
        self.n = x.shape[0]
        self.handle = bc_shape_create(ctx.handle, x, l, self.n, dev)

    @staticmethod
    def _arrays(xyz, level):
        """(xyz as contiguous n x 3 FP32, level as contiguous int32, on_device)."""
        if hasattr(xyz, "is_cuda") and xyz.is_cuda:
            import torch
            return xyz.to(torch.float32).reshape(-1, 3).contiguous(), level.to(torch.int32).reshape(-1).contiguous(), 1
        return (np.ascontiguousarray(np.asarray(xyz, dtype=np.float32).reshape(-1, 3)),
                np.ascontiguousarray(np.asarray(level, dtype=np.int32).reshape(-1)), 0)

    def close(self):
        if self.handle is not None:
            bc_shape_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Query:
    """g at arbitrary translations from the m' lowest modes of one configuration's spectrum."""

    def __init__(self, ctx: Context, A, B, quat, mprime: int):
        self.ctx = ctx
        self.mprime = int(mprime)
        self.handle = bc_query_create(ctx.handle, A.handle, B.handle, quat, mprime)

    def eval(self, t):
        """t: (n, 3) float32 CUDA tensor (asynchronous) or array-like (host, synchronous)."""
        import torch
        if isinstance(t, torch.Tensor) and t.is_cuda:
            t = t.contiguous().float()
            g = torch.empty(t.shape[0], dtype=torch.float32, device=t.device)
            bc_query_eval(self.handle, t, t.shape[0], g, 1)
            return g
        th = np.ascontiguousarray(np.asarray(t, dtype=np.float32).reshape(-1, 3))
        g = np.empty(th.shape[0], dtype=np.float32)
        bc_query_eval(self.handle, th, th.shape[0], g, 0)
        return g

    def close(self):
        if self.handle is not None:
            bc_query_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


LIFT_CONTRACTIONS = {"nufft": 3, "tcgen05": 2, "mma": 1, "cuda": 0}


def bc_lift_create(N, Nr, L, period=2.0, period_r=None, stream=None, contraction=None):
    """contraction: "nufft" (the 4D type-1 NUFFT, Nr >= 16), or the direct 4D NDFT as "tcgen05", "mma" (legacy
    mma.sync) or "cuda" (FP32 CUDA cores), or 3 / 2 / 1 / 0; None: "nufft" where Nr >= 16, else "tcgen05"."""
    if contraction is None:
        contraction = "nufft" if int(Nr) >= 16 else "tcgen05"
    c = LIFT_CONTRACTIONS[contraction] if isinstance(contraction, str) else int(contraction)
    p = bc_lift_params(int(N), int(Nr), float(L), float(period), float(4 * L if period_r is None else period_r), c)
    h = ctypes.c_void_p()
    _check(lib().bc_lift_create(ctypes.byref(p), None if stream is None else ctypes.c_void_p(stream), ctypes.byref(h)))
    return h


def bc_lift_correlate(lf, A, nA, B, nB, quat, slices, nslices, out, on_device):
    _check(lib().bc_lift_correlate(lf, _ptr(A), int(nA), _ptr(B), int(nB), _ptr(quat), _ptr(slices), int(nslices),
                                   _ptr(out), int(on_device)))


def bc_lift_destroy(lf):
    _check(lib().bc_lift_destroy(lf))


class Lift:
    """Lifted (4D) nonequiradius correlation (Sec. 3.2) on the current CUDA device and stream."""

    def __init__(self, N, Nr, L, period=2.0, period_r=None, stream=None, contraction=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        self.N, self.Nr, self.L = int(N), int(Nr), float(L)
        self.period = float(period)
        self.period_r = float(4 * L if period_r is None else period_r)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle = None
        self.handle = bc_lift_create(N, Nr, L, period, self.period_r, stream=self.stream.cuda_stream,
                                     contraction=contraction)

    def correlate(self, A, B, quat, slices=(0.0,)):
        """A, B: (n, 4) (x, y, z, r) float32 CUDA tensors or arrays; returns (len(slices), N, N, N) CUDA tensor."""
        import torch
        q = np.ascontiguousarray(np.asarray(quat, dtype=np.float32).reshape(4))
        sl = np.ascontiguousarray(np.asarray(slices, dtype=np.float32).reshape(-1))
        dev = lambda x: (x if isinstance(x, torch.Tensor) else torch.as_tensor(np.asarray(x, np.float32))).to(
            device="cuda", dtype=torch.float32).contiguous()
        Ad, Bd = dev(A), dev(B)
        out = torch.empty((sl.size, self.N, self.N, self.N), dtype=torch.float32, device="cuda")
        bc_lift_correlate(self.handle, Ad, Ad.shape[0], Bd, Bd.shape[0], q, sl, sl.size, out, 1)
        return out

    def correlate_host(self, A, B, quat, slices=(0.0,)):
        q = np.ascontiguousarray(np.asarray(quat, dtype=np.float32).reshape(4))
        sl = np.ascontiguousarray(np.asarray(slices, dtype=np.float32).reshape(-1))
        Ah = np.ascontiguousarray(np.asarray(A, dtype=np.float32).reshape(-1, 4))
        Bh = np.ascontiguousarray(np.asarray(B, dtype=np.float32).reshape(-1, 4))
        out = np.empty((sl.size, self.N, self.N, self.N), dtype=np.float32)
        bc_lift_correlate(self.handle, Ah, Ah.shape[0], Bh, Bh.shape[0], q, sl, sl.size, out, 0)
        return out

    def close(self):
        if self.handle is not None:
            bc_lift_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
