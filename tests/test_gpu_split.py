"""Split-precision path (precision = 1): the radix-8 stages of the forward
transforms run as BF16 hi+lo DFT matmuls on the tensor cores with FP32
accumulation.  Its error against the FP64 oracle is stated next to the
all-FP32 path's; the bar for the split path is rel-L2 <= 2e-3."""
import numpy as np
import pytest

import oracle as O
from paper_1711_05075_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL, SPLIT_TOL = 1e-5, 2e-3


@pytest.fixture(scope="module")
def bc():
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    torch.cuda.set_device(0)
    import paper_1711_05075_gb300 as m
    return m


def f32(S):
    return synth.Shape(S.xyz.astype(np.float32).astype(np.float64), S.level, S.radii)


def run(bc, A, B, q, N, W, precision):
    ctx = bc.Context(N, W, A.radii, precision=precision)
    sa, sb = ctx.shape(A.xyz, A.level), ctx.shape(B.xyz, B.level)
    g = ctx.correlate(sa, sb, np.asarray(q, np.float32))
    ctx.sync()
    out = g.double().cpu().numpy()
    ctx.close()
    return out


def errs(got, ref):
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref)), float(np.abs(got - ref).max())


def test_split_precision_small_full_grid(bc):
    wl = synth.small_pair(8)
    q = synth.shoemake_quaternions(synth.SplitMix64(31), 2).astype(np.float32)
    g32 = run(bc, wl.A, wl.B, q, wl.N, wl.W, 0)
    gsp = run(bc, wl.A, wl.B, q, wl.N, wl.W, 1)
    for r in range(2):
        ref = O.band_limited_corr(f32(wl.A), f32(wl.B), q[r].astype(np.float64), wl.N)
        e32, esp = errs(g32[r], ref), errs(gsp[r], ref)
        print(f"N=32 rot {r}: FP32 rel-L2 {e32[0]:.2e} max-abs {e32[1]:.2e} | split BF16 rel-L2 {esp[0]:.2e} max-abs {esp[1]:.2e}")
        assert e32[0] <= FP32_TOL and esp[0] <= SPLIT_TOL


def test_split_precision_scale_pair_N256_sampled(bc):
    # 20,000 + 20,000 balls, L = 4, N = 256 (512^3 oversampled), W = 8; 4,096 sampled t.
    wl = synth.scale_pair(0, N=256, W=8)
    q = wl.quats.astype(np.float32)
    g32 = run(bc, wl.A, wl.B, q, wl.N, wl.W, 0)[0].reshape(-1)
    gsp = run(bc, wl.A, wl.B, q, wl.N, wl.W, 1)[0].reshape(-1)
    idx = synth.translation_sample(wl.N, 4096, seed=0)
    ghat = O.band_limited_spectrum(f32(wl.A), f32(wl.B), q[0].astype(np.float64), wl.N)
    ref = O.inverse_at(ghat, O.grid_points(wl.N, idx=idx))
    e32, esp = errs(g32[idx], ref), errs(gsp[idx], ref)
    print(f"N=256 20k+20k: FP32 rel-L2 {e32[0]:.2e} max-abs {e32[1]:.2e} | split BF16 rel-L2 {esp[0]:.2e} "
          f"max-abs {esp[1]:.2e} (|ref| max {np.abs(ref).max():.3e})")
    assert e32[0] <= FP32_TOL and esp[0] <= SPLIT_TOL


@pytest.mark.parametrize("N", [64, 96, 128])
def test_split_precision_each_N_sampled(bc, N):
    # 2,000 + 2,000 balls (L = 4), W = 8, a random rotation; 4,096 sampled t.  The
    # split passes use the radix schedules with radix-8 stages (128 = 8.16,
    # 192 = 3.8.8, 256 = 4.8.8); both transforms of every pass are compared.
    wl = synth.scale_pair(0, N=N, W=8, n=2000)
    q = synth.shoemake_quaternions(synth.SplitMix64(40 + N), 1).astype(np.float32)
    g32 = run(bc, wl.A, wl.B, q, N, wl.W, 0)[0].reshape(-1)
    gsp = run(bc, wl.A, wl.B, q, N, wl.W, 1)[0].reshape(-1)
    idx = synth.translation_sample(N, 4096, seed=1)
    ghat = O.band_limited_spectrum(f32(wl.A), f32(wl.B), q[0].astype(np.float64), N)
    ref = O.inverse_at(ghat, O.grid_points(N, idx=idx))
    e32, esp = errs(g32[idx], ref), errs(gsp[idx], ref)
    print(f"N={N} 2k+2k: FP32 rel-L2 {e32[0]:.2e} max-abs {e32[1]:.2e} | split BF16 rel-L2 {esp[0]:.2e} "
          f"max-abs {esp[1]:.2e} (|ref| max {np.abs(ref).max():.3e})")
    assert e32[0] <= FP32_TOL and esp[0] <= SPLIT_TOL
    # the split passes differ from FP32 by their BF16 roundings, not by a different transform
    assert errs(gsp[idx], g32[idx])[0] <= SPLIT_TOL
