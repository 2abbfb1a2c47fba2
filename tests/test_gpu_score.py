"""GPU shape-complementarity score (Sec. 4.2, Eq. (score)) against the FP64 oracle.

Same inputs on both sides (knots and quaternions rounded once to FP32); bar
rel-L2 <= 1e-5 over the compared points, as for the correlation.
"""
import numpy as np
import pytest

import oracle as O
from paper_1711_05075_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_TOL = 1e-5


@pytest.fixture(scope="module")
def bc():
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    torch.cuda.set_device(0)
    import paper_1711_05075_gb300 as m
    return m


def f32(S):
    return synth.Shape(S.xyz.astype(np.float32).astype(np.float64), S.level, S.radii, S.name)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("r0,lam", [(0.03, 2.0), (0.06, 0.5), (0.0, 3.0)])
def test_small_pair_full_grid(bc, r0, lam):
    wl = synth.small_pair(0)
    q = synth.shoemake_quaternions(synth.SplitMix64(12), 2).astype(np.float32)
    ctx = bc.Context(wl.N, wl.W, wl.radii)
    A, B = ctx.shape(wl.A.xyz, wl.A.level), ctx.shape(wl.B.xyz, wl.B.level)
    got = ctx.score(A, B, q, r0, lam).double().cpu().numpy()
    for r in range(2):
        ref = O.band_limited_score(f32(wl.A), f32(wl.B), q[r].astype(np.float64), wl.N, r0, lam)
        e = rel(got[r], ref)
        print(f"score r0={r0} lam={lam} rot {r}: rel-L2 {e:.3e} max-abs {np.abs(got[r] - ref).max():.3e}")
        assert e <= REL_TOL
    A.close(); B.close(); ctx.close()


def test_scale_pair_sampled(bc):
    wl = synth.scale_pair(0)
    r0, lam = 0.02, 2.0
    ctx = bc.Context(wl.N, wl.W, wl.radii)
    A, B = ctx.shape(wl.A.xyz, wl.A.level), ctx.shape(wl.B.xyz, wl.B.level)
    got = ctx.score(A, B, wl.quats, r0, lam).double().cpu().numpy()[0].reshape(-1)
    idx = synth.translation_sample(wl.N, 4096, seed=0)
    ref = O.band_limited_score(f32(wl.A), f32(wl.B), wl.quats[0].astype(np.float32).astype(np.float64), wl.N, r0,
                               lam, idx=idx)
    e = rel(got[idx], ref)
    print(f"score 20k+20k N=128, 4096 sampled t: rel-L2 {e:.3e}")
    assert e <= REL_TOL
    A.close(); B.close(); ctx.close()


def test_score_sweep_peaks(bc):
    wl = synth.small_pair(3)
    r0, lam = 0.03, 2.0
    q = synth.shoemake_quaternions(synth.SplitMix64(13), 5).astype(np.float32)
    ctx = bc.Context(wl.N, wl.W, wl.radii)
    A, B = ctx.shape(wl.A.xyz, wl.A.level), ctx.shape(wl.B.xyz, wl.B.level)
    peak, arg = ctx.score_sweep(A, B, q, r0, lam, batch=2)
    peak, arg = peak.cpu().numpy(), arg.cpu().numpy()
    grids = ctx.score(A, B, q, r0, lam).cpu().numpy().reshape(5, -1)
    for r in range(5):
        ref = O.band_limited_score(f32(wl.A), f32(wl.B), q[r].astype(np.float64), wl.N, r0, lam).reshape(-1)
        assert abs(peak[r] - ref.max()) <= 1e-5 * np.abs(ref).max()
        assert abs(ref[arg[r]] - ref.max()) <= 1e-5 * np.abs(ref).max()  # a valid maximiser
        # the full grid of the same kernels (spreading sums in another order): same peak to rounding
        assert abs(peak[r] - grids[r].max()) <= 1e-6 * np.abs(grids[r]).max()
    with pytest.raises(bc.BallCorrError):
        ctx.score(A, B, q, -0.1, lam)
    with pytest.raises(bc.BallCorrError):
        ctx.score(A, B, q, 0.1, float("nan"))
    A.close(); B.close(); ctx.close()
