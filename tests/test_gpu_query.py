"""GPU truncated single-configuration queries (Sec. 4.1, Eq. (single)) against the FP64 oracle.

Off-grid translations drawn uniformly in [-1, 1)^3 (and a few outside the
period); bar rel-L2 <= 1e-5 over the query points.
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


def points(n, seed):
    t = np.random.default_rng(seed).uniform(-1.0, 1.0, (n, 3))
    t[:5] += np.array([2.0, -4.0, 6.0])  # whole periods away: same values
    return t.astype(np.float32)


@pytest.mark.parametrize("mprime", [1, 7, 500, 14896])  # 14896 = all modes at N = 32
def test_small_pair_queries(bc, mprime):
    wl = synth.small_pair(0)
    q = synth.shoemake_quaternions(synth.SplitMix64(21), 1).astype(np.float32)
    ctx = bc.Context(wl.N, wl.W, wl.radii)
    A, B = ctx.shape(wl.A.xyz, wl.A.level), ctx.shape(wl.B.xyz, wl.B.level)
    qu = ctx.query(A, B, q[0], mprime)
    t = points(300, mprime)
    got_host = qu.eval(t).astype(np.float64)
    got_dev = qu.eval(torch.tensor(t, device="cuda")).cpu().numpy().astype(np.float64)
    g = O.band_limited_spectrum(f32(wl.A), f32(wl.B), q[0].astype(np.float64), wl.N)
    m, w = O.query_modes(wl.N, mprime)
    ref = O.query_at(g, m, w, t.astype(np.float64))
    e = rel(got_host, ref)
    print(f"query N=32 m'={mprime}: rel-L2 {e:.3e}")
    assert e <= REL_TOL
    np.testing.assert_array_equal(got_host, got_dev)  # same kernel, same inputs
    if mprime == 14896:  # all modes: the band-limited correlation itself, on the grid too
        idx = np.arange(0, wl.N ** 3, 97)
        tg = O.grid_points(wl.N, idx=idx).astype(np.float32)
        full = ctx.correlate(A, B, q).cpu().numpy().reshape(-1)[idx]
        assert rel(qu.eval(tg).astype(np.float64), full.astype(np.float64)) < 2e-6
    qu.close(); A.close(); B.close(); ctx.close()


def test_scale_pair_queries(bc):
    wl = synth.scale_pair(0)
    ctx = bc.Context(wl.N, wl.W, wl.radii)
    A, B = ctx.shape(wl.A.xyz, wl.A.level), ctx.shape(wl.B.xyz, wl.B.level)
    qu = ctx.query(A, B, wl.quats[0], 4096)
    t = points(256, 3)
    got = qu.eval(t).astype(np.float64)
    g = O.band_limited_spectrum(f32(wl.A), f32(wl.B), wl.quats[0].astype(np.float32).astype(np.float64), wl.N)
    m, w = O.query_modes(wl.N, 4096)
    e = rel(got, O.query_at(g, m, w, t.astype(np.float64)))
    print(f"query 20k+20k N=128 m'=4096: rel-L2 {e:.3e}")
    assert e <= REL_TOL
    with pytest.raises(bc.BallCorrError):
        ctx.query(A, B, wl.quats[0], 0)
    with pytest.raises(bc.BallCorrError):
        ctx.query(A, B, wl.quats[0], (127 ** 3 + 1) // 2 + 1)
    qu.close(); A.close(); B.close(); ctx.close()


def test_query_outlives_nothing_after_context_close(bc):
    wl = synth.small_pair(1)
    ctx = bc.Context(wl.N, wl.W, wl.radii)
    A, B = ctx.shape(wl.A.xyz, wl.A.level), ctx.shape(wl.B.xyz, wl.B.level)
    qu = ctx.query(A, B, wl.quats[0], 10)
    h = qu.handle
    ctx.close()  # closes the query first
    assert qu.handle is None
    del h
