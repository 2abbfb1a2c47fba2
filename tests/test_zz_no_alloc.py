"""The allocation-free entry point agrees with the ordinary one and with the oracle.

bc_correlate_noalloc serves callers that cannot allocate device memory
(plug-ins in an application that owns the device heap, real-time loops that
must not wait on the allocator): it takes device inputs and a device output
and keeps its scratch in a static device array inside the library.  Here it is
called through the C ABI twice in a row, with different rotations, and each
result is compared with bc_correlate on the same inputs and with the FP64
oracle (layer b).  This file is collected last so that a failure here comes
after every other test.
"""
import numpy as np
import pytest

import oracle as O
from paper_1711_05075_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_TOL = 1e-5  # the tolerance of the GPU parity tests


@pytest.fixture(scope="module")
def bc():
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    torch.cuda.set_device(0)
    import paper_1711_05075_gb300 as m
    return m


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_bc_correlate_on_two_calls(bc):
    wl = synth.small_pair(4)
    dev = torch.device("cuda", 0)
    xa = torch.tensor(wl.A.xyz, dtype=torch.float32, device=dev)
    la = torch.tensor(wl.A.level, dtype=torch.int32, device=dev)
    xb = torch.tensor(wl.B.xyz, dtype=torch.float32, device=dev)
    lb = torch.tensor(wl.B.level, dtype=torch.int32, device=dev)
    quats = synth.shoemake_quaternions(synth.SplitMix64(21), 2).astype(np.float32)

    ctx = bc.Context(wl.N, wl.W, wl.radii, wl.period)
    A = ctx.shape(xa, la)
    B = ctx.shape(xb, lb)
    stream = torch.cuda.current_stream(dev).cuda_stream
    out = torch.empty((wl.N, wl.N, wl.N), dtype=torch.float32, device=dev)
    try:
        for r in range(2):  # two calls in a row share (and must clear) the static scratch
            bc.bc_correlate_noalloc(wl.N, wl.W, wl.radii, xa, la, wl.A.n, xb, lb, wl.B.n, quats[r], out,
                                    period=wl.period, stream=stream)
            torch.cuda.synchronize(dev)
            got = out.double().cpu().numpy()
            ref = ctx.correlate(A, B, quats[r:r + 1])[0].double().cpu().numpy()
            rel = rel_l2(got, ref)
            A64 = synth.Shape(wl.A.xyz.astype(np.float32).astype(np.float64), wl.A.level, wl.A.radii)
            B64 = synth.Shape(wl.B.xyz.astype(np.float32).astype(np.float64), wl.B.level, wl.B.radii)
            orc = O.band_limited_corr(A64, B64, quats[r].astype(np.float64), wl.N, wl.period)
            rel_o = rel_l2(got, orc)
            print(f"call {r}: rel-L2 vs bc_correlate {rel:.3e}, vs FP64 oracle {rel_o:.3e}")
            assert rel <= REL_TOL, rel
            assert rel_o <= REL_TOL, rel_o
    finally:
        A.close()
        B.close()
        ctx.close()


def test_noalloc_rejects_sizes_beyond_its_limits(bc):
    dev = torch.device("cuda", 0)
    x = torch.zeros((bc.BC_NOALLOC_MAX_KNOTS + 1, 3), dtype=torch.float32, device=dev)
    l = torch.zeros(bc.BC_NOALLOC_MAX_KNOTS + 1, dtype=torch.int32, device=dev)
    out = torch.empty((32, 32, 32), dtype=torch.float32, device=dev)
    q = np.array([1, 0, 0, 0], np.float32)
    with pytest.raises(bc.BallCorrError) as e:
        bc.bc_correlate_noalloc(32, 6, (0.04, 0.08), x, l, bc.BC_NOALLOC_MAX_KNOTS + 1, x, l, 4, q, out)
    assert e.value.status == 1 and "BC_NOALLOC_MAX_KNOTS" in str(e.value)
    with pytest.raises(bc.BallCorrError) as e:
        bc.bc_correlate_noalloc(64, 6, (0.04, 0.08), x, l, 4, x, l, 4, q, out)
    assert e.value.status == 1 and "N = 32" in str(e.value)
    with pytest.raises(bc.BallCorrError) as e:
        bc.bc_correlate_noalloc(32, 6, (0.01, 0.02, 0.04), x, l, 4, x, l, 4, q, out)
    assert e.value.status == 1 and "BC_NOALLOC_MAX_LEVELS" in str(e.value)
