"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, layer (b).

Both sides get identical inputs: the seeded knots and quaternions rounded once
to FP32 (the library's input type) and widened back to FP64 for the oracle.
Bar: rel-L2 <= 1e-5 over the compared points (FP32 path), as the method's
accuracy target states; max-abs is reported beside it.  Every workload runs
with both spreading implementations (spread 0: boxes in HBM with global
atomics; spread 1: knots binned by x-cell and spread in shared memory inside
the z transform), and spread 0 with both z transforms (the radix FFT, and the
pruned DFT product on the tcgen05 tensor cores where N <= 128).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1711_05075_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    torch.cuda.set_device(0)
    yield


def bcmod():
    import paper_1711_05075_gb300 as bc
    return bc


def f32(shape):
    return synth.Shape(shape.xyz.astype(np.float32).astype(np.float64), shape.level, shape.radii, shape.name)


SPREADS = (0, 1)
# (spread, z_transform, persistent): boxes + radix FFT z pass, boxes + tensor-core z
# pass, binned -- with the back half as one persistent launch -- and boxes + the
# tensor-core z pass with the back half as three launches
MODES = ((0, 0, 1), (0, 1, 1), (1, 0, 1), (0, 1, 0))


def run_gpu(A, B, quats, N, W, radii=None, period=2.0, spread=1, fft_schedule=0, z_transform=0, persistent=1):
    bc = bcmod()
    radii = A.radii if radii is None else radii
    ctx = bc.Context(N, W, radii, period)
    ctx.set_tuning(spread=spread, fft_schedule=fft_schedule, z_transform=z_transform, persistent=persistent)
    try:
        sa = ctx.shape(A.xyz.astype(np.float32), A.level)
        sb = ctx.shape(B.xyz.astype(np.float32), B.level)
        g = ctx.correlate(sa, sb, np.asarray(quats, dtype=np.float32))
        ctx.sync()
        out = g.double().cpu().numpy()
        sa.close()
        sb.close()
    finally:
        ctx.close()
    return out


def run_modes(A, B, quats, N, W, **kw):
    """(label, grids) for each implementation: spreading 0 with each z transform, spreading 1."""
    for sp, zt, pe in MODES:
        if zt and N > 128:
            zt = 0
        yield (f"{sp}{' z-tc' if zt else ''}{' persistent' if pe else ' 3 launches'}",
               run_gpu(A, B, quats, N, W, spread=sp, z_transform=zt, persistent=pe, **kw))


def oracle_grid(A, B, q, N, period=2.0):
    return O.band_limited_corr(f32(A), f32(B), np.asarray(q, np.float32).astype(np.float64), N, period)


def rel_l2(got, ref):
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def check(got, ref, tol=REL_TOL, what=""):
    rel = rel_l2(got, ref)
    mx = float(np.abs(got - ref).max())
    print(f"{what}: rel-L2 {rel:.3e}  max-abs {mx:.3e}  (|ref|max {np.abs(ref).max():.3e})")
    assert rel <= tol, (what, rel, mx)
    return rel


# ------------------------------------------------------------------ workloads
def test_small_pair_full_grid():
    wl = synth.small_pair(0)
    ref = oracle_grid(wl.A, wl.B, wl.quats[0], wl.N)
    for sp, got in run_modes(wl.A, wl.B, wl.quats, wl.N, wl.W):
        check(got[0], ref, what=f"{wl.name} spread {sp}")


def test_scale_pair_full_grid_and_sampled():
    wl = synth.scale_pair(0)
    g = O.band_limited_spectrum(f32(wl.A), f32(wl.B), wl.quats[0].astype(np.float32).astype(np.float64), wl.N)
    ref = O.inverse_grid(g)
    idx = synth.translation_sample(wl.N, 4096, seed=0)
    pts = O.inverse_at(g, O.grid_points(wl.N, idx=idx))
    for sp, got in run_modes(wl.A, wl.B, wl.quats, wl.N, wl.W):
        check(got[0], ref, what=f"{wl.name} full grid, spread {sp}")
        check(got[0].reshape(-1)[idx], pts, what=f"{wl.name} 4096 sampled t, spread {sp}")


@pytest.mark.parametrize("k", [1, 3])
def test_rotations(k):
    wl = synth.small_pair(1)
    q = synth.shoemake_quaternions(synth.SplitMix64(99), k)
    refs = [oracle_grid(wl.A, wl.B, q[r], wl.N) for r in range(k)]
    for sp, got in run_modes(wl.A, wl.B, q, wl.N, wl.W):
        for r in range(k):
            check(got[r], refs[r], what=f"rotation {r} of {k}, spread {sp}")


# W = 9 is the widest window whose stencil columns the spreading kernel splits
# into (column, 4-cell group) tasks; W = 10 takes the whole-column path.
@pytest.mark.parametrize("N,W,n", [(32, 8, 300), (64, 8, 400), (96, 8, 500), (128, 6, 300), (32, 9, 300),
                                   (32, 10, 300)])
def test_grid_sizes(N, W, n):
    A = synth.ellipsoid_shape(n, 5, synth.RADII_4, synth.PROBS_4)
    B = synth.torus_shape(n, 6, synth.RADII_4, synth.PROBS_4)
    q = synth.shoemake_quaternions(synth.SplitMix64(3), 2)
    refs = [oracle_grid(A, B, q[r], N) for r in range(2)]
    for sp, got in run_modes(A, B, q, N, W):
        for r in range(2):
            check(got[r], refs[r], what=f"N={N} W={W} rot {r} spread {sp}")


def test_grid_size_256_sampled():
    N, W = 256, 8
    A = synth.ellipsoid_shape(300, 7, synth.RADII_4, synth.PROBS_4)
    B = synth.torus_shape(300, 8, synth.RADII_4, synth.PROBS_4)
    q = synth.IDENTITY_QUAT
    g = O.band_limited_spectrum(f32(A), f32(B), q[0], N)
    idx = synth.translation_sample(N, 4096, seed=1)
    ref = O.inverse_at(g, O.grid_points(N, idx=idx))
    for sp, got in run_modes(A, B, q, N, W):
        check(got[0].reshape(-1)[idx], ref, what=f"N=256 sampled, spread {sp}")


# ------------------------------------------------------------------ edge cases
@pytest.mark.parametrize("spread,zt,pe", MODES)
def test_repeated_calls_are_identical(spread, zt, pe):
    # The spreading boxes (bin counts) are cleared by the pass that consumes
    # them; a second call on the same context must not see the first call's.
    bc = bcmod()
    wl = synth.small_pair(2)
    ctx = bc.Context(wl.N, wl.W, wl.radii)
    ctx.set_tuning(spread=spread, z_transform=zt, persistent=pe)
    sa = ctx.shape(wl.A.xyz, wl.A.level)
    sb = ctx.shape(wl.B.xyz, wl.B.level)
    g1 = ctx.correlate(sa, sb, wl.quats).clone()
    g2 = ctx.correlate(sa, sb, wl.quats).clone()
    q = synth.shoemake_quaternions(synth.SplitMix64(1), 4)
    ctx.correlate(sa, sb, q)
    g3 = ctx.correlate(sa, sb, wl.quats).clone()
    ctx.sync()
    assert rel_l2(g2.double().cpu().numpy(), g1.double().cpu().numpy()) < 1e-6
    assert rel_l2(g3.double().cpu().numpy(), g1.double().cpu().numpy()) < 1e-6
    sa.close(); sb.close(); ctx.close()


def test_host_output_matches_device_output():
    bc = bcmod()
    wl = synth.small_pair(3)
    ctx = bc.Context(wl.N, wl.W, wl.radii)
    sa = ctx.shape(wl.A.xyz, wl.A.level)
    sb = ctx.shape(wl.B.xyz, wl.B.level)
    dev = ctx.correlate(sa, sb, wl.quats).cpu().numpy()
    host = np.empty_like(dev)
    ctx.correlate_host(sa, sb, wl.quats, host)
    # float atomics in the spreading pass add in a run-dependent order: results
    # agree to rounding, not bit for bit
    assert rel_l2(host.astype(np.float64), dev.astype(np.float64)) < 1e-6
    # device-resident knots give the same result as host knots
    sa2 = ctx.shape(torch.tensor(wl.A.xyz, dtype=torch.float32, device="cuda"),
                    torch.tensor(wl.A.level, dtype=torch.int32, device="cuda"))
    dev2 = ctx.correlate(sa2, sb, wl.quats).cpu().numpy()
    assert rel_l2(dev2.astype(np.float64), dev.astype(np.float64)) < 1e-6
    # page-locked host output (stored by the last kernel through its device
    # mapping) and page-locked host knots (copied asynchronously); twice, so
    # that the second call replays a recorded graph writing the same buffer
    xp = torch.tensor(wl.A.xyz, dtype=torch.float32).pin_memory()
    lp = torch.tensor(wl.A.level, dtype=torch.int32).pin_memory()
    sa3 = ctx.shape(xp, lp)
    for _ in range(3):
        pinned = torch.full(dev.shape, float("nan"), dtype=torch.float32).pin_memory()
        ctx.correlate_host(sa3, sb, wl.quats, pinned)
        assert rel_l2(pinned.numpy().astype(np.float64), dev.astype(np.float64)) < 1e-6
    # the caller may overwrite its knot arrays once the shape exists
    xp.fill_(0.5)
    again = np.empty_like(dev)
    ctx.correlate_host(sa3, sb, wl.quats, again)
    assert rel_l2(again.astype(np.float64), dev.astype(np.float64)) < 1e-6
    for s in (sa, sb, sa2, sa3):
        s.close()
    ctx.close()


def test_batched_shape_upload():
    # bc_shapes_create: several shapes (one of them empty) in one call give the
    # same correlations as shapes uploaded one by one; a bad shape anywhere in
    # the batch fails the whole call and creates nothing
    bc = bcmod()
    wl = synth.small_pair(4)
    ctx = bc.Context(wl.N, wl.W, wl.radii)
    sa, sb = ctx.shape(wl.A.xyz, wl.A.level), ctx.shape(wl.B.xyz, wl.B.level)
    ref = ctx.correlate(sa, sb, wl.quats).cpu().numpy()
    empty = (np.zeros((0, 3), np.float32), np.zeros(0, np.int32))
    for form in ("host", "device"):
        pairs = [(wl.A.xyz, wl.A.level), empty, (wl.B.xyz, wl.B.level)]
        if form == "device":
            pairs = [(torch.tensor(x, dtype=torch.float32, device="cuda"), torch.tensor(l, dtype=torch.int32, device="cuda"))
                     for x, l in pairs]
        a, e, b = ctx.shapes(pairs)
        assert (a.n, e.n, b.n) == (wl.A.n, 0, wl.B.n)
        got = ctx.correlate(a, b, wl.quats).cpu().numpy()
        assert rel_l2(got.astype(np.float64), ref.astype(np.float64)) < 1e-6
        assert float(ctx.correlate(a, e, wl.quats).abs().max()) == 0.0
        for s in (a, e, b):
            s.close()
    bad = (wl.B.xyz, np.full(wl.B.n, 7, np.int32))
    with pytest.raises(bc.BallCorrError) as err:
        ctx.shapes([(wl.A.xyz, wl.A.level), bad])
    assert err.value.status == 1 and "shape 1" in str(err.value)
    assert ctx.shapes([]) == []
    sa.close(); sb.close(); ctx.close()


def test_empty_shape_gives_zero():
    bc = bcmod()
    wl = synth.small_pair(0)
    ctx = bc.Context(wl.N, wl.W, wl.radii)
    sa = ctx.shape(wl.A.xyz, wl.A.level)
    se = ctx.shape(np.zeros((0, 3), np.float32), np.zeros(0, np.int32))
    g = ctx.correlate(sa, se, wl.quats)
    g2 = ctx.correlate(se, sa, wl.quats)
    ctx.sync()
    assert float(g.abs().max()) == 0.0 and float(g2.abs().max()) == 0.0
    sa.close(); se.close(); ctx.close()


def test_single_balls_and_two_ball_closed_form():
    # One ball each: g^(m) = h^_{r1} h^_{r2} exp(-2 pi i m.(c1 - R c2)/P); the oracle's
    # layer (b) gives it, and the GPU must match.
    A = synth.Shape(np.array([[0.1, -0.2, 0.05]]), np.array([1], np.int32), (0.04, 0.08))
    B = synth.Shape(np.array([[-0.3, 0.1, 0.2]]), np.array([0], np.int32), (0.04, 0.08))
    q = synth.shoemake_quaternions(synth.SplitMix64(5), 1)
    ref = oracle_grid(A, B, q[0], 32)
    for sp, got in run_modes(A, B, q, 32, 6):
        check(got[0], ref, what=f"one ball each, spread {sp}")


def test_empty_level_and_single_level():
    A = synth.ellipsoid_shape(200, 11)
    A0 = synth.Shape(A.xyz, np.zeros_like(A.level), A.radii)  # level 1 empty
    B = synth.torus_shape(150, 12)
    ref = oracle_grid(A0, B, synth.IDENTITY_QUAT[0], 32)
    for sp, got in run_modes(A0, B, synth.IDENTITY_QUAT, 32, 6):
        check(got[0], ref, what=f"empty level, spread {sp}")


def test_knots_outside_the_box_wrap():
    A = synth.ellipsoid_shape(150, 13)
    B = synth.torus_shape(150, 14)
    shift = np.array([2.0, -2.0, 4.0])  # whole periods: same periodic shape
    A2 = synth.Shape(A.xyz + shift, A.level, A.radii)
    ref = oracle_grid(A, B, synth.IDENTITY_QUAT[0], 32)
    for sp in SPREADS:
        g1 = run_gpu(A, B, synth.IDENTITY_QUAT, 32, 6, spread=sp)[0]
        g2 = run_gpu(A2, B, synth.IDENTITY_QUAT, 32, 6, spread=sp)[0]
        check(g2, ref, what=f"shifted by periods, spread {sp}")
        assert rel_l2(g2, g1) < 2e-6


def test_shape_straddling_the_periodic_boundary():
    A = synth.ellipsoid_shape(200, 15)
    A2 = synth.Shape(A.xyz + np.array([0.85, 0.0, -0.9]), A.level, A.radii)  # wraps in x and z
    B = synth.torus_shape(200, 16)
    q = synth.shoemake_quaternions(synth.SplitMix64(8), 2)
    refs = [oracle_grid(A2, B, q[r], 32) for r in range(2)]
    for sp, got in run_modes(A2, B, q, 32, 6):
        for r in range(2):
            check(got[r], refs[r], what=f"straddling, rot {r}, spread {sp}")


def test_wide_box_takes_the_register_path_at_N128():
    # An x extent of about 240 of the 256 fine cells is beyond the x pass's
    # staging tiles (160 rows at n = 256): that pair takes the register-fed path.
    A = synth.ellipsoid_shape(400, 21, synth.RADII_4, synth.PROBS_4, semi=(0.88, 0.3, 0.25))
    B = synth.torus_shape(400, 22, synth.RADII_4, synth.PROBS_4)
    q = synth.shoemake_quaternions(synth.SplitMix64(9), 1)
    idx = synth.translation_sample(128, 4096, seed=2)
    ref = O.band_limited_corr(f32(A), f32(B), q[0].astype(np.float32).astype(np.float64), 128, idx=idx)
    for sp, got in run_modes(A, B, q, 128, 8):
        check(got[0].reshape(-1)[idx], ref, what=f"wide box N=128, spread {sp}")


def test_invalid_arguments_raise():
    bc = bcmod()
    ctx = bc.Context(32, 6, (0.04, 0.08))
    with pytest.raises(bc.BallCorrError) as e:
        ctx.shape(np.zeros((4, 3), np.float32), np.array([0, 1, 2, 0], np.int32))
    assert e.value.status == 1
    with pytest.raises(bc.BallCorrError) as e:
        ctx.shape(np.full((2, 3), np.nan, np.float32), np.array([0, 1], np.int32))
    assert e.value.status == 1
    # the same checks on host (pageable and page-locked) and device input
    bad = [(np.array([[0.1, 0.2, np.inf]], np.float32), np.array([0], np.int32)),
           (np.zeros((3, 3), np.float32), np.array([0, -1, 1], np.int32))]
    for x, l in bad:
        for form in ("host", "pinned", "device"):
            if form == "host":
                xx, ll = x, l
            elif form == "pinned":
                xx, ll = torch.from_numpy(x).pin_memory(), torch.from_numpy(l).pin_memory()
            else:
                xx, ll = torch.from_numpy(x).cuda(), torch.from_numpy(l).cuda()
            with pytest.raises(bc.BallCorrError) as e:
                ctx.shape(xx, ll)
            assert e.value.status == 1, form
    sa = ctx.shape(np.zeros((1, 3), np.float32), np.array([0], np.int32))
    with pytest.raises(bc.BallCorrError) as e:
        ctx.correlate(sa, sa, np.zeros((1, 4), np.float32))
    assert e.value.status == 1
    sa.close()
    ctx.close()


def test_spreading_modes_agree_on_a_dense_shape_and_switch_on_one_context():
    # Many knots in few cells (long bins, several hit chunks per item) and a
    # context switched between the two implementations between calls.
    bc = bcmod()
    rng = synth.SplitMix64(21)
    n = 6000
    xyz = (rng.uniform(3 * n).reshape(n, 3) - 0.5) * 0.2  # a 0.2-wide cube: about 20 knots per x-cell
    A = synth.Shape(xyz, (rng.uniform(n) * 2).astype(np.int32), synth.RADII_2)
    B = synth.torus_shape(300, 22)
    q = synth.shoemake_quaternions(synth.SplitMix64(23), 1)
    ref = oracle_grid(A, B, q[0], 32)
    ctx = bc.Context(32, 6, synth.RADII_2)
    sa = ctx.shape(A.xyz.astype(np.float32), A.level)
    sb = ctx.shape(B.xyz.astype(np.float32), B.level)
    outs = []
    for sp, zt in ((1, 0), (0, 0), (0, 1), (1, 0)):
        ctx.set_tuning(spread=sp, z_transform=zt)
        outs.append(ctx.correlate(sa, sb, q).double().cpu().numpy()[0])
        check(outs[-1], ref, what=f"dense cube, spread {sp}, z transform {zt}")
    assert rel_l2(outs[3], outs[0]) < 1e-6
    sa.close(); sb.close(); ctx.close()


def test_autotune_keeps_a_valid_choice():
    bc = bcmod()
    wl = synth.small_pair(4)
    ctx = bc.Context(wl.N, wl.W, wl.radii)
    sa = ctx.shape(wl.A.xyz, wl.A.level)
    sb = ctx.shape(wl.B.xyz, wl.B.level)
    t = ctx.autotune(sa, sb, rotations=40)
    assert t == ctx.tuning and t["spread"] in (0, 1) and t["sweep_batch"] in (16, 32, 64) and t["graphs"] == 1
    assert 0 <= t["fft_schedule"] <= 7 and t["z_transform"] in (0, 1)
    got = ctx.correlate(sa, sb, wl.quats).double().cpu().numpy()[0]
    check(got, oracle_grid(wl.A, wl.B, wl.quats[0], wl.N), what=f"after autotune {t}")
    with pytest.raises(bc.BallCorrError):
        ctx.set_tuning(spread=2)
    with pytest.raises(bc.BallCorrError):
        ctx.set_tuning(sweep_batch=0)
    sa.close(); sb.close(); ctx.close()


@pytest.mark.parametrize("spread,zt", [(1, 0), (0, 1)])
def test_launch_overlap_matches_ordinary_launches(spread, zt):
    # overlap 1 (the default) launches every pass after the first as a programmatic
    # dependent of the one before; overlap 0 launches each after the previous one has
    # ended.  Same kernels and arithmetic: with the fixed-point binned spreading the
    # grids agree bit for bit; with the atomic spreading both meet the oracle bar.
    bc = bcmod()
    wl = synth.small_pair(6)
    q = synth.shoemake_quaternions(synth.SplitMix64(37), 1).astype(np.float32)
    ref = oracle_grid(wl.A, wl.B, q[0], wl.N)
    ctx = bc.Context(wl.N, wl.W, wl.radii)
    assert ctx.tuning["overlap"] == 1
    sa = ctx.shape(wl.A.xyz, wl.A.level)
    sb = ctx.shape(wl.B.xyz, wl.B.level)
    out = torch.empty((1, wl.N, wl.N, wl.N), dtype=torch.float32, device="cuda")
    grids = {}
    for ov in (1, 0):
        for graphs in (1, 0):
            ctx.set_tuning(spread=spread, z_transform=zt, persistent=0, overlap=ov, graphs=graphs)
            for _ in range(3):  # the second identical pass records a graph, the third replays it
                ctx.correlate(sa, sb, q, out)
            grids[(ov, graphs)] = out.double().cpu().numpy()[0].copy()
            check(grids[(ov, graphs)], ref, what=f"overlap {ov}, graphs {graphs}, spread {spread}")
    if spread == 1:
        for key, g in grids.items():
            assert np.array_equal(g, grids[(0, 0)]), key
    with pytest.raises(bc.BallCorrError):
        ctx.set_tuning(overlap=2)
    sa.close(); sb.close(); ctx.close()


@pytest.mark.parametrize("spread,zt,pe", MODES)
def test_graph_replay_matches_oracle_and_kernel_by_kernel(spread, zt, pe):
    # Identical passes (same descriptors and buffers) replay the recorded graph;
    # a changed rotation re-records; switching replay off launches kernel by kernel.
    bc = bcmod()
    wl = synth.small_pair(5)
    q = synth.shoemake_quaternions(synth.SplitMix64(31), 2).astype(np.float32)
    refs = [oracle_grid(wl.A, wl.B, q[r], wl.N) for r in range(2)]
    ctx = bc.Context(wl.N, wl.W, wl.radii)
    ctx.set_tuning(spread=spread, graphs=1, z_transform=zt, persistent=pe)
    sa = ctx.shape(wl.A.xyz, wl.A.level)
    sb = ctx.shape(wl.B.xyz, wl.B.level)
    out = torch.empty((1, wl.N, wl.N, wl.N), dtype=torch.float32, device="cuda")
    for r in (0, 0, 0, 1, 1, 0):
        ctx.correlate(sa, sb, q[r:r + 1], out)
        check(out.double().cpu().numpy()[0], refs[r], what=f"graph replay, rotation {r}, spread {spread}")
    ctx.set_tuning(graphs=0)
    assert ctx.tuning["graphs"] == 0
    ctx.correlate(sa, sb, q[1:2], out)
    check(out.double().cpu().numpy()[0], refs[1], what=f"kernel by kernel, spread {spread}")
    sa.close(); sb.close(); ctx.close()


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    # failure detection without a fault: device waits that nothing satisfies (an
    # mbarrier of the tensor-core kernels, a work-queue counter of the persistent
    # launch) expire (about 2 s each), are reported as BC_ERR_TIMEOUT (4), and the
    # next correlations on the same context -- with the tensor-core z pass and with
    # the persistent back half -- are correct
    bc = bcmod()
    wl = synth.small_pair(6)
    ctx = bc.Context(wl.N, wl.W, wl.radii)
    assert ctx.selftest_wait() == 4
    ctx.sync()  # the error word was cleared
    sa = ctx.shape(wl.A.xyz, wl.A.level)
    sb = ctx.shape(wl.B.xyz, wl.B.level)
    ref = oracle_grid(wl.A, wl.B, wl.quats[0], wl.N)
    for pe in (0, 1):
        ctx.set_tuning(z_transform=1, persistent=pe)
        got = ctx.correlate(sa, sb, wl.quats).double().cpu().numpy()[0]
        check(got, ref, what=f"after the expired waits, persistent {pe}")
    sa.close(); sb.close(); ctx.close()


def test_z_transform_availability():
    # the tensor-core z transform: FP32 contexts with N <= 128 start with it;
    # elsewhere selecting it is refused (BC_ERR_UNSUPPORTED = 5)
    bc = bcmod()
    ctx = bc.Context(128, 8, synth.RADII_4)
    assert ctx.tuning["z_transform"] == 1
    ctx.set_tuning(z_transform=0)
    assert ctx.tuning["z_transform"] == 0
    with pytest.raises(bc.BallCorrError):
        ctx.set_tuning(z_transform=2)
    ctx.close()
    ctx = bc.Context(256, 8, synth.RADII_4)
    assert ctx.tuning["z_transform"] == 0
    with pytest.raises(bc.BallCorrError) as e:
        ctx.set_tuning(z_transform=1)
    assert e.value.status == 5
    ctx.close()
    ctx = bc.Context(32, 8, synth.RADII_4, precision=1)
    assert ctx.tuning["z_transform"] == 0
    ctx.close()


@pytest.mark.parametrize("N,W,n", [(32, 8, 300), (64, 8, 400), (96, 8, 500), (128, 8, 300)])
def test_alternative_radix_schedules(N, W, n):
    # fft_schedule 1: 64 = 4.16, 128 = 16.8, 192 = 3.4.16, 256 = 4.8.8 for the forward passes
    A = synth.ellipsoid_shape(n, 25, synth.RADII_4, synth.PROBS_4)
    B = synth.torus_shape(n, 26, synth.RADII_4, synth.PROBS_4)
    q = synth.shoemake_quaternions(synth.SplitMix64(27), 1)
    ref = oracle_grid(A, B, q[0], N)
    for sp in SPREADS:
        got = run_gpu(A, B, q, N, W, spread=sp, fft_schedule=7)
        check(got[0], ref, what=f"schedule 1, N={N}, spread {sp}")


def test_alternative_radix_schedule_512_sampled():
    N, W = 256, 8
    A = synth.ellipsoid_shape(300, 28, synth.RADII_4, synth.PROBS_4)
    B = synth.torus_shape(300, 29, synth.RADII_4, synth.PROBS_4)
    q = synth.IDENTITY_QUAT
    g = O.band_limited_spectrum(f32(A), f32(B), q[0], N)
    idx = synth.translation_sample(N, 4096, seed=2)
    ref = O.inverse_at(g, O.grid_points(N, idx=idx))
    got = run_gpu(A, B, q, N, W, spread=0, fft_schedule=7)[0]
    check(got.reshape(-1)[idx], ref, what="schedule 1 (512 = 8.4.16), N=256 sampled")
