"""GPU rotation sweep (bc_sweep): peak of g over the translation grid per rotation.

The oracle computes the full band-limited grid per rotation (layer b); the
peak value must agree within the parity tolerance (relative to max |g|), and
the GPU's argmax must be a valid maximiser: the oracle's value there equals
the oracle's maximum within the same tolerance (on near-ties several indices
are correct).  The sweep must also agree with bc_correlate's full grids.
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
    return synth.Shape(S.xyz.astype(np.float32).astype(np.float64), S.level, S.radii)


def check_peaks(peak, arg, grids, what):
    for r, g in enumerate(grids):
        scale = np.abs(g).max()
        flat = g.reshape(-1)
        assert abs(peak[r] - flat.max()) <= REL_TOL * scale, (what, r, peak[r], flat.max())
        assert flat[arg[r]] >= flat.max() - REL_TOL * scale, (what, r, arg[r], flat[arg[r]], flat.max())
        print(f"{what} rot {r}: peak {peak[r]:.6e} oracle {flat.max():.6e} argmax {arg[r]} oracle {int(flat.argmax())}")


@pytest.mark.parametrize("batch", [0, 2])
def test_sweep_matches_oracle_small(bc, batch):
    wl = synth.small_pair(5)
    q = np.concatenate([synth.IDENTITY_QUAT, synth.shoemake_quaternions(synth.SplitMix64(12), 4)]).astype(np.float32)
    ctx = bc.Context(wl.N, wl.W, wl.radii)
    A = ctx.shape(wl.A.xyz, wl.A.level)
    B = ctx.shape(wl.B.xyz, wl.B.level)
    peak, arg = ctx.sweep(A, B, q, batch=batch)
    full = ctx.correlate(A, B, q)
    ctx.sync()
    peak, arg = peak.cpu().numpy(), arg.cpu().numpy()
    full = full.double().cpu().numpy()
    grids = [O.band_limited_corr(f32(wl.A), f32(wl.B), q[r].astype(np.float64), wl.N) for r in range(len(q))]
    check_peaks(peak, arg, grids, f"small batch={batch}")
    # the fused peak equals the maximum of the written grid (same kernels, other rounding order)
    for r in range(len(q)):
        assert abs(peak[r] - full[r].max()) <= 1e-6 * np.abs(full[r]).max()
    A.close(); B.close(); ctx.close()


def test_sweep_host_output(bc):
    wl = synth.small_pair(6)
    q = synth.shoemake_quaternions(synth.SplitMix64(13), 3).astype(np.float32)
    ctx = bc.Context(wl.N, wl.W, wl.radii)
    A = ctx.shape(wl.A.xyz, wl.A.level)
    B = ctx.shape(wl.B.xyz, wl.B.level)
    pd, ad = ctx.sweep(A, B, q)
    ph = np.empty(3, np.float32)
    ah = np.empty(3, np.int32)
    bc.bc_sweep(ctx.handle, A.handle, B.handle, q, 3, 0, ph, ah, 0)
    np.testing.assert_allclose(ph, pd.cpu().numpy(), rtol=1e-6)
    A.close(); B.close(); ctx.close()


def test_sweep_receptor_ligand_sampled_rotations(bc):
    # 50,000-ball receptor (union of 3 ellipsoids), 5,000-ball ligand (torus),
    # N = 96, W = 8: a 64-rotation sweep, four rotations checked against the oracle.
    wl = synth.sweep_pair(0, k=64)
    ctx = bc.Context(wl.N, wl.W, wl.radii)
    A = ctx.shape(wl.A.xyz, wl.A.level)
    B = ctx.shape(wl.B.xyz, wl.B.level)
    q = wl.quats.astype(np.float32)
    peak, arg = ctx.sweep(A, B, q, batch=16)
    ctx.sync()
    peak, arg = peak.cpu().numpy(), arg.cpu().numpy()
    fa = O.shape_spectrum(f32(wl.A).xyz, wl.A.level, wl.A.radii, wl.N)
    pick = [0, 17, 40, 63]
    grids = []
    for r in pick:
        fb = O.shape_spectrum(f32(wl.B).xyz, wl.B.level, wl.B.radii, wl.N, q[r].astype(np.float64))
        grids.append(O.inverse_grid(O.corr_spectrum(fa, fb)))
    check_peaks(peak[pick], arg[pick], grids, "receptor/ligand")
    A.close(); B.close(); ctx.close()


def test_ragged_pairs_match_oracle(bc):
    # Pairs of uneven knot counts (log-uniform in [100, 3000]) in one call; grids and peaks.
    rng = synth.SplitMix64(77)
    counts = np.exp(np.log(100) + rng.uniform(8) * (np.log(3000) - np.log(100))).astype(int)
    N, W = 32, 6
    ctx = bc.Context(N, W, synth.RADII_2)
    shapesA, shapesB, hA, hB = [], [], [], []
    for i in range(4):
        a = synth.ellipsoid_shape(int(counts[2 * i]), 100 + i)
        b = synth.torus_shape(int(counts[2 * i + 1]), 200 + i)
        shapesA.append(a); shapesB.append(b)
        hA.append(ctx.shape(a.xyz, a.level)); hB.append(ctx.shape(b.xyz, b.level))
    q = synth.shoemake_quaternions(synth.SplitMix64(78), 4).astype(np.float32)
    grids, peak, arg = ctx.pairs(hA, hB, q, grids=True, peaks=True)
    ctx.sync()
    grids = grids.double().cpu().numpy()
    peak, arg = peak.cpu().numpy(), arg.cpu().numpy()
    ref = []
    for i in range(4):
        g = O.band_limited_corr(f32(shapesA[i]), f32(shapesB[i]), q[i].astype(np.float64), N)
        rel = np.linalg.norm(grids[i] - g) / np.linalg.norm(g)
        print(f"pair {i} ({shapesA[i].n}+{shapesB[i].n} knots): rel-L2 {rel:.3e}")
        assert rel <= REL_TOL
        ref.append(g)
    check_peaks(peak, arg, ref, "ragged pairs")
    # host outputs: grids into page-locked memory (stored through its device
    # mapping), peaks into pageable arrays
    hg = torch.empty((4, N, N, N), dtype=torch.float32).pin_memory()
    hp, ha = np.empty(4, np.float32), np.empty(4, np.int32)
    bc.bc_pairs(ctx.handle, [h.handle for h in hA], [h.handle for h in hB], q, 4, hg, hp, ha, 0)
    for i in range(4):
        assert np.linalg.norm(hg[i].double().numpy() - ref[i]) / np.linalg.norm(ref[i]) <= REL_TOL
    check_peaks(hp, ha, ref, "ragged pairs, host outputs")
    for h in hA + hB:
        h.close()
    ctx.close()


def test_ragged_pairs_at_full_size(bc):
    # The ragged batch at its benchmark size: 64 pairs with knot counts log-uniform
    # in [1,000, 100,000] (2.9M knots in all), N = 96, W = 8, L = 4, in one call.
    # The largest, the smallest and the median pair are checked against the oracle
    # at 4,096 sampled translations; every pair's fused peak against its own grid.
    pairs, q = synth.ragged_pairs(0)
    q = q.astype(np.float32)
    N, W = 96, 8
    ctx = bc.Context(N, W, synth.RADII_4)
    hA = [ctx.shape(a.xyz, a.level) for a, _ in pairs]
    hB = [ctx.shape(b.xyz, b.level) for _, b in pairs]
    grids, peak, arg = ctx.pairs(hA, hB, q, grids=True, peaks=True)
    ctx.sync()
    idx = synth.translation_sample(N, 4096, 0)
    sizes = np.array([a.n + b.n for a, b in pairs])
    order = np.argsort(sizes, kind="stable")
    check = [int(order[-1]), int(order[0]), int(order[len(order) // 2])]
    for i in check:
        a, b = pairs[i]
        got = grids[i].reshape(-1)[torch.as_tensor(idx, device=grids.device)].double().cpu().numpy()
        ref = O.band_limited_corr(f32(a), f32(b), q[i].astype(np.float64), N, idx=idx)
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        print(f"pair {i} ({a.n}+{b.n} knots): rel-L2 at 4,096 t {rel:.3e}")
        assert rel <= REL_TOL, (i, rel)
    gmax = grids.reshape(len(pairs), -1).max(dim=1).values.cpu().numpy()
    scale = grids.reshape(len(pairs), -1).abs().max(dim=1).values.cpu().numpy()
    peak, arg = peak.cpu().numpy(), arg.cpu().numpy()
    np.testing.assert_array_less(np.abs(peak - gmax), 1e-6 * scale + 1e-30)
    flat = grids.reshape(len(pairs), -1)
    at_arg = flat[torch.arange(len(pairs), device=flat.device), torch.as_tensor(arg, device=flat.device).long()]
    np.testing.assert_array_less(gmax - at_arg.cpu().numpy(), 1e-6 * scale + 1e-30)
    for h in hA + hB:
        h.close()
    ctx.close()


@pytest.mark.parametrize("N,k", [(32, 48), (64, 24), (128, 12)])
def test_many_pairs_take_the_planewise_inverse(bc, N, k):
    # With many pairs in one pass (here k rotations of one correlate call) the
    # inverse y and z transforms run plane by plane in shared memory
    # (k_ifft_yz); three of the k grids against the oracle, all k against the
    # same rotations computed one per call (the two inverse kernels).
    A = synth.ellipsoid_shape(300, 31, synth.RADII_4, synth.PROBS_4)
    B = synth.torus_shape(250, 32, synth.RADII_4, synth.PROBS_4)
    q = synth.shoemake_quaternions(synth.SplitMix64(33), k).astype(np.float32)
    ctx = bc.Context(N, 8, synth.RADII_4)
    hA, hB = ctx.shape(A.xyz, A.level), ctx.shape(B.xyz, B.level)
    grids = ctx.correlate(hA, hB, q).double().cpu().numpy()
    for r in (0, k // 2, k - 1):
        ref = O.band_limited_corr(f32(A), f32(B), q[r].astype(np.float64), N)
        rel = np.linalg.norm(grids[r] - ref) / np.linalg.norm(ref)
        print(f"N={N} k={k} rot {r}: rel-L2 {rel:.3e}")
        assert rel <= REL_TOL
    for r in range(k):
        one = ctx.correlate(hA, hB, q[r:r + 1])[0].double().cpu().numpy()
        assert np.linalg.norm(grids[r] - one) <= 1e-6 * np.linalg.norm(one), r
    hA.close(); hB.close(); ctx.close()


def test_captured_sweep_plan_replays(bc):
    # The same sweep as one CUDA graph: identical peaks to bc_sweep, replayable.
    wl = synth.small_pair(9)
    q = synth.shoemake_quaternions(synth.SplitMix64(41), 10).astype(np.float32)
    ctx = bc.Context(wl.N, wl.W, wl.radii)
    A = ctx.shape(wl.A.xyz, wl.A.level)
    B = ctx.shape(wl.B.xyz, wl.B.level)
    ref_p, ref_a = ctx.sweep(A, B, q, batch=4)
    peak = torch.empty(10, dtype=torch.float32, device="cuda")
    arg = torch.empty(10, dtype=torch.int32, device="cuda")
    plan = bc.bc_sweep_plan(ctx.handle, A.handle, B.handle, q, 10, 4, peak, arg)
    for _ in range(3):
        peak.fill_(-1.0)
        bc.bc_plan_run(plan)
        ctx.sync()
        np.testing.assert_allclose(peak.cpu().numpy(), ref_p.cpu().numpy(), rtol=1e-6)
    # the context's own calls in between do not disturb the plan's workspaces
    ctx.correlate(A, B, q[:2])
    bc.bc_plan_run(plan)
    ctx.sync()
    np.testing.assert_allclose(peak.cpu().numpy(), ref_p.cpu().numpy(), rtol=1e-6)
    bc.bc_plan_destroy(plan)
    A.close(); B.close(); ctx.close()
