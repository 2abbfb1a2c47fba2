"""GPU learned proposal, end to end at a small size: what the trained network
gains over ranking rotations without it, and the multi-step training call.

Training labels come from the batched sweep with the binned spreading, whose
sums are order-independent fixed point, so the labels -- and with the
deterministic training the network -- are the same on every run.  The network
takes the moments of the ligand as given or, in the second case, turned by
each rotation.  The gain is
measured on held-out receptor/ligand pairs against a random choice of the same
number of rotations (the method without a network must correlate rotations it
cannot rank: a random subset is the fair baseline for a fixed budget of full
correlations): the rank correlation of the network's scores with the true peaks,
and the standardised peaks of the rotations the network picks against those of
a random pick.  The share of the true best K among the picks and the best peak
inside them are printed beside the random choice's: at this small
size (N = 32, 3,000 + 600 knots) the peak varies little over rotations and a
random choice of 64 already reaches about 95% of the best peak, while the
network's picks crowd into one region.
"""
import numpy as np
import pytest

from paper_1711_05075_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bc():
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    torch.cuda.set_device(0)
    import paper_1711_05075_gb300 as m
    return m


def pair(seed):
    return (synth.ellipsoid_union_shape(3000, seed),
            synth.torus_shape(600, seed + 7000, synth.RADII_4, synth.PROBS_4, R=0.35, r=0.08))


def spearman(a, b):
    ra = np.argsort(np.argsort(a)).astype(np.float64)
    rb = np.argsort(np.argsort(b)).astype(np.float64)
    ra -= ra.mean()
    rb -= rb.mean()
    return float((ra * rb).sum() / np.sqrt((ra * ra).sum() * (rb * rb).sum()))


def labelled(bc, ctx, net, seeds, nrot, augment, dev, rotated):
    def ligand(hB, qd, fb):
        return bc.moments_rot(ctx, hB, qd) if rotated else fb

    Xs, ts = [], []
    for seed in seeds:
        A, B = pair(seed)
        hA, hB = ctx.shape(A.xyz, A.level), ctx.shape(B.xyz, B.level)
        q = synth.shoemake_quaternions(synth.SplitMix64(seed + 100), nrot).astype(np.float32)
        peak, _ = ctx.sweep(hA, hB, q, batch=128)
        z = (peak - peak.mean()) / peak.std()
        qd = torch.tensor(q, device=dev)
        fb = bc.moments(ctx, hB)
        Xs.append(net.features(qd, bc.moments(ctx, hA), ligand(hB, qd, fb)))
        ts.append(z)
        # (S A, S R B) has the peak of (A, R B): the same labels for turned receptors
        for s_q in synth.shoemake_quaternions(synth.SplitMix64(seed + 200), augment):
            hS = ctx.shape(synth.rotate_points(A.xyz, s_q), A.level)
            qs = torch.tensor(synth.compose_quaternions(s_q, q).astype(np.float32), device=dev)
            Xs.append(net.features(qs, bc.moments(ctx, hS), ligand(hB, qs, fb)))
            ts.append(z)
            hS.close()
        hA.close()
        hB.close()
    return torch.cat(Xs).contiguous(), torch.cat(ts).contiguous()


# the ligand's moments as given (the same for every rotation) or turned by each rotation
@pytest.mark.parametrize("rotated", [False, True])
def test_trained_network_beats_random_choice_on_held_out_pairs(bc, rotated):
    dev = torch.device("cuda", 0)
    N, W, H, K = 32, 6, 64, 64
    ctx = bc.Context(N, W, synth.RADII_4)
    ctx.set_tuning(spread=1)  # fixed-point spreading sums: bit-reproducible labels
    net = bc.MLP(ctx, H, synth.mlp_init(H, 3), rotated_moments=rotated)
    X, T = labelled(bc, ctx, net, range(1, 9), 1024, 8, dev, rotated)
    X2, T2 = labelled(bc, ctx, net, range(1, 9), 1024, 8, dev, rotated)
    assert torch.equal(X, X2) and torch.equal(T, T2)  # the labels are reproducible
    loss = torch.empty(1, device=dev)
    net.train(X, T, epochs=40, batch=1024, lr=3e-3, seed=5, loss=loss)
    ctx.sync()
    print(f"training: {X.shape[0]} samples, final batch loss {float(loss.item()):.3f}")
    learned, rand, rhos, over, over_rand, zsel, zrand = [], [], [], [], [], [], []
    R = 4096
    for seed in range(101, 107):
        A, B = pair(seed)
        hA, hB = ctx.shape(A.xyz, A.level), ctx.shape(B.xyz, B.level)
        q = synth.shoemake_quaternions(synth.SplitMix64(seed + 300), R).astype(np.float32)
        peak, _ = ctx.sweep(hA, hB, q, batch=128)
        p = peak.cpu().numpy().astype(np.float64)
        idx, psel, _, scores = bc.learned_sweep(ctx, net, hA, hB, torch.tensor(q, device=dev), K)
        ctx.sync()
        s = scores.cpu().numpy().astype(np.float64)
        chosen = idx.cpu().numpy()
        # the learned sweep's peaks are the exhaustive sweep's peaks of the chosen rotations
        np.testing.assert_allclose(psel.cpu().numpy(), p[chosen], rtol=1e-5, atol=1e-6 * np.abs(p).max())
        learned.append(p[chosen].max() / p.max())
        rnd = np.argsort(synth.SplitMix64(seed + 400).uniform(R))[:K]
        rand.append(p[rnd].max() / p.max())
        rhos.append(spearman(s, p))
        top = set(np.argsort(-p, kind="stable")[:K].tolist())  # the K best rotations by their true peaks
        over.append(len(top & set(chosen.tolist())) / K)
        over_rand.append(len(top & set(rnd.tolist())) / K)
        z = (p - p.mean()) / p.std()
        zsel.append(float(z[chosen].mean()))
        zrand.append(float(z[rnd].mean()))
        print(f"pair {seed}: best-in-top-{K} / best {learned[-1]:.4f} (random {rand[-1]:.4f}), "
              f"rank correlation {rhos[-1]:.3f}, true top-{K} found {over[-1]:.3f} (random {over_rand[-1]:.3f}), "
              f"mean standardised peak of the picks {zsel[-1]:.2f} (random {zrand[-1]:.2f})")
        hA.close()
        hB.close()
    print(f"mean best-in-top-{K} / best: learned {np.mean(learned):.4f}, random {np.mean(rand):.4f}; "
          f"mean rank correlation {np.mean(rhos):.3f}; true top-{K} found {np.mean(over):.3f} "
          f"(random {np.mean(over_rand):.3f}, expected {K / R:.3f}); mean standardised peak of the picks "
          f"{np.mean(zsel):.2f} (random {np.mean(zrand):.2f})")
    # what the network gains: its ranking follows the true peaks (a random order has
    # rank correlation 0), and the rotations it picks have peaks well above those of
    # a random choice of the same number (whose standardised mean is 0 +- 1/sqrt(K))
    assert np.mean(rhos) > 0.3
    assert np.mean(zsel) > 0.5 and np.mean(zsel) > np.mean(zrand) + 0.5
    net.close()
    ctx.close()


def test_multi_step_training_matches_single_steps_and_is_deterministic(bc):
    dev = torch.device("cuda", 0)
    H, n = 64, 2048
    rng = synth.SplitMix64(11)
    q = synth.shoemake_quaternions(rng, n).astype(np.float32)
    fa, fb = rng.uniform(64).astype(np.float32), rng.uniform(64).astype(np.float32)
    t = torch.tensor((np.sin(3 * q[:, 1]) + q[:, 2] * q[:, 3]).astype(np.float32), device=dev)
    ctx = bc.Context(32, 6, synth.RADII_2)
    init = synth.mlp_init(H, 4)
    nets = [bc.MLP(ctx, H, init) for _ in range(3)]
    X = nets[0].features(torch.tensor(q, device=dev), torch.tensor(fa, device=dev), torch.tensor(fb, device=dev))
    # one pass with the whole set as the batch: the same gradient as one single step
    # (the order of the rows only changes the rounding of the sums)
    nets[0].train(X, t, epochs=1, batch=n, lr=1e-3, seed=9)
    nets[1].train_step(X, t, 1e-3)
    a, b = nets[0].state(), nets[1].state()
    assert a["step"] == b["step"] == 1
    # the first moments are (1 - beta1) times the two gradients
    m_ref = b["adam_m"]
    np.testing.assert_allclose(a["adam_m"], m_ref, rtol=1e-4, atol=1e-5 * float(np.abs(m_ref).max()))
    # many passes twice from the same start: bit-identical, and the loss falls
    nets[2].load_state({"params": init, "adam_m": np.zeros_like(init), "adam_v": np.zeros_like(init), "step": 0})
    _, loss0 = nets[2].grads(X, t)
    loss = torch.empty(1, device=dev)
    for k in (0, 2):
        nets[k].load_state({"params": init, "adam_m": np.zeros_like(init), "adam_v": np.zeros_like(init), "step": 0})
        nets[k].train(X, t, epochs=20, batch=256, lr=3e-3, seed=9, loss=loss)
    a, c = nets[0].state(), nets[2].state()
    assert a["step"] == c["step"] == 20 * (n // 256)
    np.testing.assert_array_equal(a["params"], c["params"])
    print(f"loss {float(loss0.item()):.4f} -> {float(loss.item()):.4f}")
    assert float(loss.item()) < 0.3 * float(loss0.item())
    for net in nets:
        net.close()
    ctx.close()


def test_coarse_stage_matches_its_composed_calls(bc):
    # bc_learned_sweep_coarse against the same stages composed from single calls:
    # network scores -> top coarse_keep -> coarse sweep (N = 32) -> top K -> full
    # sweep (N = 64).  The coarse context runs on a stream of its own (the entry
    # point orders the two streams with events).  Fixed-point spreading on both
    # contexts: the peaks do not depend on the batches, so both sides agree bit for bit.
    dev = torch.device("cuda", 0)
    ctx = bc.Context(64, 6, synth.RADII_4)
    ctxc = bc.Context(32, 6, synth.RADII_4, stream=torch.cuda.Stream(dev))
    ctx.set_tuning(spread=1)
    ctxc.set_tuning(spread=1)
    net = bc.MLP(ctx, 64, synth.mlp_init(64, 13))
    A, B = pair(41)
    hA, hB = ctx.shape(A.xyz, A.level), ctx.shape(B.xyz, B.level)
    hAc, hBc = ctxc.shape(A.xyz, A.level), ctxc.shape(B.xyz, B.level)
    R, M, K = 2048, 256, 32
    q = synth.shoemake_quaternions(synth.SplitMix64(17), R).astype(np.float32)
    qd = torch.tensor(q, device=dev)
    idx, peak, arg, scores = bc.learned_sweep(ctx, net, hA, hB, qd, K, coarse=(ctxc, hAc, hBc, M))
    torch.cuda.synchronize(dev)
    # the composed reference
    s_ref = net.predict(net.features(qd, bc.moments(ctx, hA), bc.moments(ctx, hB)))
    iM = torch.empty(M, dtype=torch.int32, device=dev)
    bc.bc_topk(ctx.handle, s_ref, R, M, iM)
    torch.cuda.synchronize(dev)
    pc, _ = ctxc.sweep(hAc, hBc, q[iM.cpu().numpy()])
    torch.cuda.synchronize(dev)
    iK = torch.empty(K, dtype=torch.int32, device=dev)
    bc.bc_topk(ctx.handle, pc, M, K, iK)
    torch.cuda.synchronize(dev)
    sel = iM.cpu().numpy()[iK.cpu().numpy()]
    p_ref, a_ref = ctx.sweep(hA, hB, q[sel])
    torch.cuda.synchronize(dev)
    assert torch.equal(scores, s_ref)
    np.testing.assert_array_equal(idx.cpu().numpy(), sel)
    np.testing.assert_array_equal(peak.cpu().numpy(), p_ref.cpu().numpy())
    np.testing.assert_array_equal(arg.cpu().numpy(), a_ref.cpu().numpy())
    # the ranking is by coarse peak: the picks' coarse peaks are the largest M..K of them
    pcs = np.sort(pc.cpu().numpy())[::-1]
    got = pc.cpu().numpy()[iK.cpu().numpy()]
    np.testing.assert_array_equal(np.sort(got)[::-1], pcs[:K])
    with pytest.raises(bc.BallCorrError):  # topk above coarse_keep
        bc.learned_sweep(ctx, net, hA, hB, qd, M + 1, coarse=(ctxc, hAc, hBc, M))
    with pytest.raises(bc.BallCorrError):  # coarse shapes swapped (other knot counts)
        bc.learned_sweep(ctx, net, hA, hB, qd, K, coarse=(ctxc, hBc, hAc, M))
    for h in (hA, hB, hAc, hBc):
        h.close()
    net.close()
    ctxc.close()
    ctx.close()


def test_coarse_stage_finds_the_exhaustive_best(bc):
    # What the coarse stage gains at a small size: ranking every rotation by its peak
    # at the coarse band limit (N = 32; coarse_keep = n, so the network does not
    # matter) puts the exhaustive best at full resolution (N = 64) among the K picks,
    # where a random choice of K holds it with probability K / R.
    dev = torch.device("cuda", 0)
    ctx = bc.Context(64, 6, synth.RADII_4)
    ctxc = bc.Context(32, 6, synth.RADII_4)
    ctx.set_tuning(spread=1)
    ctxc.set_tuning(spread=1)
    net = bc.MLP(ctx, 64, synth.mlp_init(64, 13))
    R, K = 4096, 64
    hits, ratios = 0, []
    for seed in range(201, 207):
        A, B = pair(seed)
        hA, hB = ctx.shape(A.xyz, A.level), ctx.shape(B.xyz, B.level)
        hAc, hBc = ctxc.shape(A.xyz, A.level), ctxc.shape(B.xyz, B.level)
        q = synth.shoemake_quaternions(synth.SplitMix64(seed + 300), R).astype(np.float32)
        peak, _ = ctx.sweep(hA, hB, q, batch=256)
        p = peak.cpu().numpy().astype(np.float64)
        best = int(np.argmax(p))
        idx, psel, _, _ = bc.learned_sweep(ctx, net, hA, hB, torch.tensor(q, device=dev), K,
                                           coarse=(ctxc, hAc, hBc, R))
        torch.cuda.synchronize(dev)
        chosen = idx.cpu().numpy()
        hits += best in set(chosen.tolist())
        ratios.append(float(psel.max()) / p[best])
        print(f"pair {seed}: exhaustive best in the coarse top-{K}: {best in set(chosen.tolist())}, "
              f"best picked / best {ratios[-1]:.5f}")
        for h in (hA, hB, hAc, hBc):
            h.close()
    print(f"coarse stage: {hits} of 6 (a random choice of {K} of {R}: {K / R:.3f} expected)")
    assert hits >= 5 and min(ratios) > 0.99
    net.close()
    ctxc.close()
    ctx.close()


def test_coarse_stage_after_orientation_average_ranks_the_cascade_picks(bc):
    # With orientations, the network's ranking is bc_learned_sweep_cascade's (one view,
    # then the orientation average for the best `keep`); the coarse stage must take
    # exactly the cascade's best coarse_keep, and pick its K among them by coarse peak.
    dev = torch.device("cuda", 0)
    ctx = bc.Context(64, 6, synth.RADII_4)
    ctxc = bc.Context(32, 6, synth.RADII_4)
    ctx.set_tuning(spread=1)
    ctxc.set_tuning(spread=1)
    net = bc.MLP(ctx, 64, synth.mlp_init(64, 19), rotated_moments=True)
    A, B = pair(43)
    hA, hB = ctx.shape(A.xyz, A.level), ctx.shape(B.xyz, B.level)
    hAc, hBc = ctxc.shape(A.xyz, A.level), ctxc.shape(B.xyz, B.level)
    R, keep, M, K = 2048, 512, 128, 16
    q = synth.shoemake_quaternions(synth.SplitMix64(23), R).astype(np.float32)
    qd = torch.tensor(q, device=dev)
    orients = synth.shoemake_quaternions(synth.SplitMix64(29), 3).astype(np.float32)
    iM, _, _, s1 = bc.learned_sweep(ctx, net, hA, hB, qd, M, orientations=orients, keep=keep)
    idx, peak, _, s2 = bc.learned_sweep(ctx, net, hA, hB, qd, K, orientations=orients, keep=keep,
                                        coarse=(ctxc, hAc, hBc, M))
    torch.cuda.synchronize(dev)
    assert torch.equal(s1, s2)  # the same one-view scores
    cand = iM.cpu().numpy()
    got = idx.cpu().numpy()
    assert set(got.tolist()) <= set(cand.tolist()) and len(set(got.tolist())) == K
    pc, _ = ctxc.sweep(hAc, hBc, q[cand])
    pc = pc.cpu().numpy()
    order = cand[np.argsort(-pc, kind="stable")[:K]]  # coarse ranking, ties to the earlier candidate
    np.testing.assert_array_equal(got, order)
    pf, _ = ctx.sweep(hA, hB, q[got])
    np.testing.assert_array_equal(peak.cpu().numpy(), pf.cpu().numpy())
    for h in (hA, hB, hAc, hBc):
        h.close()
    net.close()
    ctxc.close()
    ctx.close()
