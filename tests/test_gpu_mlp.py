"""GPU learned proposal: forward, gradients and Adam against the FP64 MLP oracle
(BF16 rounding emulated where the GPU rounds), moment features (of the shapes
as given and turned by rotations) against the spectrum oracle, top-k against a stable sort, checkpoint/resume, and the
learned sweep against the plain sweep of the same rotations."""
import ctypes

import numpy as np
import pytest

import oracle as O
from oracle import mlp as M
from paper_1711_05075_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-2  # rel-L2 per parameter tensor (BF16 operands, FP32 accumulation)


@pytest.fixture(scope="module")
def bc():
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    torch.cuda.set_device(0)
    import paper_1711_05075_gb300 as m
    return m


def split(flat, H):
    o = 0
    out = {}
    for k, shape in (("W1", (H, 132)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", (1,))):
        size = int(np.prod(shape))
        out[k] = np.asarray(flat[o:o + size], dtype=np.float64).reshape(shape)
        o += size
    return out


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-30))


def problem(H=64, n=200, seed=0):
    init = synth.mlp_init(H, seed)
    rng = synth.SplitMix64(seed + 1)
    q = synth.shoemake_quaternions(rng, n)
    fa, fb = rng.uniform(64), rng.uniform(64)
    t = (np.sin(3 * q[:, 1]) + q[:, 2] * q[:, 3] + 0.1 * fa.sum()).astype(np.float32)
    return init, q.astype(np.float32), fa.astype(np.float32), fb.astype(np.float32), t


# (hidden, batch): ragged row tiles (200, 203 = 4 k + 3), 20,000 rows (forward on
# 256-column tiles), hidden 1024 (weight gradients on 128-column tiles)
@pytest.mark.parametrize("H,n", [(64, 200), (256, 200), (64, 203), (256, 20000), (1024, 200)])
def test_forward_and_gradients_match_oracle(bc, H, n):
    init, q, fa, fb, t = problem(H, n)
    ctx = bc.Context(32, 6, synth.RADII_2)
    net = bc.MLP(ctx, H, init)
    dev = torch.device("cuda")
    X = net.features(torch.tensor(q, device=dev), torch.tensor(fa, device=dev), torch.tensor(fb, device=dev))
    Xh = X.cpu().numpy()
    Xo = M.features(q.astype(np.float64), fa.astype(np.float64), fb.astype(np.float64))
    np.testing.assert_allclose(Xh[:, :132], Xo, rtol=1e-6, atol=1e-7)
    assert np.all(Xh[:, 132:] == 0)
    y = net.predict(X).cpu().numpy()
    p = split(init, H)
    yo, _ = M.forward(p, Xh[:, :132].astype(np.float64), bf=True)
    assert rel(y, yo) < 1e-3, rel(y, yo)  # FP32 accumulation of BF16 products
    g, loss = net.grads(X, torch.tensor(t, device=dev))
    g = split(g.cpu().numpy(), H)
    lo, go = M.loss_and_grads(p, Xh[:, :132].astype(np.float64), t.astype(np.float64), bf=True)
    assert abs(float(loss.item()) - lo) <= 1e-4 * abs(lo)
    for k in go:
        r = rel(g[k], go[k])
        print(f"H={H} n={n} grad {k}: rel-L2 {r:.2e}")
        assert r < GRAD_TOL, (k, r)
    net.close()
    ctx.close()


def test_adam_steps_match_oracle(bc):
    # Three consecutive updates: from the second step on m^/sqrt(v^) is no longer
    # sign(g), so swapped betas or a missing bias correction would show.
    H = 64
    init, q, fa, fb, t = problem(H, seed=3)
    ctx = bc.Context(32, 6, synth.RADII_2)
    net = bc.MLP(ctx, H, init)
    dev = torch.device("cuda")
    X = net.features(torch.tensor(q, device=dev), torch.tensor(fa, device=dev), torch.tensor(fb, device=dev))
    td = torch.tensor(t, device=dev)
    p = split(init, H)
    state = {}
    for step in range(1, 4):
        g, _ = net.grads(X, td)  # the gradient the update will use (same parameters, same batch)
        net.train_step(X, td, 1e-3)
        st = net.state()
        # the kernel holds the hyperparameters as FP32 values: 1 - float32(0.999) differs from
        # 1e-3 by 1.3e-5 relative, so the oracle is given the same rounded betas
        M.adam_step(p, split(g.cpu().numpy(), H), state, lr=float(np.float32(1e-3)),
                    beta1=float(np.float32(0.9)), beta2=float(np.float32(0.999)), eps=float(np.float32(1e-8)))
        got = split(st["params"], H)
        gm, gv = split(st["adam_m"], H), split(st["adam_v"], H)
        for k in p:
            np.testing.assert_allclose(got[k], p[k], rtol=1e-5, atol=1e-6, err_msg=f"step {step} {k}")
            for name, mine in (("m_", gm), ("v_", gv)):  # the moment recurrences themselves
                ref = state[name + k]
                np.testing.assert_allclose(mine[k], ref, rtol=1e-5, atol=1e-6 * float(np.abs(ref).max()),
                                           err_msg=f"step {step} {name}{k}")
        assert st["step"] == step
        # continue the oracle from the GPU's parameters so rounding does not accumulate
        p = {k: got[k].copy() for k in got}
    net.close()
    ctx.close()


def test_training_reduces_loss_and_resume_is_exact(bc):
    H = 64
    init, q, fa, fb, t = problem(H, n=512, seed=5)
    ctx = bc.Context(32, 6, synth.RADII_2)
    dev = torch.device("cuda")
    qd, fad, fbd, td = (torch.tensor(a, device=dev) for a in (q, fa, fb, t))
    net = bc.MLP(ctx, H, init)
    X = net.features(qd, fad, fbd)
    loss = torch.empty(1, device=dev)
    net.grads(X, td)
    first = None
    for i in range(200):
        net.train_step(X, td, 3e-3, loss)
        if i == 0:
            first = float(loss.item())
        if i == 99:
            ckpt = net.state()
    last = float(loss.item())
    final = net.state()["params"]
    print(f"loss {first:.4f} -> {last:.4f}")
    assert last < 0.3 * first
    net2 = bc.MLP(ctx, H, init)
    net2.load_state(ckpt)
    for i in range(100):
        net2.train_step(X, td, 3e-3)
    np.testing.assert_array_equal(net2.state()["params"], final)  # deterministic resume
    net.close()
    net2.close()
    ctx.close()


def test_moments_match_oracle(bc):
    wl = synth.small_pair(2)
    ctx = bc.Context(wl.N, wl.W, wl.radii)
    for S in (wl.A, wl.B):
        h = ctx.shape(S.xyz, S.level)
        got = bc.moments(ctx, h).cpu().numpy()
        spec = O.shape_spectrum(S.xyz.astype(np.float32).astype(np.float64), S.level, S.radii, wl.N)
        ref = M.moments(spec, M.moment_modes(wl.N))
        np.testing.assert_allclose(got, ref, rtol=5e-5, atol=1e-7)
        h.close()
    ctx.close()


def test_rotated_moments_match_oracle(bc):
    # |f^_B(R^T m)| / f^_B(0) by direct sums on the device against the oracle's
    # spectrum of the turned shape (layer (b)), for the identity, random rotations,
    # an unnormalised quaternion and one with w < 0; a zero quaternion is reported.
    wl = synth.small_pair(2)
    ctx = bc.Context(wl.N, wl.W, wl.radii)
    qs = np.concatenate([[[1.0, 0, 0, 0]], synth.shoemake_quaternions(synth.SplitMix64(21), 5),
                         [[0.0, 3.0, -4.0, 0.0], [-0.5, 0.5, 0.5, 0.5]]]).astype(np.float32)
    for S in (wl.A, wl.B):
        h = ctx.shape(S.xyz, S.level)
        got = bc.moments_rot(ctx, h, torch.tensor(qs, device="cuda")).cpu().numpy()
        ctx.sync()
        for r, q in enumerate(qs):
            spec = O.shape_spectrum(S.xyz.astype(np.float32).astype(np.float64), S.level, S.radii, wl.N,
                                    q=q.astype(np.float64))
            ref = M.moments(spec, M.moment_modes(wl.N))
            np.testing.assert_allclose(got[r], ref, rtol=2e-5, atol=2e-6)
        # the identity row is the pipeline's moments of the shape as given
        np.testing.assert_allclose(got[0], bc.moments(ctx, h).cpu().numpy(), rtol=5e-5, atol=1e-6)
        h.close()
    h = ctx.shape(wl.B.xyz, wl.B.level)
    bc.moments_rot(ctx, h, torch.zeros((2, 4), device="cuda"))
    with pytest.raises(bc.BallCorrError) as e:
        ctx.sync()
    assert e.value.status == 1
    ctx.sync()  # the word is cleared; the context stays usable
    h.close()
    ctx.close()


def test_learned_sweep_with_rotated_ligand_moments(bc):
    # a network set to take the rotated ligand's moments: the sweep's scores are the
    # network's predictions on [q, m_A, m_{R B}] built from moments_rot, with and
    # without orientation averaging (S A against S R B)
    wl = synth.small_pair(7)
    ctx = bc.Context(wl.N, wl.W, wl.radii)
    A, B = ctx.shape(wl.A.xyz, wl.A.level), ctx.shape(wl.B.xyz, wl.B.level)
    net = bc.MLP(ctx, 64, synth.mlp_init(64, 9), rotated_moments=True)
    assert net.rotated_moments
    qn = synth.shoemake_quaternions(synth.SplitMix64(4), 2000).astype(np.float32)
    q = torch.tensor(qn, device="cuda")
    idx, peak, arg, scores = bc.learned_sweep(ctx, net, A, B, q, 32)
    fa = bc.moments(ctx, A)
    ref = net.predict(net.features(q, fa, bc.moments_rot(ctx, B, q))).cpu().numpy()
    np.testing.assert_allclose(scores.cpu().numpy(), ref, rtol=1e-6, atol=1e-7)
    S = synth.shoemake_quaternions(synth.SplitMix64(11), 2)
    _, _, _, s_avg = bc.learned_sweep(ctx, net, A, B, q, 32, orientations=S.astype(np.float32))
    per = [ref]
    for s_q in S:
        hS = ctx.shape(synth.rotate_points(wl.A.xyz, s_q), wl.A.level)
        qs = torch.tensor(synth.compose_quaternions(s_q, qn).astype(np.float32), device="cuda")
        per.append(net.predict(net.features(qs, bc.moments(ctx, hS), bc.moments_rot(ctx, B, qs))).cpu().numpy())
        hS.close()
    # The rotations S R are composed in FP32 on the device here and in FP64 on the
    # host above, and the turned receptor's moments come from spectra whose
    # spreading sums round in a run-dependent order: features that differ in the
    # last bits, which the BF16 rounding of the network's inputs turns into steps
    # of about 2^-8 of a feature for the few that straddle a rounding boundary.
    ref_avg = np.mean(per, axis=0)
    d = np.abs(s_avg.cpu().numpy() - ref_avg)
    assert np.mean(d <= 1e-5 + 1e-4 * np.abs(ref_avg)) >= 0.99
    assert d.max() <= 5e-3 * np.abs(ref_avg).max()
    sel = qn[idx.cpu().numpy()]
    p2, _ = ctx.sweep(A, B, sel)
    np.testing.assert_allclose(peak.cpu().numpy(), p2.cpu().numpy(), rtol=1e-5)
    net.close(); A.close(); B.close(); ctx.close()


@pytest.mark.parametrize("rotated", [False, True])
def test_learned_sweep_cascade(bc, rotated):
    # bc_learned_sweep_cascade: with keep = n and no orientations it is the plain learned
    # sweep; with keep < n the picks come from the one-view top-keep, ranked by the mean
    # over the views (the turned receptor's moments by direct sums), and their peaks are
    # the plain sweep's peaks of the same rotations
    wl = synth.small_pair(7)
    ctx = bc.Context(wl.N, wl.W, wl.radii)
    ctx.set_tuning(spread=1)  # fixed-point spreading sums: spectra and peaks repeat bit for bit
    A, B = ctx.shape(wl.A.xyz, wl.A.level), ctx.shape(wl.B.xyz, wl.B.level)
    net = bc.MLP(ctx, 64, synth.mlp_init(64, 9), rotated_moments=rotated)
    qn = synth.shoemake_quaternions(synth.SplitMix64(4), 2000).astype(np.float32)
    q = torch.tensor(qn, device="cuda")
    i0, p0, a0, s0 = bc.learned_sweep(ctx, net, A, B, q, 32)
    i1, p1, a1, s1 = bc.learned_sweep(ctx, net, A, B, q, 32, keep=2000)
    np.testing.assert_array_equal(i1.cpu().numpy(), i0.cpu().numpy())
    np.testing.assert_array_equal(p1.cpu().numpy(), p0.cpu().numpy())
    np.testing.assert_array_equal(s1.cpu().numpy(), s0.cpu().numpy())
    S = synth.shoemake_quaternions(synth.SplitMix64(11), 3).astype(np.float32)
    keep = 300
    idx, peak, arg, sv = bc.learned_sweep(ctx, net, A, B, q, 32, orientations=S, keep=keep)
    sv = sv.cpu().numpy()
    np.testing.assert_array_equal(sv, s0.cpu().numpy())  # the one-view scores
    kept = np.lexsort((np.arange(sv.size), -sv))[:keep]
    chosen = idx.cpu().numpy()
    assert set(chosen.tolist()) <= set(kept.tolist())
    # the mean over the views, formed on the host (rotations composed in FP64)
    fo = bc.moments_rot(ctx, A, torch.tensor(S, device="cuda"))
    fb = bc.moments(ctx, B)
    q1 = qn[kept]
    views = [sv[kept]]
    for k, s_q in enumerate(S):
        qs = torch.tensor(synth.compose_quaternions(s_q, q1).astype(np.float32), device="cuda")
        lig = bc.moments_rot(ctx, B, qs) if rotated else fb
        views.append(net.predict(net.features(qs, fo[k].contiguous(), lig)).cpu().numpy())
    avg = np.mean(views, axis=0)
    top_host = set(kept[np.lexsort((np.arange(keep), -avg))[:32]].tolist())
    assert len(top_host & set(chosen.tolist())) >= 29  # near the cut the last bits may reorder a pick
    p2, _ = ctx.sweep(A, B, qn[chosen])
    np.testing.assert_allclose(peak.cpu().numpy(), p2.cpu().numpy(), rtol=1e-5)
    with pytest.raises(bc.BallCorrError):
        bc.learned_sweep(ctx, net, A, B, q, 32, orientations=S, keep=16)  # topk > keep
    net.close(); A.close(); B.close(); ctx.close()


def test_topk_is_a_stable_descending_selection(bc):
    rng = np.random.default_rng(0)
    ctx = bc.Context(32, 6, synth.RADII_2)
    for n, k in ((1000, 10), (16384, 256), (5, 5), (3, 1)):
        s = rng.integers(0, 50, size=n).astype(np.float32) * 0.5 - 7.0  # many ties, negatives
        ref = np.lexsort((np.arange(n), -s))[:k]
        idx = torch.empty(k, dtype=torch.int32, device="cuda")
        bc.bc_topk(ctx.handle, torch.tensor(s, device="cuda"), n, k, idx)
        np.testing.assert_array_equal(idx.cpu().numpy(), ref)
    ctx.close()


def test_learned_sweep_selects_and_scores_consistently(bc):
    wl = synth.small_pair(7)
    ctx = bc.Context(wl.N, wl.W, wl.radii)
    A, B = ctx.shape(wl.A.xyz, wl.A.level), ctx.shape(wl.B.xyz, wl.B.level)
    net = bc.MLP(ctx, 64, synth.mlp_init(64, 9))
    q = torch.tensor(synth.shoemake_quaternions(synth.SplitMix64(4), 3000).astype(np.float32), device="cuda")
    idx, peak, arg, scores = bc.learned_sweep(ctx, net, A, B, q, 40)
    s = scores.cpu().numpy()
    ref = np.lexsort((np.arange(s.size), -s))[:40]
    np.testing.assert_array_equal(idx.cpu().numpy(), ref)
    # the network's scores are its prediction on the documented features
    fa, fb = bc.moments(ctx, A), bc.moments(ctx, B)
    np.testing.assert_allclose(s, net.predict(net.features(q, fa, fb)).cpu().numpy(), rtol=1e-6)
    # the selected rotations' peaks equal the plain sweep's peaks for the same rotations
    sel = q.cpu().numpy()[ref]
    p2, a2 = ctx.sweep(A, B, sel)
    np.testing.assert_allclose(peak.cpu().numpy(), p2.cpu().numpy(), rtol=1e-5)
    net.close(); A.close(); B.close(); ctx.close()


def test_learned_sweep_orientation_averaging(bc):
    # bc_learned_sweep_avg: with no orientations it is the plain learned sweep; with
    # two it scores each rotation by the mean of the network's scores for the receptor
    # as given and turned by each orientation S (rotations S R), which the test forms
    # on the host: the receptor's knots rotated and uploaded, the rotations composed.
    wl = synth.small_pair(7)
    ctx = bc.Context(wl.N, wl.W, wl.radii)
    A, B = ctx.shape(wl.A.xyz, wl.A.level), ctx.shape(wl.B.xyz, wl.B.level)
    net = bc.MLP(ctx, 64, synth.mlp_init(64, 9))
    qn = synth.shoemake_quaternions(synth.SplitMix64(4), 3000).astype(np.float32)
    q = torch.tensor(qn, device="cuda")
    i0, p0, a0, s0 = bc.learned_sweep(ctx, net, A, B, q, 40)
    i1, p1, a1, s1 = bc.learned_sweep(ctx, net, A, B, q, 40, orientations=np.zeros((0, 4), np.float32))
    # (the moments come from spectra whose spreading sums round in a run-dependent order)
    np.testing.assert_allclose(s1.cpu().numpy(), s0.cpu().numpy(), rtol=1e-5, atol=1e-6)
    s1n = s1.cpu().numpy()
    np.testing.assert_array_equal(i1.cpu().numpy(), np.lexsort((np.arange(s1n.size), -s1n))[:40])
    S = synth.shoemake_quaternions(synth.SplitMix64(11), 2)
    fb = bc.moments(ctx, B)
    per = [s0.cpu().numpy()]
    for s_q in S:
        hS = ctx.shape(synth.rotate_points(wl.A.xyz, s_q), wl.A.level)
        qs = torch.tensor(synth.compose_quaternions(s_q, qn).astype(np.float32), device="cuda")
        per.append(net.predict(net.features(qs, bc.moments(ctx, hS), fb)).cpu().numpy())
        hS.close()
    ref = np.mean(per, axis=0)
    idx, peak, arg, sc = bc.learned_sweep(ctx, net, A, B, q, 40, orientations=S.astype(np.float32))
    s = sc.cpu().numpy()
    # the receptor is turned in FP32 on the device here and in FP64 on the host above
    np.testing.assert_allclose(s, ref, rtol=1e-3, atol=1e-4 * np.abs(ref).max())
    assert np.abs(s - s0.cpu().numpy()).max() > 1e-3 * np.abs(ref).max()  # the average differs from one view
    np.testing.assert_array_equal(idx.cpu().numpy(), np.lexsort((np.arange(s.size), -s))[:40])
    p2, _ = ctx.sweep(A, B, qn[idx.cpu().numpy()])
    np.testing.assert_allclose(peak.cpu().numpy(), p2.cpu().numpy(), rtol=1e-5)
    with pytest.raises(bc.BallCorrError):
        bc.learned_sweep(ctx, net, A, B, q, 40, orientations=np.zeros((1, 4), np.float32))
    net.close(); A.close(); B.close(); ctx.close()
