"""GPU lifted (4D) nonequiradius correlation (Sec. 3.2) against the FP64 oracle.

Knots with individual radii in (0, L); sections r = 0 (the obstacle of the
ball unions) and offsets.  Bar rel-L2 <= 1e-5 per section.
"""
import numpy as np
import pytest

import oracle as O
from paper_1711_05075_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_TOL = 1e-5
L, P, PR = 0.1, 2.0, 0.4


@pytest.fixture(scope="module")
def bc():
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    torch.cuda.set_device(0)
    import paper_1711_05075_gb300 as m
    return m


def knots(shape, seed, lo=0.01, hi=0.09):
    """(n, 4) float32 (x, y, z, r): a seeded shape's centres with radii uniform in [lo, hi)."""
    rng = synth.SplitMix64(seed)
    r = lo + (hi - lo) * rng.uniform(shape.xyz.shape[0])
    return np.concatenate([shape.xyz, r[:, None]], axis=1).astype(np.float32)


def oracle(A, B, q, N, Nr, slices, idx=None):
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    g = O.lifted_corr_spectrum((A64[:, :3], A64[:, 3]), (B64[:, :3], B64[:, 3]), q.astype(np.float64), N, Nr, L, P, PR)
    return O.lifted_slices(g, [float(np.float32(s)) for s in slices], P, PR)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# tcgen05: tcgen05.mma with tensor-memory accumulators; mma: legacy mma.sync; both
# 3-pass split TF32.  cuda: FP32 on the CUDA cores.
@pytest.mark.parametrize("contraction", ["tcgen05", "mma", "cuda"])
@pytest.mark.parametrize("N,Nr,nA,nB,slices", [(32, 32, 6, 6, (0.0, 0.03, -0.02)),
                                                 (32, 16, 2000, 1500, (0.0, 0.04)),
                                                 (32, 8, 12000, 7000, (0.0, 0.05)),
                                                 (32, 8, 40000, 3000, (0.0,)),  # two passes of 32,768 knots
                                                 (64, 16, 800, 600, (0.0,)),
                                                 (96, 8, 300, 200, (0.0, 0.03)),
                                                 (128, 8, 200, 150, (0.0,))])
def test_lifted_sections_match_oracle(bc, N, Nr, nA, nB, slices, contraction):
    A = knots(synth.ellipsoid_shape(nA, 40 + nA), 1)
    B = knots(synth.torus_shape(nB, 41 + nB), 2)
    q = synth.shoemake_quaternions(synth.SplitMix64(42), 1)[0].astype(np.float32)
    lf = bc.Lift(N, Nr, L, P, PR, contraction=contraction)
    got = lf.correlate(A, B, q, slices).double().cpu().numpy()
    ref = oracle(A, B, q, N, Nr, slices)
    for s, rs in enumerate(slices):
        e = rel(got[s], ref[s])
        print(f"lifted N={N} Nr={Nr} {nA}+{nB} knots, contraction {contraction}, section {rs}: rel-L2 {e:.3e}")
        assert e <= REL_TOL
    host = lf.correlate_host(A, B, q, slices)
    assert rel(host.astype(np.float64), got) < 1e-6  # split-knot partial sums add in another order
    lf.close()


# the 4D type-1 NUFFT (contraction 3): spreading onto the (2N)^3 x 2Nr grid, 4D FFT,
# deconvolution; the same sections as the direct NDFT within the same bar
@pytest.mark.parametrize("N,Nr,nA,nB,slices", [(32, 32, 6, 6, (0.0, 0.03, -0.02)),
                                                 (32, 16, 2000, 1500, (0.0, 0.04)),
                                                 (64, 16, 800, 600, (0.0,)),
                                                 (64, 32, 3000, 2000, (0.0, 0.02)),
                                                 (96, 16, 300, 200, (0.0, 0.03)),
                                                 (128, 16, 200, 150, (0.0,))])
def test_lifted_nufft_matches_oracle_and_the_direct_form(bc, N, Nr, nA, nB, slices):
    A = knots(synth.ellipsoid_shape(nA, 40 + nA), 1)
    B = knots(synth.torus_shape(nB, 41 + nB), 2)
    q = synth.shoemake_quaternions(synth.SplitMix64(42), 1)[0].astype(np.float32)
    lf = bc.Lift(N, Nr, L, P, PR, contraction="nufft")
    got = lf.correlate(A, B, q, slices).double().cpu().numpy()
    lf.close()
    ref = oracle(A, B, q, N, Nr, slices)
    direct = bc.Lift(N, Nr, L, P, PR, contraction="tcgen05")
    gd = direct.correlate(A, B, q, slices).double().cpu().numpy()
    direct.close()
    for s, rs in enumerate(slices):
        e, ed = rel(got[s], ref[s]), rel(got[s], gd[s])
        print(f"lifted NUFFT N={N} Nr={Nr} {nA}+{nB} knots, section {rs}: rel-L2 {e:.3e} (against the tcgen05 "
              f"NDFT {ed:.3e})")
        assert e <= REL_TOL and ed <= REL_TOL


def test_lifted_nufft_box_falls_back_to_whole_axes(bc):
    # knots on both sides of the period boundary in x (and spread over all of z): the
    # support box of those axes is the whole axis, the others stay boxes; radii outside
    # (0, L) as well (the r box then widens, still without wrapping errors)
    N, Nr = 32, 16
    rng = synth.SplitMix64(77)
    n = 300
    xyz = np.stack([0.97 * np.sign(rng.uniform(n) - 0.5), 0.3 * (rng.uniform(n) - 0.5), 1.9 * (rng.uniform(n) - 0.5)],
                   axis=1)
    r = 0.01 + 0.15 * rng.uniform(n)
    A = np.concatenate([xyz, r[:, None]], axis=1).astype(np.float32)
    B = knots(synth.torus_shape(250, 79), 80)
    q = synth.shoemake_quaternions(synth.SplitMix64(81), 1)[0].astype(np.float32)
    slices = (0.0, 0.05)
    lf = bc.Lift(N, Nr, L, P, PR, contraction="nufft")
    got = lf.correlate(A, B, q, slices).double().cpu().numpy()
    lf.close()
    ref = oracle(A, B, q, N, Nr, slices)
    for s, rs in enumerate(slices):
        e = rel(got[s], ref[s])
        print(f"lifted NUFFT, knots across the period boundary, section {rs}: rel-L2 {e:.3e}")
        assert e <= REL_TOL


def test_lifted_arguments(bc):
    with pytest.raises(bc.BallCorrError) as e:
        bc.Lift(48, 16, L)
    assert e.value.status == 5
    lf = bc.Lift(32, 8, L)
    A = knots(synth.ellipsoid_shape(10, 3), 4)
    with pytest.raises(bc.BallCorrError):
        lf.correlate(A, A, np.zeros(4, np.float32))
    with pytest.raises(bc.BallCorrError):
        lf.correlate(A, A, synth.IDENTITY_QUAT[0], slices=np.zeros(17))
    with pytest.raises(bc.BallCorrError) as e:
        bc.Lift(32, 8, L, contraction=4)
    assert e.value.status == 1
    with pytest.raises(bc.BallCorrError) as e:  # the 4D NUFFT needs Nr >= 16
        bc.Lift(32, 8, L, contraction=3)
    assert e.value.status == 5
    # empty shapes give zero
    z = lf.correlate(np.zeros((0, 4), np.float32), A, synth.IDENTITY_QUAT[0])
    assert float(z.abs().max()) == 0.0
    lf.close()
