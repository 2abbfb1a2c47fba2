"""Seeded synthetic inputs: knot sets grouped into radius levels, and rotations.

This module only draws inputs. It holds none of the correlation arithmetic, so
the FP64 oracle and the CUDA path can both be fed from it without sharing any
step of the method.

Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state advances by the golden
gamma 0x9E3779B97F4A7C15 and each output is the state passed through the
published 64-bit finaliser.  A uniform double keeps the top 53 bits.

The shapes stand in for the paper's spherical decompositions of meshes
(Sec. 2.2-2.3, Sec. 5): every shape is a set of knots c_i in R^3, each with a
radius drawn from a small set of levels {rho_1..rho_L}, the grouping that lets
the equiradius form of Eq. (ballconv) apply level by level (Sec. 2.2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class SplitMix64:
    """Sequential splitmix64 stream; `uniform(k)` returns k doubles in [0, 1)."""

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def next_u64(self, k: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            steps = np.arange(1, k + 1, dtype=np.uint64)
            z = self.state + steps * _GAMMA
            self.state = self.state + np.uint64(k) * _GAMMA
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, k: int) -> np.ndarray:
        return (self.next_u64(k) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclass
class Shape:
    """A union of balls: knot centres `xyz` (n x 3, float64), level ids, radii per level."""

    xyz: np.ndarray
    level: np.ndarray
    radii: tuple
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def L(self) -> int:
        return len(self.radii)

    def r(self) -> np.ndarray:
        return np.asarray(self.radii, dtype=np.float64)[self.level]


# ---------------------------------------------------------------- point samplers
def _rejection(rng: SplitMix64, n: int, lo: np.ndarray, hi: np.ndarray, inside) -> np.ndarray:
    """Uniform points in a region by rejection from its bounding box (batched, deterministic)."""
    out = []
    have = 0
    while have < n:
        batch = max(1024, 2 * (n - have))
        u = rng.uniform(3 * batch).reshape(batch, 3)
        p = lo + (hi - lo) * u
        p = p[inside(p)]
        out.append(p)
        have += p.shape[0]
    return np.concatenate(out, axis=0)[:n]


def ellipsoid_points(rng, n, semi=(0.5, 0.35, 0.25), centre=(0.0, 0.0, 0.0), frame=None):
    """Uniform points inside an ellipsoid; `frame` (3x3 orthonormal columns) orients its axes."""
    a = np.asarray(semi, dtype=np.float64)
    c = np.asarray(centre, dtype=np.float64)
    F = np.eye(3) if frame is None else np.asarray(frame, dtype=np.float64)
    reach = float(a.max())
    lo, hi = c - reach, c + reach

    def inside(p):
        q = (p - c) @ F  # coordinates along the ellipsoid's axes
        return ((q / a) ** 2).sum(axis=1) <= 1.0

    return _rejection(rng, n, lo, hi, inside)


def torus_points(rng, n, R=0.4, r=0.12):
    """Uniform points inside a solid torus with axis z, tube radius r, centre-line radius R."""
    lo = np.array([-(R + r), -(R + r), -r])
    hi = -lo

    def inside(p):
        rho = np.sqrt(p[:, 0] ** 2 + p[:, 1] ** 2)
        return (rho - R) ** 2 + p[:, 2] ** 2 <= r * r

    return _rejection(rng, n, lo, hi, inside)


def draw_levels(rng, n, probs) -> np.ndarray:
    """Categorical level ids with the given probabilities."""
    cdf = np.cumsum(np.asarray(probs, dtype=np.float64))
    cdf /= cdf[-1]
    u = rng.uniform(n)
    return np.minimum(np.searchsorted(cdf, u, side="right"), len(cdf) - 1).astype(np.int32)


def random_frame(rng) -> np.ndarray:
    """A random orthonormal 3x3 frame from the QR factorisation of a uniform matrix."""
    m = rng.uniform(9).reshape(3, 3) - 0.5
    q, rr = np.linalg.qr(m)
    return q * np.sign(np.diag(rr))


def shoemake_quaternions(rng, k) -> np.ndarray:
    """k uniform random unit quaternions (w, x, y, z) by Shoemake's three-uniform method
    (K. Shoemake, "Uniform random rotations", Graphics Gems III, 1992)."""
    u = rng.uniform(3 * k).reshape(k, 3)
    a = np.sqrt(1.0 - u[:, 0])
    b = np.sqrt(u[:, 0])
    t1 = 2.0 * math.pi * u[:, 1]
    t2 = 2.0 * math.pi * u[:, 2]
    q = np.stack([b * np.cos(t2), a * np.sin(t1), a * np.cos(t1), b * np.sin(t2)], axis=1)
    q[q[:, 0] < 0] *= -1.0
    return q


IDENTITY_QUAT = np.array([[1.0, 0.0, 0.0, 0.0]])

# ------------------------------------------------------------- named workloads
RADII_2 = (0.04, 0.08)
PROBS_2 = (0.5, 0.5)
RADII_4 = (0.01, 0.02, 0.04, 0.08)
PROBS_4 = (0.4, 0.3, 0.2, 0.1)


def ellipsoid_shape(n, seed, radii=RADII_2, probs=PROBS_2, semi=(0.5, 0.35, 0.25)) -> Shape:
    rng = SplitMix64(seed)
    xyz = ellipsoid_points(rng, n, semi)
    lev = draw_levels(rng, n, probs)
    return Shape(xyz, lev, tuple(radii), f"ellipsoid{semi} n={n} seed={seed}")


def torus_shape(n, seed, radii=RADII_2, probs=PROBS_2, R=0.4, r=0.12) -> Shape:
    rng = SplitMix64(seed)
    xyz = torus_points(rng, n, R, r)
    lev = draw_levels(rng, n, probs)
    return Shape(xyz, lev, tuple(radii), f"torus(R={R},r={r}) n={n} seed={seed}")


def ellipsoid_union_shape(n, seed, radii=RADII_4, probs=PROBS_4, count=3) -> Shape:
    """Union of `count` random ellipsoids: centres U[-0.3,0.3]^3, semi-axes U[0.15,0.35],
    random orientation; knots uniform in the union (rejection from its bounding box)."""
    rng = SplitMix64(seed)
    parts = []
    for _ in range(count):
        c = rng.uniform(3) * 0.6 - 0.3
        a = rng.uniform(3) * 0.2 + 0.15
        parts.append((c, a, random_frame(rng)))

    def inside(p):
        ok = np.zeros(p.shape[0], dtype=bool)
        for c, a, F in parts:
            q = (p - c) @ F
            ok |= ((q / a) ** 2).sum(axis=1) <= 1.0
        return ok

    lo = np.min([c - a.max() for c, a, _ in parts], axis=0)
    hi = np.max([c + a.max() for c, a, _ in parts], axis=0)
    xyz = _rejection(rng, n, lo, hi, inside)
    lev = draw_levels(rng, n, probs)
    return Shape(xyz, lev, tuple(radii), f"ellipsoid-union({count}) n={n} seed={seed}")


@dataclass
class Workload:
    """One correlation problem: shapes A, B, rotations and the NUFFT parameters."""

    name: str
    A: Shape
    B: Shape
    quats: np.ndarray
    N: int
    W: int
    sigma: int = 2
    period: float = 2.0

    @property
    def radii(self):
        return self.A.radii


def small_pair(seed=0) -> Workload:
    """128-ball ellipsoid (semi-axes 0.5, 0.35, 0.25) vs 128-ball torus (R=0.4, r=0.12),
    levels {0.04, 0.08} drawn 50/50, identity rotation, 32^3 modes, KB width 6."""
    A = ellipsoid_shape(128, seed)
    B = torus_shape(128, seed + 1)
    return Workload("ellipsoid128-torus128-N32-W6", A, B, IDENTITY_QUAT.copy(), N=32, W=6)


def scale_pair(seed=0, N=128, W=8, n=20000) -> Workload:
    """20,000-ball ellipsoid vs 20,000-ball torus, levels {0.01,0.02,0.04,0.08} drawn with
    p = {0.4,0.3,0.2,0.1}, identity rotation, 128^3 modes (256^3 oversampled), KB width 8."""
    A = ellipsoid_shape(n, seed, RADII_4, PROBS_4)
    B = torus_shape(n, seed + 1, RADII_4, PROBS_4)
    return Workload(f"ellipsoid{n}-torus{n}-N{N}-W{W}", A, B, IDENTITY_QUAT.copy(), N=N, W=W)


def sweep_pair(seed=0, k=2048, n_rec=50000, n_lig=5000, N=96, W=8) -> Workload:
    """Receptor: union of 3 random ellipsoids (50,000 balls); ligand: torus (5,000 balls);
    L=4 levels as the 20k-ball pair; k Shoemake rotations; 96^3 grid; KB width 8."""
    A = ellipsoid_union_shape(n_rec, seed)
    B = torus_shape(n_lig, seed + 1, RADII_4, PROBS_4)
    q = shoemake_quaternions(SplitMix64(seed + 2), k)
    return Workload(f"union{n_rec}-torus{n_lig}-rot{k}-N{N}-W{W}", A, B, q, N=N, W=W)


def ragged_pairs(seed=0, npairs=64, lo=1000, hi=100000, N=96, W=8):
    """A ragged batch of `npairs` independent shape pairs whose knot counts are
    log-uniform in [lo, hi]: A_i a union of 3 random ellipsoids, B_i a torus, both
    with the L=4 levels of the 20k-ball pair, one Shoemake rotation per pair;
    96^3 grid, KB width 8.  Returns (pairs, quats) with pairs a list of (A_i, B_i)."""
    rng = SplitMix64(seed)
    u = rng.uniform(2 * npairs)
    counts = np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo))).astype(np.int64)
    pairs = []
    for i in range(npairs):
        A = ellipsoid_union_shape(int(counts[2 * i]), 10000 + 97 * seed + i)
        B = torus_shape(int(counts[2 * i + 1]), 20000 + 97 * seed + i, RADII_4, PROBS_4)
        pairs.append((A, B))
    q = shoemake_quaternions(SplitMix64(seed + 30000), npairs)
    return pairs, q


def translation_sample(N: int, count: int, seed: int = 0) -> np.ndarray:
    """`count` distinct linear indices into the N^3 translation grid (without replacement)."""
    rng = SplitMix64(seed)
    total = N ** 3
    count = min(count, total)
    keys = rng.next_u64(total) if total <= (1 << 22) else None
    if keys is not None:
        return np.sort(np.argsort(keys, kind="stable")[:count]).astype(np.int64)
    chosen = set()
    out = []
    while len(out) < count:
        for v in (rng.uniform(count) * total).astype(np.int64):
            if v not in chosen:
                chosen.add(int(v))
                out.append(int(v))
                if len(out) == count:
                    break
    return np.sort(np.asarray(out, dtype=np.int64))


def mlp_init(hidden: int, seed: int, in_features: int = 132) -> np.ndarray:
    """Initial network parameters (FP32, layout W1 [H][132], b1, W2 [H][H], b2, w3, b3):
    He-uniform weights U(-sqrt(6/fan_in), sqrt(6/fan_in)) from splitmix64, zero biases."""
    rng = SplitMix64(seed)
    H = hidden

    def u(fan_in, count):
        lim = math.sqrt(6.0 / fan_in)
        return (rng.uniform(count) * 2.0 - 1.0) * lim

    parts = [u(in_features, H * in_features), np.zeros(H), u(H, H * H), np.zeros(H), u(H, H), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


def compose_quaternions(s, q) -> np.ndarray:
    """Hamilton products s * q_i (rotation by q_i followed by s), canonicalised to w >= 0."""
    s = np.asarray(s, dtype=np.float64).reshape(4)
    q = np.asarray(q, dtype=np.float64).reshape(-1, 4)
    w1, x1, y1, z1 = s
    w2, x2, y2, z2 = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    out = np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                    w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                    w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                    w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], axis=1)
    out[out[:, 0] < 0] *= -1.0
    return out


def rotate_points(xyz, q) -> np.ndarray:
    """Input transform for augmentation: points rotated by the unit quaternion q (w, x, y, z)."""
    w, x, y, z = np.asarray(q, dtype=np.float64) / np.linalg.norm(q)
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    return np.asarray(xyz, dtype=np.float64) @ R.T
