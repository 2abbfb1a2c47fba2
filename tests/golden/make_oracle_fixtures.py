"""Writes oracle_regression.txt: values of the FP64 oracle on a small hand-written
configuration, as a regression fixture of the oracle (a later change to the oracle's
arithmetic shows up as a mismatch and must be justified by the passage it follows).
This is not an independent pin: the pins are the closed forms, quadratures and
invariants of test_oracle_pins.py.  It calls only oracle/.

Quantities (paper references by section and equation label):
  lens    two-ball intersection volume V(r1, r2, d)      (Sec. 3.1, Eq. (relg) with indicator balls)
  ballft  4 pi (sin kr - kr cos kr) / k^3 and its series (Sec. 2.5, Eq. (fballhat))
  exact   layer (a): periodised sum of lens volumes       (Sec. 3.1, Eq. (relg))
  band    layer (b): band-limited correlation, N = 8      (Sec. 3.2, Eq. (ccghat); App. C)

Run from the repository root:  python tests/golden/make_oracle_fixtures.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402


class _Shape:
    def __init__(self, xyz, level, radii):
        self.xyz, self.level, self.radii = np.asarray(xyz, float), np.asarray(level, np.int32), tuple(radii)


RADII = (0.05, 0.11)
A = _Shape([[0.10, -0.20, 0.05], [0.25, 0.00, -0.10], [-0.30, 0.15, 0.20]], [0, 1, 1], RADII)
B = _Shape([[-0.05, 0.10, 0.00], [0.20, -0.25, 0.15]], [1, 0], RADII)
Q = np.array([0.9, 0.1, -0.3, 0.2]) / np.linalg.norm([0.9, 0.1, -0.3, 0.2])
# translations near c_i - R c_j (overlapping balls), one far from every pair, one across the period
OFFS = np.array([[0.01, -0.02, 0.015], [-0.03, 0.0, 0.02], [0.0, 0.04, -0.01], [0.5, 0.5, 0.5], [0.02, 0.01, 0.0]])
LENS = [(0.1, 0.05, 0.0), (0.1, 0.05, 0.07), (0.1, 0.1, 0.1), (0.08, 0.05, 0.12), (0.1, 0.05, 0.2)]
BALLFT = [(0.05, 0.0), (0.05, 9.0), (0.05, 10.5), (0.11, 30.0), (0.08, 200.0)]
IDX = [0, 37, 100, 255, 511]


def values():
    rows = []
    for r1, r2, d in LENS:
        rows.append(("lens", (r1, r2, d), float(O.lens_volume(r1, r2, d))))
    for r, k in BALLFT:
        rows.append(("ballft", (r, k), float(O.ball_ft(r, k))))
    ra = np.array(RADII)[A.level]
    rb = np.array(RADII)[B.level]
    RB = O.rotate(B.xyz, Q)
    T = np.array([A.xyz[0] - RB[0], A.xyz[1] - RB[1], A.xyz[2] - RB[0], A.xyz[0] - RB[1], A.xyz[2] - RB[1] + 2.0]) + OFFS
    ex = O.exact_corr(A.xyz, ra, B.xyz, rb, T, Q)
    for t, v in zip(T, ex):
        rows.append(("exact", tuple(t), float(v)))
    band = O.band_limited_corr(A, B, Q, 8, idx=np.array(IDX))
    for i, v in zip(IDX, band):
        rows.append(("band", (i,), float(v)))
    return rows


def main():
    with open(os.path.join(HERE, "oracle_regression.txt"), "w") as f:
        f.write("# kind  arguments  value  (see make_oracle_fixtures.py for the configuration and citations)\n")
        for kind, args, v in values():
            f.write(f"{kind} {' '.join(repr(float(a)) for a in args)} {v!r}\n")


if __name__ == "__main__":
    main()
