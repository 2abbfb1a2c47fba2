"""Host side of bench.py (CPU): the workload it times, and the reference arm's
JSON line (the FP64 oracle on the whole workload, through the same code path
`bench.py --impl reference` runs)."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_workload_is_the_scale_pair():
    wl = bench.workload()
    assert (wl.A.n, wl.B.n, wl.N, wl.W, wl.sigma) == (20000, 20000, 128, 8, 2)
    assert tuple(wl.radii) == (0.01, 0.02, 0.04, 0.08)
    # level mix {0.4, 0.3, 0.2, 0.1} within sampling noise
    frac = np.bincount(wl.A.level, minlength=4) / wl.A.n
    assert np.all(np.abs(frac - [0.4, 0.3, 0.2, 0.1]) < 0.02)
    cfg = bench.config_of(wl)
    assert cfg["poses_per_step"] == 128 ** 3 and cfg["knots"] == [20000, 20000]


def test_kernel_source_hash_covers_existing_files():
    h1, h2 = bench.kernel_source_hash(), bench.kernel_source_hash()
    assert h1 == h2 and len(h1) == 16
    for f in bench.KERNEL_SOURCES:
        assert os.path.exists(os.path.join(ROOT, "paper_1711_05075_gb300", "csrc", f)), f


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "poses/s" and line["value"] > 0
    assert line["higher_is_better"] is True and line["dtype"] == "f64"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert cb["sample"].startswith("full workload") and "20000+20000 knots" in cb["sample"]
    # the timed steps are whole oracle runs: the line's time is what was measured
    assert line["warmup"] >= 3 and line["steps"] == 1 and line["ms_per_step"] > 0


def test_learned_target_picks_the_fastest_form_that_meets_it():
    ls = {"recall_best_in_topk": 0.4, "recall_within_1e-3_of_best": 0.6, "learned_vs_plain": 200.0,
          "ms_learned_sweep": 9.0,
          "cascade": {"recall_best": 0.75, "recall_within_1e-3": 0.85, "vs_plain": 97.0, "ms_learned_sweep": 19.0},
          "coarse": {"recall_best": 1.0, "recall_within_1e-3": 1.0, "vs_plain": 95.0, "ms_learned_sweep": 20.0},
          "rotated_ligand_moments": {"recall_best_in_topk": 0.6, "recall_within_1e-3_of_best": 0.7,
                                     "learned_vs_plain": 170.0, "ms_learned_sweep": 11.0,
                                     "coarse": {"recall_best": 0.95, "recall_within_1e-3": 1.0, "vs_plain": 88.0,
                                                "ms_learned_sweep": 21.0}},
          "config": {"eval_pairs": 20, "topk": 256}}
    t = bench.learned_target(ls)
    assert t["met"] and t["recall_best"] == 1.0 and t["vs_plain"] == 95.0 and "coarse stage" in t["form"]
    assert "configuration's ligand moments" in t["form"] and t["held_out_pairs"] == 20
    # no form meets the target: the best recall is reported, met is false
    ls["coarse"]["recall_best"] = 0.9
    ls["rotated_ligand_moments"]["coarse"]["recall_best"] = 0.85
    t = bench.learned_target(ls)
    assert not t["met"] and t["recall_best"] == 0.9
    # a form above the recall bar but below 10x plain does not count
    ls["coarse"].update(recall_best=1.0, vs_plain=8.0)
    t = bench.learned_target(ls)
    assert not t["met"]
