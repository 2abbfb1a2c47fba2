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
