"""Multi-process sweep logic on CPU: two gloo ranks shard the rotations, sweep
their blocks with an injected sweeper (no GPU), gather the peaks and agree on
the best rotation exactly as a single process would (ties to the lowest index)."""
import os
import socket

import numpy as np
import pytest

from paper_1711_05075_gb300 import dist as D

torch = pytest.importorskip("torch")


def free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def fake_peaks(quats):
    # a deterministic stand-in for the GPU sweep: a smooth function of the rotation, with
    # exact ties planted so the lowest-index rule is exercised
    q = np.asarray(quats, np.float64)
    p = np.round(np.cos(3 * q[:, 0]) + q[:, 1] * q[:, 2], 2).astype(np.float32)
    return p, (np.abs(q[:, 3]) * 1000).astype(np.int64)


def worker(rank, world, port, k, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1711_05075_gb300 import synth
    q = synth.shoemake_quaternions(synth.SplitMix64(3), k)
    peak, arg, best = D.distributed_sweep(fake_peaks, q)
    t = D.max_over_ranks(float(rank + 1))
    np.savez(f"{out_path}.{rank}.npz", peak=peak, arg=arg, best=best, tmax=t)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,k", [(2, 1001), (3, 10), (2, 1)])
def test_distributed_sweep_matches_single_process(tmp_path, world, k):
    import torch.multiprocessing as mp
    from paper_1711_05075_gb300 import synth
    out = str(tmp_path / "res")
    mp.spawn(worker, args=(world, free_port(), k, out), nprocs=world, join=True)
    q = synth.shoemake_quaternions(synth.SplitMix64(3), k)
    ref_p, ref_a = fake_peaks(q)
    for r in range(world):
        d = np.load(f"{out}.{r}.npz")
        np.testing.assert_array_equal(d["peak"], ref_p)
        np.testing.assert_array_equal(d["arg"], ref_a)
        assert int(d["best"]) == int(np.argmax(ref_p))
        assert float(d["tmax"]) == float(world)


def test_shard_ranges_partition():
    for k in (0, 1, 7, 1000, 1001):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                s0, s1 = D.shard_range(k, r, world)
                assert 0 <= s0 <= s1 <= k
                seen.extend(range(s0, s1))
            assert seen == list(range(k))
            sizes = [D.shard_range(k, r, world)[1] - D.shard_range(k, r, world)[0] for r in range(world)]
            assert max(sizes) - min(sizes) <= 1
