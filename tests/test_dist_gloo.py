"""The multi-rank host path on CPU: two gloo ranks each run their shard of one ensemble
(the oracle stands in for a GPU context, since shards are defined by the run indices
alone) and combine histograms and counters; the result must equal one process, also under
the state-following bound, where a run depends on the other runs of its group."""
import os
import socket

import numpy as np
import pytest

from paper_2412_16613_gb300 import sharding

INIT = (64, 64, 128)
N_RUNS = 1000
SNAPS = [0.002, 0.01, 0.05]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _oracle_shard(first, n, pad=0):
    import oracle
    r = oracle.run(oracle.frank(), INIT, n, first_run=first, seed=5, t_end=1.0, snap_times=SNAPS, threads=2,
                   pad_pow2=pad, ensemble_runs=N_RUNS if pad == 2 else None)
    hist = oracle.ee_histogram(r["snap_counts"]) if n else np.zeros((len(SNAPS), 65), dtype=np.uint64)
    counters = np.zeros(10, dtype=np.uint64)
    counters[1] = r["steps"].sum()
    counters[2] = r["reactions"].sum()
    counters[5] = (r["outcome"] >= 0).sum()
    counters[8] = r["steps"].max() if n else 0
    counters[9] = 1 if first == 0 else 2  # stands in for the layout each rank ran
    return hist, counters, r


def _worker(rank, world, port, out_dir, pad):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    first, n = sharding.shard(N_RUNS, rank, world)
    hist, counters, r = _oracle_shard(first, n, pad)
    hist, counters = sharding.combine(hist, counters, dist)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), hist=hist, counters=counters,
             final=r["final_counts"], first=first, n=n)
    dist.barrier()
    dist.destroy_process_group()


def test_shards_cover_the_runs_in_whole_groups():
    for total in (0, 1, 31, 32, 33, 1000, 4096):
        for world in (1, 2, 3, 8):
            spans = [sharding.shard(total, r, world) for r in range(world)]
            covered = []
            for first, n in spans:
                assert first % 32 == 0 and n >= 0
                covered += list(range(first, first + n))
            assert covered == list(range(total))
    assert sharding.weak_shard(1 << 20, 3) == (3 << 20, 1 << 20)


@pytest.mark.parametrize("pad", [0, 2])
def test_two_gloo_ranks_equal_one_process(tmp_path, pad):
    import oracle
    import torch.multiprocessing as mp
    oracle.build()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path), pad), nprocs=2, join=True, start_method="spawn")
    whole_hist, whole_counters, whole = _oracle_shard(0, N_RUNS, pad)
    parts = [np.load(os.path.join(tmp_path, f"rank{r}.npz")) for r in range(2)]
    whole_counters[9] = 3  # rank 0 ran layout bit 0, rank 1 layout bit 1
    for p in parts:
        assert np.array_equal(p["hist"], whole_hist)
        assert np.array_equal(p["counters"], whole_counters)
    final = np.concatenate([p["final"] for p in parts])
    assert np.array_equal(final, whole["final_counts"])
