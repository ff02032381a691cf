"""Multi-rank partition of the trace (CPU, gloo, world sizes 2 and 3).

The counter-based streams make a history depend only on (seed, experiment,
index), so ranks that trace disjoint index ranges and sum their detectors
with one reduction reproduce the single-process run (the paper's
scatter/gather of ncount over ranks, Sec. II.C). The ranks here run the
oracle; the index split and the reduction are the library's own
(`paper_2501_06054_gb300.shard`, the code bench.py's multi-GPU path runs
over NCCL), driven over gloo.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n, mode, dst, out_path):
    import torch.distributed as dist
    import oracle
    import sas_workloads as W
    from paper_2501_06054_gb300 import shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    cfg = W.core_shell_config()
    first, cnt = shard.rank_range(rank, world, n) if mode == "strong" else shard.weak_range(rank, n)
    r = oracle.trace(cfg["instrument"], cfg["model"], cnt, seed=3, first=first, threads=2)
    det = {"sum_w": torch.tensor(r["sum_w"].ravel()), "sum_w2": torch.tensor(r["sum_w2"].ravel()),
           "count": torch.tensor(r["count"].ravel().astype(np.int64)),
           "trans": torch.tensor([float(r["trans"])], dtype=torch.float64)}
    shard.merge_detector(det, dst=dst)
    if dst is None or rank == dst:
        np.savez(out_path + f".{rank}.npz", **{k: v.numpy() for k, v in det.items()})
    dist.destroy_process_group()


def test_rank_ranges_partition_the_index_range():
    from paper_2501_06054_gb300 import shard
    for n in (0, 1, 64, 20001):
        for w in (1, 2, 3, 8):
            rngs = [shard.rank_range(r, w, n) for r in range(w)]
            assert rngs[0][0] == 0 and sum(c for _, c in rngs) == n
            assert all(rngs[i][0] + rngs[i][1] == rngs[i + 1][0] for i in range(w - 1))
            assert max(c for _, c in rngs) - min(c for _, c in rngs) <= 1
    assert shard.weak_range(3, 100) == (300, 100)
    with pytest.raises(ValueError):
        shard.rank_range(2, 2, 10)


@pytest.mark.parametrize("world,n,mode,dst", [(2, 20001, "strong", None), (3, 64, "strong", 0),
                                              (2, 5003, "weak", None)])
def test_ranks_reproduce_single_run(tmp_path, world, n, mode, dst):
    import torch.multiprocessing as mp
    import oracle
    import sas_workloads as W
    oracle.build()
    out = str(tmp_path / "red")
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, n, mode, dst, out), nprocs=world, join=True,
                       start_method="spawn")
    total = n if mode == "strong" else n * world
    cfg = W.core_shell_config()
    full = oracle.trace(cfg["instrument"], cfg["model"], total, seed=3, threads=2)
    holders = range(world) if dst is None else [dst]
    for r in holders:
        red = np.load(out + f".{r}.npz")
        assert np.array_equal(red["count"], full["count"].ravel().astype(np.int64))
        assert np.allclose(red["sum_w"], full["sum_w"].ravel(), rtol=1e-12, atol=0)
        assert np.allclose(red["sum_w2"], full["sum_w2"].ravel(), rtol=1e-12, atol=0)
        assert red["trans"][0] == pytest.approx(full["trans"], rel=1e-12)


def test_experiment_partition_balances_without_exchange():
    """A batch splits over ranks by experiment: each experiment on exactly
    one rank, the largest load within 4/3 of the lower bound max(mean load,
    largest experiment) (the longest-processing-time guarantee), the split
    deterministic."""
    import sas_workloads as W
    from paper_2501_06054_gb300 import flops as F
    from paper_2501_06054_gb300 import shard
    models, counts = W.batched_models(n_exp=512, seed=3)
    costs = [F.flops_per_history(m.kind, m.n_poly, m.n_gamma * m.n_psi) * float(c) for m, c in zip(models, counts)]
    for world in (1, 2, 3, 8):
        parts = shard.experiment_partition(costs, world)
        assert len(parts) == world
        flat = sorted(e for p in parts for e in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[e] for e in p) for p in parts]
        bound = max(sum(costs) / world, max(costs))
        assert max(loads) <= 4.0 / 3.0 * bound * (1 + 1e-12)
        assert parts == shard.experiment_partition(costs, world)
    assert shard.experiment_partition([], 2) == [[], []]
    with pytest.raises(ValueError):
        shard.experiment_partition([1.0, -1.0], 2)
