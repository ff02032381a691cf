"""Multi-rank partition of the trace (CPU, gloo, world size 2).

The counter-based streams make a history depend only on (seed, experiment,
index), so ranks that trace disjoint index ranges and sum their detectors
with one reduction reproduce the single-process run (the paper's
scatter/gather of ncount over ranks, Sec. II.C). The ranks here run the
oracle; the partition and the reduction are what is tested.
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


def _rank_range(rank, world, n):
    """The split bench.py uses for weak scaling generalised to a fixed total:
    contiguous, disjoint, covering [0, n)."""
    base, extra = divmod(n, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def _worker(rank, world, port, n, out_path):
    import torch.distributed as dist
    import oracle
    import sas_workloads as W
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    cfg = W.core_shell_config()
    first, cnt = _rank_range(rank, world, n)
    r = oracle.trace(cfg["instrument"], cfg["model"], cnt, seed=3, first=first, threads=2)
    t = torch.tensor(np.concatenate([r["sum_w"].ravel(), r["sum_w2"].ravel(),
                                     r["count"].ravel().astype(np.float64), [r["trans"]]]))
    dist.all_reduce(t)
    if rank == 0:
        np.save(out_path, t.numpy())
    dist.destroy_process_group()


@pytest.mark.parametrize("n", [20001, 64])
def test_two_rank_partition_reproduces_single_run(tmp_path, n):
    import torch.multiprocessing as mp
    import oracle
    import sas_workloads as W
    oracle.build()
    for w in (2, 3):
        rngs = [_rank_range(r, w, n) for r in range(w)]
        assert rngs[0][0] == 0 and sum(c for _, c in rngs) == n
        assert all(rngs[i][0] + rngs[i][1] == rngs[i + 1][0] for i in range(w - 1))
    out = str(tmp_path / "red.npy")
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, n, out), nprocs=2, join=True, start_method="spawn")
    red = np.load(out)
    cfg = W.core_shell_config()
    full = oracle.trace(cfg["instrument"], cfg["model"], n, seed=3, threads=2)
    npix = full["sum_w"].size
    assert np.array_equal(red[2 * npix:3 * npix], full["count"].ravel().astype(np.float64))
    assert np.allclose(red[:npix], full["sum_w"].ravel(), rtol=1e-12, atol=0)
    assert np.allclose(red[npix:2 * npix], full["sum_w2"].ravel(), rtol=1e-12, atol=0)
    assert red[-1] == pytest.approx(full["trans"])
