"""The scatter/gather pieces of the multi-GPU path on one GPU.

* `shard.detector_views` aliases the library's device detector (no copy);
* index ranges traced separately and summed reproduce one trace of the
  whole range (counts exact; sums to the FP32 per-CTA tally precision,
  since the histories land in other CTAs' shared-memory histograms);
* `shard.merge_detector` over a one-rank NCCL group (the collective the
  multi-GPU bench runs) leaves a single rank's detector unchanged.
No kernel waits on another rank: the ranges run one after the other.
"""
import os
import socket

import numpy as np
import pytest

import paper_2501_06054_gb300 as sas
import sas_workloads as W
from paper_2501_06054_gb300 import shard

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def test_views_alias_the_device_detector():
    cfg = W.core_shell_config()
    e = sas.Experiment(cfg["instrument"], cfg["model"], stream=torch.cuda.current_stream())
    e.trace(200_003, 1)
    v = shard.detector_views(e.h, e.npix)
    torch.cuda.synchronize()
    d = e.read()
    assert np.array_equal(v["sum_w"].cpu().numpy(), d["sum_w"].ravel())
    assert np.array_equal(v["count"].cpu().numpy().astype(np.uint64), d["count"].ravel())
    assert v["trans"].item() == d["trans"]
    e.close()


def test_ranges_sum_to_the_whole_run():
    cfg = W.core_shell_config()
    n, world = 1_000_003, 3
    st = torch.cuda.current_stream()
    acc = None
    for r in range(world):
        first, cnt = shard.rank_range(r, world, n)
        e = sas.Experiment(cfg["instrument"], cfg["model"], stream=st)
        e.trace_range(first, cnt, 1)
        v = {k: t.clone() for k, t in shard.detector_views(e.h, e.npix).items()}
        torch.cuda.synchronize()
        e.close()
        acc = v if acc is None else {k: acc[k] + v[k] for k in acc}
    ef = sas.Experiment(cfg["instrument"], cfg["model"], stream=st)
    ef.trace(n, 1)
    d = ef.read()
    ef.close()
    assert np.array_equal(acc["count"].cpu().numpy().astype(np.uint64), d["count"].ravel())
    so = d["sum_w"].ravel()
    big = so > 1e-6 * so.max()
    got = acc["sum_w"].cpu().numpy()
    assert np.all(np.abs(got - so)[big] <= 1e-6 * so[big])
    assert abs(acc["trans"].item() / d["trans"] - 1) < 1e-12


def test_one_rank_nccl_merge_is_identity():
    import torch.distributed as dist
    if dist.is_initialized():
        pytest.skip("a process group is already initialised")
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1,
                            device_id=torch.device("cuda", torch.cuda.current_device()))
    try:
        cfg = W.core_shell_config()
        e = sas.Experiment(cfg["instrument"], cfg["model"], stream=torch.cuda.current_stream())
        e.trace(100_000, 2)
        before = e.read()
        shard.merge_detector(shard.detector_views(e.h, e.npix))
        torch.cuda.synchronize()
        after = e.read()
        e.close()
        for k in ("sum_w", "sum_w2", "count"):
            assert np.array_equal(before[k], after[k])
        assert before["trans"] == after["trans"]
    finally:
        dist.destroy_process_group()
