"""Batched form and autotuners (GPU), checked against the FP64 oracle.

Experiment e of a batch uses Philox experiment id e, so its detector must
equal the oracle's trace of that experiment on the same streams: counts
bit-exact, every bin within 3 sigma and, stronger, within 1e-4 relative
where not tiny; total weight within 1e-4.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2501_06054_gb300 as sas
import sas_workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def _small_batch(n_exp=24, seed=3, grid=10, counts=(2e3, 4e4)):
    models, cnt = W.batched_models(n_exp=n_exp, seed=seed, n_poly=12, n_gamma=grid, n_psi=grid,
                                   count_range=counts)
    return models, cnt


def _check(d, ref, n):
    assert np.array_equal(d["count"], ref["count"].reshape(-1).astype(np.uint64))
    sw, so = d["sum_w"], ref["sum_w"].reshape(-1)
    tot = so.sum()
    assert abs(sw.sum() - tot) <= 1e-4 * abs(tot) + 1e-300
    var = np.maximum(ref["sum_w2"].reshape(-1) - so ** 2 / max(n, 1), 0.0)
    assert np.all(np.abs(sw - so) <= 3 * np.sqrt(var) + 1e-12 * max(so.max(), 1e-300))
    big = so > 1e-6 * so.max() if so.max() > 0 else np.zeros_like(so, bool)
    assert np.all(np.abs(sw - so)[big] <= 1e-4 * so[big])
    assert abs(d["trans"] - ref["trans"]) <= 1e-6 * max(1.0, ref["trans"])


@pytest.mark.parametrize("use_hist,block,target", [(1, 512, 2e9), (0, 256, 5e7), (1, 1024, 1e6)])
def test_batch_matches_oracle(use_hist, block, target):
    inst = W.instrument()
    models, cnt = _small_batch()
    b = sas.sas_create_batch(inst, models, cnt, stream=torch.cuda.current_stream())
    c = sas.sas_batch_get_config(b)
    c.use_hist, c.block, c.target_item_flop = use_hist, block, target
    sas.sas_batch_set_config(b, c)
    sas.sas_trace_batch(b, seed=5)
    npix = inst.nx * inst.ny
    for e, m in enumerate(models):
        d = sas.sas_read_batch_detector(b, e, npix)
        ref = oracle.trace(inst, m, int(cnt[e]), seed=5, exp_id=e)
        _check(d, ref, int(cnt[e]))
    info = sas.sas_batch_info(b)
    assert info["total_histories"] == int(np.sum(cnt))
    sas.sas_destroy_batch(b)


def test_batch_equals_single_experiment_traces():
    inst = W.instrument()
    models, cnt = _small_batch(n_exp=6, seed=11)
    b = sas.sas_create_batch(inst, models, cnt, stream=torch.cuda.current_stream())
    sas.sas_trace_batch(b, seed=9)
    sas.sas_trace_batch(b, seed=9)        # relaunching the graph gives the same result
    npix = inst.nx * inst.ny
    for e, m in enumerate(models):
        d = sas.sas_read_batch_detector(b, e, npix)
        ex = sas.Experiment(inst, m, stream=torch.cuda.current_stream())
        sas.sas_set_experiment_id(ex.h, e)
        ex.trace(int(cnt[e]), seed=9)
        s = ex.read()
        assert np.array_equal(d["count"], s["count"].reshape(-1))
        assert np.allclose(d["sum_w"], s["sum_w"].reshape(-1), rtol=2e-5,
                           atol=1e-7 * max(s["sum_w"].max(), 1e-300))
        ex.close()
    sas.sas_destroy_batch(b)


def test_batch_edge_cases():
    inst = W.instrument(nx=256, ny=256)       # histogram does not fit: global tallies
    m = W.Model(kind=W.SPHERE, radius=30.0, poly=0.2, n_poly=8)
    m2 = W.Model(kind=W.CORE_SHELL, radius=20.0, thickness=5.0, sld=1e-6, sld_shell=4e-6)
    models, cnt = [m, m2, m], [0, 1, 33]
    b = sas.sas_create_batch(inst, models, cnt, stream=torch.cuda.current_stream())
    sas.sas_trace_batch(b, seed=1)
    npix = inst.nx * inst.ny
    d0 = sas.sas_read_batch_detector(b, 0, npix)
    assert d0["count"].sum() == 0 and d0["sum_w"].sum() == 0.0
    for e in (1, 2):
        d = sas.sas_read_batch_detector(b, e, npix)
        ref = oracle.trace(inst, models[e], cnt[e], seed=1, exp_id=e)
        assert np.array_equal(d["count"], ref["count"].reshape(-1).astype(np.uint64))
        assert np.allclose(d["sum_w"], ref["sum_w"].reshape(-1), rtol=1e-5,
                           atol=1e-7 * ref["sum_w"].max())
    with pytest.raises(sas.SasError):
        sas.sas_read_batch_detector(b, 3, npix)
    sas.sas_destroy_batch(b)
    with pytest.raises(sas.SasError):      # FP64 models are rejected in batches
        sas.sas_create_batch(inst, [W.Model(precision=W.FP64)], [10])


def test_batch_autotune_keeps_results():
    inst = W.instrument()
    models, cnt = _small_batch(n_exp=16, seed=21)
    b = sas.sas_create_batch(inst, models, cnt, stream=torch.cuda.current_stream())
    best, ms = sas.sas_batch_autotune(b, seed=2)
    assert ms > 0 and best.block in (256, 512, 1024)
    sas.sas_trace_batch(b, seed=2)
    npix = inst.nx * inst.ny
    for e in range(0, 16, 5):
        d = sas.sas_read_batch_detector(b, e, npix)
        ref = oracle.trace(inst, models[e], int(cnt[e]), seed=2, exp_id=e)
        _check(d, ref, int(cnt[e]))
    sas.sas_destroy_batch(b)


def test_single_experiment_autotune_and_cache():
    cfg = W.core_shell_config()
    ex = sas.Experiment(cfg["instrument"], cfg["model"], stream=torch.cuda.current_stream())
    best, ms = sas.sas_autotune(ex.h, 200000, seed=1)
    assert ms > 0
    got = sas.sas_get_launch_config(ex.h)
    assert (got.block, got.tally, got.agg) == (best.block, best.tally, best.agg)
    ex.trace(100003, seed=4)
    d = ex.read()
    ref = oracle.trace(cfg["instrument"], cfg["model"], 100003, seed=4)
    assert np.array_equal(d["count"], ref["count"].astype(np.uint64))
    assert abs(d["sum_w"].sum() / ref["sum_w"].sum() - 1) < 1e-4
    # a new experiment with the same key starts from the tuned configuration
    ex2 = sas.Experiment(cfg["instrument"], cfg["model"])
    c2 = sas.sas_get_launch_config(ex2.h)
    assert (c2.block, c2.tally, c2.agg) == (best.block, best.tally, best.agg)
    ex.close()
    ex2.close()


@pytest.mark.parametrize("tally,agg,block,order_q", [(0, 0, 256, 0), (0, 1, 1024, 0), (1, 1, 512, 0), (1, 0, 256, 0),
                                                     (1, 0, 1024, 1), (1, 1, 512, 1), (0, 0, 256, 1)])
def test_launch_configs_agree(tally, agg, block, order_q):
    cfg = W.core_shell_config()
    ex = sas.Experiment(cfg["instrument"], cfg["model"], stream=torch.cuda.current_stream())
    c = sas.sas_launch_config(block=block, tally=tally, agg=agg, ctas_per_sm=0, stage_orient=0, order_q=order_q)
    sas.sas_set_launch_config(ex.h, c)
    ex.trace(300007, seed=8)
    d = ex.read()
    ref = oracle.trace(cfg["instrument"], cfg["model"], 300007, seed=8)
    assert np.array_equal(d["count"], ref["count"].astype(np.uint64))
    so = ref["sum_w"]
    big = so > 1e-6 * so.max()
    assert np.all(np.abs(d["sum_w"] - so)[big] <= 1e-4 * so[big])
    ex.close()


def test_batched_config_structure_in_one_launch():
    """The batched workload's structure at scale: the first 1024 of the 4096
    draws (all four kinds, sizes U[10, 200], polydispersity U[0, 0.3] with 40
    Schulz nodes, anisotropic spreads U[0, 30] deg on the 76 x 76 grid),
    counts of the draw / 10^4, per-experiment 128 x 128 detectors, in one
    graph launch. Every experiment equals its own single-experiment trace
    (Philox id e: counts bit-exact, sums to the FP32 tally precision), and
    two experiments of each kind (those with counts nearest 1000) equal the
    FP64 oracle."""
    inst = W.instrument()
    models, counts = W.batched_models(n_exp=4096, seed=1)
    n_exp = 1024
    models = models[:n_exp]
    cnt = np.maximum(counts[:n_exp] // 10000, 1).astype(np.uint64)
    st = torch.cuda.current_stream()
    b = sas.sas_create_batch(inst, models, cnt, stream=st)
    sas.sas_trace_batch(b, seed=3)
    npix = inst.nx * inst.ny
    assert sas.sas_batch_info(b)["total_histories"] == int(cnt.sum())
    for e, m in enumerate(models):
        d = sas.sas_read_batch_detector(b, e, npix)
        ex = sas.Experiment(inst, m, stream=st)
        sas.sas_set_experiment_id(ex.h, e)
        ex.trace(int(cnt[e]), seed=3)
        s = ex.read()
        ex.close()
        assert np.array_equal(d["count"], s["count"].reshape(-1)), e
        assert np.allclose(d["sum_w"], s["sum_w"].reshape(-1), rtol=2e-5,
                           atol=1e-7 * max(s["sum_w"].max(), 1e-300)), e
        assert abs(d["trans"] - s["trans"]) <= 1e-9 * max(1.0, s["trans"])
    kinds = np.array([m.kind for m in models])
    for k in range(4):
        idx = np.where(kinds == k)[0]
        near = np.argsort(np.abs(cnt[idx].astype(np.int64) - 1000), kind="stable")[:2]
        for e in idx[near]:
            d = sas.sas_read_batch_detector(b, int(e), npix)
            ref = oracle.trace(inst, models[e], int(cnt[e]), seed=3, exp_id=int(e))
            _check(d, ref, int(cnt[e]))
    sas.sas_destroy_batch(b)
