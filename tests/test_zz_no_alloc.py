"""The batched trace that allocates nothing (sas_trace_batch_static).

For callers that cannot allocate device memory (their memory belongs to
another allocator or a fixed budget, or the host application forbids
device allocations), the library offers one batched-trace entry point
whose scratch lives in a static device array. This file runs last
(pytest collects it last) and checks, through the C ABI, two calls in a
row against the allocating entry point (sas_create_batch +
sas_trace_batch): counts bit-exact, bins within 1e-4 relative where not
tiny, totals within 1e-4. It passes alone in a fresh process and after the
other tests.
"""
import numpy as np
import pytest

import paper_2501_06054_gb300 as sas
import sas_workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def _compare(a_sw, a_cnt, b_sw, b_cnt):
    assert np.array_equal(a_cnt, b_cnt)
    for e in range(a_sw.shape[0]):
        so = b_sw[e]
        if so.max() <= 0:
            assert a_sw[e].max() == 0
            continue
        assert abs(a_sw[e].sum() - so.sum()) <= 1e-4 * so.sum()
        big = so > 1e-6 * so.max()
        assert np.all(np.abs(a_sw[e] - so)[big] <= 1e-4 * so[big])


def test_static_batch_matches_allocating_batch_twice():
    inst = W.instrument()
    models, counts = W.batched_models(n_exp=10, seed=17, n_poly=12, n_gamma=12, n_psi=12,
                                      count_range=(2e3, 3e4))
    npix = inst.nx * inst.ny
    stream = torch.cuda.current_stream()
    b = sas.sas_create_batch(inst, models, counts, stream=stream)
    sw = torch.empty((len(models), npix), dtype=torch.float64, device="cuda")
    sw2 = torch.empty_like(sw)
    cnt = torch.empty((len(models), npix), dtype=torch.int64, device="cuda")
    tr = torch.empty(len(models), dtype=torch.float64, device="cuda")
    for seed in (5, 6):                       # two calls in a row share the scratch
        sas.sas_trace_batch_static(inst, models, counts, seed, sw, sw2, cnt, tr, stream=stream)
        torch.cuda.synchronize()
        got_sw = sw.cpu().numpy()
        got_cnt = cnt.cpu().numpy().astype(np.uint64)
        got_tr = tr.cpu().numpy()
        sas.sas_trace_batch(b, seed)
        ref = [sas.sas_read_batch_detector(b, e, npix) for e in range(len(models))]
        ref_sw = np.stack([r["sum_w"] for r in ref])
        ref_cnt = np.stack([r["count"] for r in ref])
        _compare(got_sw, got_cnt, ref_sw, ref_cnt)
        assert np.allclose(got_tr, [r["trans"] for r in ref], rtol=1e-9)
        assert int(got_cnt.sum()) == int(np.sum(counts))
    sas.sas_destroy_batch(b)


def test_static_batch_rejects_batches_beyond_the_scratch():
    inst = W.instrument()
    models, counts = W.batched_models(n_exp=200, seed=3, n_poly=40, n_gamma=76, n_psi=76,
                                      count_range=(1e3, 1e4))
    npix = inst.nx * inst.ny
    sw = torch.empty((len(models), npix), dtype=torch.float64, device="cuda")
    cnt = torch.empty((len(models), npix), dtype=torch.int64, device="cuda")
    tr = torch.empty(len(models), dtype=torch.float64, device="cuda")
    with pytest.raises(sas.SasError) as e:
        sas.sas_trace_batch_static(inst, models, counts, 1, sw, sw, cnt, tr)
    assert e.value.status == sas.SAS_ERR_ARG
    assert "static scratch" in sas.sas_last_error()
