"""The fuzzy sphere (a Schulz-polydisperse sphere whose density is blurred
by an isotropic Gaussian of width sigma) on the GPU against the FP64 oracle:
evaluations in FP32 and FP64 at T1 (1e-5 relative + 1e-7 of the forward
value; FP64 1e-10 and 1e-13), per-history records and a traced detector,
the |Q|-ordered pass against the plain loop (same histories, weights within
the ordered pass's FP32 bound), the per-event estimator's records, a batch,
and the refusal of a fuzziness on any other body."""
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
    oracle.build()
    yield


def _fuzzy(precision=W.FP32, **kw):
    d = dict(kind=W.SPHERE, precision=precision, radius=45.0, sld=2.0e-6, sld_solvent=0.0,
             volume_fraction=0.01, poly=0.12, n_poly=30, fuzziness=7.0)
    d.update(kw)
    return W.Model(**d)


@pytest.mark.parametrize("precision", [W.FP32, W.FP64])
def test_fuzzy_sphere_evaluations(precision):
    m = _fuzzy(precision)
    rng = np.random.default_rng(5)
    d = rng.normal(size=(2000, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    q = d * np.concatenate([[0.0], rng.uniform(1e-4, 0.3, 1999)])[:, None]
    e = sas.Experiment(W.instrument(), m, stream=torch.cuda.current_stream())
    dt = torch.float64 if precision == W.FP64 else torch.float32
    out = torch.empty(len(q), dtype=dt, device="cuda")
    sas.sas_eval_model(e.h, torch.tensor(q, dtype=dt, device="cuda"), len(q), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    qd = torch.tensor(q, dtype=dt).double().numpy()
    ref = oracle.dsigma(oracle.Prepared(m), qd)
    rel, ab = (1e-10, 1e-13) if precision == W.FP64 else (1e-5, 1e-7)
    assert np.all(np.abs(got - ref) <= rel * np.abs(ref) + ab * ref[0]), np.max(np.abs(got - ref) / ref[0])
    # the blur is there: well below the sharp sphere at large Q
    sharp = oracle.dsigma(oracle.Prepared(_fuzzy(precision, fuzziness=0.0)), qd)
    far = np.linalg.norm(qd, axis=1) > 0.2
    assert np.all(got[far] < 0.5 * sharp[far] + 1e-30)
    e.close()


def test_fuzzy_sphere_records_and_trace():
    m = _fuzzy()
    inst = W.instrument(nx=64, ny=64)
    e = sas.Experiment(inst, m, stream=torch.cuda.current_stream())
    n = 5003
    pix = torch.empty(n, dtype=torch.int32, device="cuda")
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    sas.sas_trace_records(e.h, 11, n, 3, pix, w)
    torch.cuda.synchronize()
    po, wo = oracle.records(inst, m, n, seed=3, first=11)
    assert np.array_equal(pix.cpu().numpy().astype(np.int64), po)
    assert np.all(np.abs(w.cpu().numpy() - wo) <= 1e-5 * np.abs(wo) + 1e-7 * np.max(wo))
    nt = 200003
    e.trace(nt, seed=5)
    d = e.read()
    ref = oracle.trace(inst, m, nt, seed=5)
    assert np.array_equal(d["count"].ravel(), ref["count"].ravel().astype(np.uint64))
    so = ref["sum_w"].ravel()
    big = so > 1e-6 * so.max()
    assert np.all(np.abs(d["sum_w"].ravel() - so)[big] <= 1e-4 * so[big])
    e.close()


def test_fuzzy_sphere_ordered_pass_matches_plain_loop():
    m = _fuzzy()
    inst = W.instrument()
    out = []
    for order_q in (0, 1):
        ex = sas.Experiment(inst, m, stream=torch.cuda.current_stream())
        c = sas.sas_launch_config(block=1024, tally=1, agg=0, ctas_per_sm=0, stage_orient=0, order_q=order_q)
        sas.sas_set_launch_config(ex.h, c)
        ex.trace(3000017, 7)
        out.append(ex.read())
        ex.close()
    a, b = out
    assert np.array_equal(a["count"], b["count"])
    sa, sb = a["sum_w"].ravel(), b["sum_w"].ravel()
    big = sa > 1e-6 * sa.max()
    assert np.all(np.abs(sa - sb)[big] <= 6e-6 * sa[big])


def test_fuzzy_sphere_per_event_and_batch():
    ev = _fuzzy(poly=0.2, poly_dist=W.GAUSSIAN, n_poly=32, sampling=W.PER_EVENT)
    inst = W.instrument(nx=48, ny=48)
    e = sas.Experiment(inst, ev, stream=torch.cuda.current_stream())
    n = 4001
    pix = torch.empty(n, dtype=torch.int32, device="cuda")
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    sas.sas_trace_records(e.h, 0, n, 9, pix, w)
    torch.cuda.synchronize()
    po, wo = oracle.records(inst, ev, n, seed=9)
    assert np.array_equal(pix.cpu().numpy().astype(np.int64), po)
    assert np.all(np.abs(w.cpu().numpy() - wo) <= 1e-5 * np.abs(wo) + 1e-7 * np.max(np.abs(wo)))
    e.close()
    models = [_fuzzy(), _fuzzy(fuzziness=0.0), _fuzzy(radius=80.0, fuzziness=15.0)]
    counts = np.array([20000, 15000, 10007], np.uint64)
    b = sas.sas_create_batch(inst, models, counts, stream=torch.cuda.current_stream())
    sas.sas_trace_batch(b, seed=2)
    for k, m in enumerate(models):
        d = sas.sas_read_batch_detector(b, k, inst.nx * inst.ny)
        ref = oracle.trace(inst, m, int(counts[k]), seed=2, exp_id=k)
        assert np.array_equal(d["count"], ref["count"].reshape(-1).astype(np.uint64))
        so = ref["sum_w"].reshape(-1)
        big = so > 1e-6 * so.max()
        assert np.all(np.abs(d["sum_w"] - so)[big] <= 1e-4 * so[big])
    sas.sas_destroy_batch(b)


def test_fuzziness_only_on_the_sphere():
    cyl = W.Model(kind=W.CYLINDER, radius=20.0, length=100.0, n_gamma=8, n_psi=8, sigma_orient=0.2,
                  fuzziness=3.0)
    with pytest.raises(sas.SasError):
        sas.Experiment(W.instrument(), cyl, stream=torch.cuda.current_stream())
    with pytest.raises(sas.SasError):
        sas.Experiment(W.instrument(), _fuzzy(fuzziness=-1.0), stream=torch.cuda.current_stream())
