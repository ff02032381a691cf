"""Cylinder radial table on the GPU (radial_table = 1) against the FP64
oracle, which sums the radius nodes directly: the table changes nothing
beyond the parity tolerances of the plain path.

* model evaluations at the Q of real histories of the instrument (oracle
  geometry): FP32 1e-5 relative + 1e-7 P(0), FP64 1e-10 + 1e-13 P(0);
* per-history records, FP32 and FP64;
* a batched experiment with the table against the oracle's trace.
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


def _cyl(**kw):
    base = dict(W.cylinder_config()["model"].as_dict(), n_gamma=20, n_psi=20, radial_table=1)
    base.update(kw)
    return W.Model(**base)


CASES = {
    "workload_schulz": (W.cylinder_config()["instrument"], _cyl()),
    "gauss_isotropic": (W.instrument(nx=64, ny=64, pixel_x=0.012, pixel_y=0.012),
                        _cyl(poly=0.3, poly_dist=W.GAUSSIAN, isotropic=W.ISOTROPIC, n_poly=48)),
    "monodisperse_fixed_axis": (W.instrument(), _cyl(poly=0.0, n_poly=1, sigma_orient=0.0, radius=35.0,
                                                     length=150.0)),
    "fp64_schulz": (W.instrument(nx=40, ny=40), _cyl(precision=W.FP64, n_gamma=12, n_psi=12)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_radial_table_model_parity(name):
    inst, m = CASES[name]
    g = oracle.geometry_records(inst, 3000, seed=2)
    q = g["q"][g["pixel"] >= 0][:2000]
    q = np.concatenate([q, np.zeros((1, 3))])            # and Q = 0
    e = sas.Experiment(inst, m, stream=torch.cuda.current_stream())
    fp64 = m.precision == W.FP64
    dt = torch.float64 if fp64 else torch.float32
    qd = torch.tensor(q, dtype=dt, device="cuda").contiguous()
    out = torch.empty(len(q), dtype=dt, device="cuda")
    sas.sas_eval_model(e.h, qd, len(q), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    prep = oracle.Prepared(m)
    ref = oracle.dsigma(prep, q)
    p0 = ref[-1]
    rel, ab = (1e-10, 1e-13) if fp64 else (1e-5, 1e-7)
    err = np.abs(got - ref)
    assert np.all(err <= rel * np.abs(ref) + ab * p0), (name, np.max(err / (np.abs(ref) + ab * p0 / rel)))
    e.close()


def _records(e, first, n, seed):
    pix = torch.empty(n, dtype=torch.int32, device="cuda")
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    sas.sas_trace_records(e.h, first, n, seed, pix, w)
    torch.cuda.synchronize()
    return pix.cpu().numpy().astype(np.int64), w.cpu().numpy()


@pytest.mark.parametrize("name", ["workload_schulz", "fp64_schulz"])
def test_radial_table_records_parity(name):
    inst, m = CASES[name]
    e = sas.Experiment(inst, m, stream=torch.cuda.current_stream())
    n = 3001
    pix, w = _records(e, 77, n, seed=3)
    po, wo = oracle.records(inst, m, n, seed=3, first=77)
    assert np.array_equal(pix, po)
    rel, ab = (1e-10, 1e-13) if m.precision == W.FP64 else (1e-5, 1e-7)
    assert np.all(np.abs(w - wo) <= rel * np.abs(wo) + ab * np.max(wo))
    e.close()


def test_radial_table_in_a_batch():
    inst = W.instrument(nx=64, ny=64)
    models = [_cyl(n_poly=20), W.Model(kind=W.SPHERE, radius=30.0, poly=0.1, n_poly=10),
              _cyl(radius=15.0, poly=0.2, poly_dist=W.GAUSSIAN, n_poly=24, isotropic=W.UNIFORM_ANGLES)]
    counts = np.array([20000, 30000, 15001], dtype=np.uint64)
    b = sas.sas_create_batch(inst, models, counts, stream=torch.cuda.current_stream())
    sas.sas_trace_batch(b, seed=6)
    npix = inst.nx * inst.ny
    for k, m in enumerate(models):
        d = sas.sas_read_batch_detector(b, k, npix)
        ref = oracle.trace(inst, m, int(counts[k]), seed=6, exp_id=k)
        assert np.array_equal(d["count"], ref["count"].reshape(-1).astype(np.uint64))
        so = ref["sum_w"].reshape(-1)
        big = so > 1e-6 * so.max()
        assert np.all(np.abs(d["sum_w"] - so)[big] <= 1e-4 * so[big])
        assert abs(d["sum_w"].sum() - so.sum()) <= 1e-4 * so.sum()
    sas.sas_destroy_batch(b)
