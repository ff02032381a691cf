"""Capped cylinder and barbell (cylinders closed by spherical caps, Eq. 1
over disk slices) on the GPU against the FP64 oracle: model evaluations over
every form of 2 J1(x)/x (small to large |Q| R), records (quadrature and
per-event draws), detectors, a batch, the self-attenuation table, and the
refusals (the Gaussian-cap axis law stays a quadrature option). Tolerances
as for the other models: FP32 1e-5 relative + 1e-7 of P(0), FP64 1e-10 +
1e-13 P(0); pixels and counts bit-exact."""
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


def _m(kind, **kw):
    base = dict(kind=kind, radius=20.0, radius_polar=25.0, length=100.0, sld=2e-6, volume_fraction=0.01,
                poly=0.1, n_poly=10, axis_theta=1.2, axis_phi=0.3, n_cap=16)
    base.update(kw)
    return W.Model(**base)


MODELS = {
    "capped_cap": _m(W.CAPPED_CYLINDER, sigma_orient=0.25, n_gamma=8, n_psi=8),
    "capped_fixed_fp64": _m(W.CAPPED_CYLINDER, precision=W.FP64),
    "barbell_iso": _m(W.BARBELL, radius=10.0, radius_polar=20.0, length=80.0, isotropic=W.ISOTROPIC,
                      n_gamma=10, n_psi=10),
    "barbell_angles_fp64": _m(W.BARBELL, precision=W.FP64, radius=10.0, radius_polar=20.0, length=80.0,
                              isotropic=W.UNIFORM_ANGLES, n_gamma=6, n_psi=6, n_cap=12),
    "spherocylinder": _m(W.CAPPED_CYLINDER, radius=15.0, radius_polar=15.0, length=60.0, poly=0.0, n_poly=1),
    "sphere_limit": _m(W.BARBELL, radius=30.0, radius_polar=30.0, length=0.0, n_cap=24),
    "barbell_one_slice": _m(W.BARBELL, n_cap=1, radius_polar=40.0, poly=0.3, n_poly=32, sigma_orient=0.4,
                            n_gamma=6, n_psi=6),
    # the per-event estimator (Sec. II.B): one Gaussian radius and one axis per history
    "capped_event": _m(W.CAPPED_CYLINDER, poly=0.2, poly_dist=W.GAUSSIAN, n_poly=16, isotropic=W.ISOTROPIC,
                       sampling=W.PER_EVENT),
    "barbell_event_fp64": _m(W.BARBELL, precision=W.FP64, radius=10.0, radius_polar=20.0, length=80.0,
                             poly=0.15, poly_dist=W.GAUSSIAN, n_poly=16, isotropic=W.UNIFORM_ANGLES,
                             sampling=W.PER_EVENT),
}


def _eval(e, m, q):
    fp64 = m.precision == W.FP64
    dt = torch.float64 if fp64 else torch.float32
    out = torch.empty(len(q), dtype=dt, device="cuda")
    sas.sas_eval_model(e.h, torch.tensor(q, dtype=dt, device="cuda"), len(q), out)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def _tol(m):
    return (1e-10, 1e-13) if m.precision == W.FP64 else (1e-5, 1e-7)


@pytest.mark.parametrize("name", [k for k in MODELS if "event" not in k])
def test_model_parity(name):
    """Scattering vectors from |Q| ~ 0 to |Q| R ~ 50: every 2 J1(x)/x tier."""
    m = MODELS[name]
    rng = np.random.default_rng(5)
    d = rng.normal(size=(2400, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    qm = np.concatenate([rng.uniform(0.0, 0.05, 1200), rng.uniform(0.05, 0.15, 800), rng.uniform(0.15, 1.5, 400)])
    q = np.concatenate([d * qm[:, None], np.zeros((1, 3))])
    e = sas.Experiment(W.instrument(), m, stream=torch.cuda.current_stream())
    got = _eval(e, m, q)
    ref = oracle.dsigma(oracle.Prepared(m), q)
    rel, ab = _tol(m)
    err = np.abs(got - ref)
    assert np.all(err <= rel * np.abs(ref) + ab * ref[-1]), (name, np.max(err / (np.abs(ref) + ref[-1])))
    e.close()


def _records(e, first, n, seed):
    pix = torch.empty(n, dtype=torch.int32, device="cuda")
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    sas.sas_trace_records(e.h, first, n, seed, pix, w)
    torch.cuda.synchronize()
    return pix.cpu().numpy().astype(np.int64), w.cpu().numpy()


@pytest.mark.parametrize("name", ["capped_cap", "capped_fixed_fp64", "barbell_iso", "barbell_angles_fp64",
                                  "capped_event", "barbell_event_fp64"])
def test_records_parity(name):
    m = MODELS[name]
    inst = W.instrument(nx=64, ny=64)
    e = sas.Experiment(inst, m, stream=torch.cuda.current_stream())
    n = 3001
    for first in (0, (1 << 35) + 7):
        pix, w = _records(e, first, n, seed=6)
        po, wo = oracle.records(inst, m, n, seed=6, first=first)
        assert np.array_equal(pix, po)
        rel, ab = _tol(m)
        assert np.all(np.abs(w - wo) <= rel * np.abs(wo) + ab * np.max(wo)), (name, first)
    e.close()


def _check_detector(d, ref):
    assert np.array_equal(d["count"].ravel(), ref["count"].ravel().astype(np.uint64))
    so = ref["sum_w"].ravel()
    sw = d["sum_w"].ravel()
    assert abs(sw.sum() - so.sum()) <= 1e-4 * abs(so.sum())
    big = so > 1e-6 * so.max()
    assert np.all(np.abs(sw - so)[big] <= 1e-4 * so[big])


@pytest.mark.parametrize("name", ["capped_cap", "barbell_iso", "capped_event"])
def test_trace_and_batch(name):
    m = MODELS[name]
    inst = W.instrument(nx=48, ny=48)
    n = 60001
    e = sas.Experiment(inst, m, stream=torch.cuda.current_stream())
    e.trace(n, seed=3)
    ref = oracle.trace(inst, m, n, seed=3)
    _check_detector(e.read(), ref)
    e.close()
    b = sas.sas_create_batch(inst, [m, W.Model(kind=W.SPHERE, radius=20.0)], np.array([n, 5000], np.uint64),
                             stream=torch.cuda.current_stream())
    sas.sas_trace_batch(b, seed=3)
    _check_detector(sas.sas_read_batch_detector(b, 0, inst.nx * inst.ny), ref)
    sas.sas_destroy_batch(b)


def test_self_attenuation_table():
    inst = W.instrument(nx=48, ny=48)
    m = W.Model(**{**MODELS["barbell_iso"].as_dict(), "self_attenuation": 1})
    e = sas.Experiment(inst, m, stream=torch.cuda.current_stream())
    t = sas.sas_attenuation_table(e.h)
    lam, mu, c = oracle.att_table(inst, m)
    assert np.allclose(t["lam"], lam, rtol=1e-15, atol=0)
    assert np.all(np.abs(t["mu_s"] - mu) <= 1e-5 * np.abs(mu))
    n = 3001
    pix, w = _records(e, 0, n, seed=4)
    po, wo = oracle.records(inst, m, n, seed=4)
    assert np.array_equal(pix, po)
    assert np.all(np.abs(w - wo) <= 1e-5 * np.abs(wo) + 1e-7 * np.max(wo))
    e.close()


@pytest.mark.parametrize("bad", [dict(n_cap=0), dict(n_cap=65), dict(radius_polar=19.0), dict(length=-1.0),
                                 dict(sampling=W.PER_EVENT, poly_dist=W.GAUSSIAN)])
def test_refusals(bad):
    m = W.Model(**{**MODELS["capped_cap"].as_dict(), **bad})
    with pytest.raises(sas.SasError):
        sas.Experiment(W.instrument(), m, stream=torch.cuda.current_stream())
