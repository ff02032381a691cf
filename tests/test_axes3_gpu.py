"""Particles without a symmetry axis (triaxial ellipsoid, parallelepiped,
elliptical cylinder, hollow rectangular prism; Sec. II.B) on the GPU
against the FP64 oracle: model evaluations, records (quadrature and
per-event draws of the three angles), detectors and a batch, at the plain
path's tolerances (T1); the hollow prism's evaluations, whose outer and
inner terms cancel, at T2 (FP32 records of it are left to FP64)."""
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


def _m(kind, **kw):
    base = dict(kind=kind, radius=12.0, radius_b=20.0, radius_polar=40.0, sld=2e-6, volume_fraction=0.01,
                poly=0.1, n_poly=16, axis_theta=1.2, axis_phi=0.3, axis_psi=0.7)
    base.update(kw)
    return W.Model(**base)


MODELS = {
    "tri_cap": _m(W.TRIAXIAL_ELLIPSOID, sigma_orient=0.25, n_gamma=10, n_psi=10),
    "tri_iso_fp64": _m(W.TRIAXIAL_ELLIPSOID, precision=W.FP64, isotropic=W.ISOTROPIC, n_gamma=8, n_psi=8,
                       n_rot=8),
    "box_angles": _m(W.PARALLELEPIPED, isotropic=W.UNIFORM_ANGLES, n_gamma=10, n_psi=10, n_rot=10),
    "box_fixed": _m(W.PARALLELEPIPED, poly=0.0, n_poly=1),
    "box_fixed_fp64": _m(W.PARALLELEPIPED, precision=W.FP64, poly=0.2, poly_dist=W.GAUSSIAN, n_poly=24),
    "tri_event": _m(W.TRIAXIAL_ELLIPSOID, poly=0.2, poly_dist=W.GAUSSIAN, isotropic=W.UNIFORM_ANGLES,
                    sampling=W.PER_EVENT),
    "box_event_iso_fp64": _m(W.PARALLELEPIPED, precision=W.FP64, poly_dist=W.GAUSSIAN, isotropic=W.ISOTROPIC,
                             sampling=W.PER_EVENT),
    # elliptical cylinder (semi-axes 12, 20, length 150) and hollow rectangular prism (walls 3)
    "ellcyl_cap": _m(W.ELLIPTICAL_CYLINDER, length=150.0, sigma_orient=0.25, n_gamma=10, n_psi=10),
    "ellcyl_iso_fp64": _m(W.ELLIPTICAL_CYLINDER, precision=W.FP64, length=150.0, isotropic=W.ISOTROPIC,
                          n_gamma=8, n_psi=8, n_rot=8),
    "hprism_angles": _m(W.HOLLOW_RECTANGULAR_PRISM, thickness=3.0, isotropic=W.UNIFORM_ANGLES, n_gamma=8,
                        n_psi=8, n_rot=8),
    "hprism_fixed_fp64": _m(W.HOLLOW_RECTANGULAR_PRISM, precision=W.FP64, thickness=3.0),
    "ellcyl_event": _m(W.ELLIPTICAL_CYLINDER, length=150.0, poly=0.2, poly_dist=W.GAUSSIAN,
                       isotropic=W.UNIFORM_ANGLES, sampling=W.PER_EVENT),
    "hprism_event_fp64": _m(W.HOLLOW_RECTANGULAR_PRISM, precision=W.FP64, thickness=3.0, poly_dist=W.GAUSSIAN,
                            isotropic=W.ISOTROPIC, sampling=W.PER_EVENT),
}


def _cancel(m):
    """P_S / P(0): the hollow prism's outer and inner terms have opposite
    signs, |F| is bounded by their sum (the same ratio for every size node,
    since one factor scales all edges)."""
    if m.kind != W.HOLLOW_RECTANGULAR_PRISM:
        return 1.0
    a, b, c, t = m.radius, m.radius_b, m.radius_polar, m.thickness
    vo, vi = a * b * c, (a - t) * (b - t) * (c - t)
    return ((vo + vi) / (vo - vi)) ** 2


@pytest.mark.parametrize("name", [k for k in MODELS if "event" not in k])
def test_axes3_model_parity(name):
    m = MODELS[name]
    inst = W.instrument()
    q = np.random.default_rng(3).normal(size=(1500, 3)) * 0.04
    q = np.concatenate([q, np.zeros((1, 3))])
    e = sas.Experiment(inst, m, stream=torch.cuda.current_stream())
    fp64 = m.precision == W.FP64
    dt = torch.float64 if fp64 else torch.float32
    out = torch.empty(len(q), dtype=dt, device="cuda")
    sas.sas_eval_model(e.h, torch.tensor(q, dtype=dt, device="cuda"), len(q), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    ref = oracle.dsigma(oracle.Prepared(m), q)
    # T1, or for the hollow prism's cancelling terms T2 with P_S = ratio x P(0)
    ps = _cancel(m) * ref[-1]
    if fp64:
        tol = 1e-10 * np.abs(ref) + 1e-13 * ps
    elif ps > ref[-1]:
        tol = 1e-5 * np.abs(ref) + 6e-6 * np.sqrt(np.abs(ref) * ps) + 1e-7 * ps
    else:
        tol = 1e-5 * np.abs(ref) + 1e-7 * ref[-1]
    assert np.all(np.abs(got - ref) <= tol), (name, np.max(np.abs(got - ref) / tol))
    e.close()


def _records(e, first, n, seed):
    pix = torch.empty(n, dtype=torch.int32, device="cuda")
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    sas.sas_trace_records(e.h, first, n, seed, pix, w)
    torch.cuda.synchronize()
    return pix.cpu().numpy().astype(np.int64), w.cpu().numpy()


@pytest.mark.parametrize("name", [k for k in MODELS if k != "hprism_angles"])
def test_axes3_records_parity(name):
    m = MODELS[name]
    inst = W.instrument(nx=64, ny=64)
    e = sas.Experiment(inst, m, stream=torch.cuda.current_stream())
    n = 4001
    for first in (0, (1 << 37) + 11):
        pix, w = _records(e, first, n, seed=8)
        po, wo = oracle.records(inst, m, n, seed=8, first=first)
        assert np.array_equal(pix, po)
        rel, ab = (1e-10, 1e-13) if m.precision == W.FP64 else (1e-5, 1e-7)
        assert np.all(np.abs(w - wo) <= rel * np.abs(wo) + ab * np.max(wo)), (name, first)
    e.close()


@pytest.mark.parametrize("name", ["tri_cap", "box_angles", "tri_event", "ellcyl_cap", "ellcyl_event"])
def test_axes3_trace_and_batch(name):
    m = MODELS[name]
    inst = W.instrument(nx=48, ny=48)
    n = 100003
    e = sas.Experiment(inst, m, stream=torch.cuda.current_stream())
    e.trace(n, seed=2)
    d = e.read()
    ref = oracle.trace(inst, m, n, seed=2)
    assert np.array_equal(d["count"].ravel(), ref["count"].ravel().astype(np.uint64))
    so = ref["sum_w"].ravel()
    big = so > 1e-6 * so.max()
    assert np.all(np.abs(d["sum_w"].ravel() - so)[big] <= 1e-4 * so[big])
    e.close()
    b = sas.sas_create_batch(inst, [m, W.Model(kind=W.SPHERE, radius=20.0)], np.array([n, 5000], np.uint64),
                             stream=torch.cuda.current_stream())
    sas.sas_trace_batch(b, seed=2)
    db = sas.sas_read_batch_detector(b, 0, inst.nx * inst.ny)
    assert np.array_equal(db["count"], ref["count"].reshape(-1).astype(np.uint64))
    assert np.all(np.abs(db["sum_w"] - so)[big] <= 1e-4 * so[big])
    sas.sas_destroy_batch(b)
