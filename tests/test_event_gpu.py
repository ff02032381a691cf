"""Per-event sampling mode (Sec. II.B) on the GPU against the FP64 oracle.

Each history draws one radius (Gaussian restricted to R > 0, by inversion)
and one axis (uniform on the sphere or in the angles) from its Philox block
2. The oracle makes the same draws in FP64, so:

* per-history weights agree to the FP32 tolerance of the records test
  (1e-5 relative + 1e-7 of the largest weight), FP64 to 1e-10;
* detectors: counts bit-exact, bins within 3 sigma and 1e-4 where not
  tiny, totals within 1e-4;
* batched experiments in per-event mode equal the oracle's single traces;
* at full size (2e6 histories) the GPU per-event estimator agrees with the
  GPU quadrature over the same laws, bin by bin (z-scores of per-history
  differences on the same histories);
* invalid combinations are refused, and the model-evaluation hook refuses
  per-event models.
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


def _ev(kind, precision=W.FP32, iso=W.UNIFORM_ANGLES, **kw):
    base = dict(kind=kind, precision=precision, radius=30.0, sld=2e-6, sld_solvent=0.0,
                volume_fraction=0.01, poly=0.2, poly_dist=W.GAUSSIAN, n_poly=32, isotropic=iso,
                n_gamma=24, n_psi=24, sampling=W.PER_EVENT)
    if kind == W.CORE_SHELL:
        base.update(radius=40.0, thickness=10.0, sld=1e-6, sld_shell=3e-6, sld_solvent=6e-6,
                    sq_kind=W.SQ_HARD_SPHERE_PY, sq_radius=50.0, sq_fraction=0.2, poly=0.15)
    if kind == W.CYLINDER:
        base.update(radius=20.0, length=400.0)
    if kind == W.ELLIPSOID:
        base.update(radius=25.0, radius_polar=70.0)
    base.update(kw)
    return W.Model(**base)


CASES = {
    "sphere": (W.instrument(), _ev(W.SPHERE)),
    "sphere_fp64": (W.instrument(), _ev(W.SPHERE, precision=W.FP64)),
    "core_shell_py": (W.instrument(), _ev(W.CORE_SHELL)),
    "cylinder_angles": (W.instrument(nx=64, ny=64, pixel_x=0.01, pixel_y=0.01), _ev(W.CYLINDER)),
    "cylinder_sphere": (W.instrument(nx=64, ny=64, pixel_x=0.01, pixel_y=0.01),
                        _ev(W.CYLINDER, iso=W.ISOTROPIC, poly=0.3)),
    "cylinder_fixed_axis_fp64": (W.instrument(nx=48, ny=40), _ev(W.CYLINDER, precision=W.FP64, iso=W.CAP,
                                                                 sigma_orient=0.0, axis_theta=1.2,
                                                                 axis_phi=0.4)),
    "ellipsoid_angles": (W.Instrument(nx=50, ny=30, mu=40.0), _ev(W.ELLIPSOID)),
    "monodisperse": (W.instrument(), _ev(W.SPHERE, poly=0.0)),
}


def _records(e, first, n, seed):
    pix = torch.empty(n, dtype=torch.int32, device="cuda")
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    sas.sas_trace_records(e.h, first, n, seed, pix, w)
    torch.cuda.synchronize()
    return pix.cpu().numpy().astype(np.int64), w.cpu().numpy()


@pytest.mark.parametrize("name", list(CASES))
def test_event_records_parity(name):
    inst, m = CASES[name]
    e = sas.Experiment(inst, m, stream=torch.cuda.current_stream())
    n = 6007
    for first in (0, 987654321, (1 << 41) + 3):
        pix, w = _records(e, first, n, seed=11)
        po, wo = oracle.records(inst, m, n, seed=11, first=first)
        assert np.array_equal(pix, po)
        scale = np.max(np.abs(wo))
        rel, absf = (1e-10, 1e-13) if m.precision == W.FP64 else (1e-5, 1e-7)
        err = np.abs(w - wo)
        assert np.all(err <= rel * np.abs(wo) + absf * scale), (name, first, err.max() / scale)
    e.close()


def _check_detector(d, ref, n):
    assert np.array_equal(d["count"].ravel(), ref["count"].ravel().astype(np.uint64))
    sw, so = d["sum_w"].ravel(), ref["sum_w"].ravel()
    tot = so.sum()
    assert abs(sw.sum() - tot) <= 1e-4 * abs(tot)
    var = np.maximum(ref["sum_w2"].ravel() - so ** 2 / n, 0.0)
    assert np.all(np.abs(sw - so) <= 3 * np.sqrt(var) + 1e-12 * so.max())
    big = so > 1e-6 * so.max()
    assert np.all(np.abs(sw - so)[big] <= 1e-4 * so[big])
    assert abs(d["trans"] - ref["trans"]) <= 1e-6 * max(1.0, ref["trans"])


@pytest.mark.parametrize("name", ["sphere", "core_shell_py", "cylinder_angles", "ellipsoid_angles"])
def test_event_trace_parity(name):
    inst, m = CASES[name]
    n = 300001
    e = sas.Experiment(inst, m, stream=torch.cuda.current_stream())
    e.trace(n, seed=4)
    d = e.read()
    ref = oracle.trace(inst, m, n, seed=4)
    _check_detector(d, ref, n)
    e.close()


def test_event_batch_matches_oracle():
    inst = W.instrument(nx=64, ny=64)
    models = [_ev(W.SPHERE), _ev(W.CYLINDER, n_poly=8), _ev(W.CORE_SHELL),
              W.Model(kind=W.SPHERE, radius=35.0, poly=0.1, n_poly=12),          # quadrature, Schulz
              _ev(W.ELLIPSOID, iso=W.ISOTROPIC)]
    counts = np.array([40000, 25000, 30001, 20000, 15000], dtype=np.uint64)
    b = sas.sas_create_batch(inst, models, counts, stream=torch.cuda.current_stream())
    sas.sas_trace_batch(b, seed=9)
    npix = inst.nx * inst.ny
    for k, m in enumerate(models):
        d = sas.sas_read_batch_detector(b, k, npix)
        ref = oracle.trace(inst, m, int(counts[k]), seed=9, exp_id=k)
        _check_detector(d, ref, int(counts[k]))
    sas.sas_destroy_batch(b)


def test_event_estimator_agrees_with_quadrature_at_full_size():
    """Same 2e6 histories, two estimators (GPU): per-pixel sums of the
    per-history differences are consistent with zero."""
    inst = W.instrument(nx=32, ny=32, pixel_x=0.02, pixel_y=0.02)
    ev = _ev(W.CYLINDER, n_poly=40, n_gamma=48, n_psi=48)
    qd = W.Model(**{**ev.as_dict(), "sampling": W.QUADRATURE})
    n = 2_000_000
    e1 = sas.Experiment(inst, ev, stream=torch.cuda.current_stream())
    e2 = sas.Experiment(inst, qd, stream=torch.cuda.current_stream())
    p1, w1 = _records(e1, 0, n, seed=21)
    p2, w2 = _records(e2, 0, n, seed=21)
    assert np.array_equal(p1, p2)
    ok = p1 >= 0
    npix = inst.nx * inst.ny
    dlt = w1[ok] - w2[ok]
    s1 = np.bincount(p1[ok], weights=dlt, minlength=npix)
    s2 = np.bincount(p1[ok], weights=dlt * dlt, minlength=npix)
    z = s1[s2 > 0] / np.sqrt(s2[s2 > 0])
    assert np.max(np.abs(z)) < 4.8 and np.mean(z * z) < 1.3, (np.max(np.abs(z)), np.mean(z * z))
    tot = dlt.sum() / math.sqrt((dlt * dlt).sum())
    assert abs(tot) < 4.0
    e1.close()
    e2.close()


def test_event_mode_refusals():
    inst = W.instrument()
    with pytest.raises(sas.SasError):
        sas.Experiment(inst, _ev(W.SPHERE, poly_dist=W.SCHULZ), stream=torch.cuda.current_stream())
    with pytest.raises(sas.SasError):
        sas.Experiment(inst, _ev(W.CYLINDER, iso=W.CAP, sigma_orient=0.2), stream=torch.cuda.current_stream())
    e = sas.Experiment(inst, _ev(W.SPHERE), stream=torch.cuda.current_stream())
    q = torch.zeros((4, 3), device="cuda")
    out = torch.empty(4, device="cuda")
    with pytest.raises(sas.SasError) as ex:
        sas.sas_eval_model(e.h, q, 4, out)
    assert ex.value.status == sas.SAS_ERR_STATE
    e.close()
