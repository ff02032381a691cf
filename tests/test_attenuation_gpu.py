"""Self-attenuation (the beam depleted by the particles' own scattering) on
the GPU against the FP64 oracle.

* the total cross section Sigma_s at the 8 Chebyshev wavelengths of the
  band, evaluated by the GPU kernel of the model's kind and precision, vs the
  oracle's FP64 evaluation of the same rule: FP32 models 1e-5 relative,
  FP64 1e-10; the Chebyshev coefficients follow;
* the full-size cylinder model (40 Schulz nodes x 76 x 76 orientation
  nodes), sampled: single |Q| panels of Sigma_s at one wavelength;
* per-history records with self-attenuation on: pixels bit-exact, weights
  to the records tolerance (FP32 1e-5 relative + 1e-7 of the largest,
  FP64 1e-10);
* traced detectors and the transmitted sum; a batch mixing models with and
  without it; refusals.
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


def _att(m):
    return W.Model(**{**m.as_dict(), "self_attenuation": 1})


CASES = {
    "sphere_fp64": (W.instrument(), _att(W.Model(kind=W.SPHERE, precision=W.FP64, radius=50.0, poly=0.1,
                                                 n_poly=12))),
    "core_shell_py": (W.instrument(), _att(W.core_shell_config()["model"])),
    "cylinder_fixed": (W.instrument(nx=64, ny=64), _att(W.Model(kind=W.CYLINDER, radius=20.0, length=300.0,
                                                                axis_theta=1.2, axis_phi=0.3))),
    "cylinder_cap": (W.instrument(nx=64, ny=64), _att(W.Model(kind=W.CYLINDER, radius=20.0, length=200.0,
                                                              poly=0.1, n_poly=6, sigma_orient=0.25,
                                                              n_gamma=6, n_psi=8))),
    "ellipsoid_iso": (W.Instrument(nx=50, ny=30, mu=30.0),
                      _att(W.Model(kind=W.ELLIPSOID, radius=25.0, radius_polar=60.0, isotropic=W.ISOTROPIC,
                                   n_gamma=8, n_psi=8))),
    "triaxial_fp64": (W.instrument(nx=48, ny=48),
                      _att(W.Model(kind=W.TRIAXIAL_ELLIPSOID, precision=W.FP64, radius=15.0, radius_b=25.0,
                                   radius_polar=40.0, axis_theta=0.8, axis_phi=0.2, axis_psi=0.5))),
    "parallelepiped": (W.instrument(nx=48, ny=48),
                       _att(W.Model(kind=W.PARALLELEPIPED, radius=12.0, radius_b=20.0, radius_polar=35.0,
                                    poly=0.1, n_poly=4, isotropic=W.UNIFORM_ANGLES, n_gamma=4, n_psi=4,
                                    n_rot=4))),
    "monochromatic": (W.Instrument(dlambda_rel=0.0), _att(W.Model(kind=W.SPHERE, radius=40.0))),
}


def _tol(m):
    return (1e-10, 1e-13) if m.precision == W.FP64 else (1e-5, 1e-7)


@pytest.mark.parametrize("name", list(CASES))
def test_table_parity(name):
    inst, m = CASES[name]
    e = sas.Experiment(inst, m, stream=torch.cuda.current_stream())
    t = sas.sas_attenuation_table(e.h)
    lam, mu, c = oracle.att_table(inst, m)
    assert len(t["lam"]) == len(lam) == (1 if inst.dlambda_rel == 0.0 else 8)
    assert np.allclose(t["lam"], lam, rtol=1e-15, atol=0)
    rel = _tol(m)[0]
    assert np.all(np.abs(t["mu_s"] - mu) <= rel * np.abs(mu)), (name, np.max(np.abs(t["mu_s"] / mu - 1)))
    assert np.all(np.abs(t["coef"] - c) <= rel * abs(c[0]) + 1e-12)
    # any wavelength, through the general entry point
    s, parts = sas.sas_total_cross_section(e.h, inst.lambda0)
    lmin = inst.lambda0 * (1 - inst.dlambda_rel)
    assert len(parts) == oracle.sigma_s_npanels(m, lmin)
    assert s == pytest.approx(oracle.sigma_s(m, inst.lambda0, lmin), rel=rel)
    assert s == pytest.approx(parts.sum(), rel=1e-12)
    e.close()


def test_plain_model_has_no_table_but_a_cross_section():
    inst = W.instrument()
    m = W.core_shell_config()["model"]
    e = sas.Experiment(inst, m, stream=torch.cuda.current_stream())
    assert len(sas.sas_attenuation_table(e.h)["lam"]) == 0
    s, _ = sas.sas_total_cross_section(e.h, 5.0)
    assert s == pytest.approx(oracle.sigma_s(m, 5.0, inst.lambda0 * (1 - inst.dlambda_rel)), rel=1e-5)
    e.close()


def test_full_size_cylinder_sampled_panels():
    """The cylinder workload's model at full size (231 040 terms per
    evaluation): single panels of Sigma_s at one wavelength."""
    cfg = W.cylinder_config()
    inst, m = cfg["instrument"], _att(cfg["model"])
    e = sas.Experiment(inst, m, stream=torch.cuda.current_stream())
    lmin = inst.lambda0 * (1 - inst.dlambda_rel)
    lam = 6.3
    s, parts = sas.sas_total_cross_section(e.h, lam)
    n = oracle.sigma_s_npanels(m, lmin)
    assert len(parts) == n
    prep = oracle.Prepared(m)
    for i in (0, 3, 9, n - 1):
        ref = oracle.sigma_s_panel(prep, lam, lmin, i)
        assert parts[i] == pytest.approx(ref, rel=1e-5), i
    # the table the trace uses is the same rule at the Chebyshev wavelengths
    t = sas.sas_attenuation_table(e.h)
    assert len(t["lam"]) == 8 and np.all(t["mu_s"] > 0)
    s0, _ = sas.sas_total_cross_section(e.h, float(t["lam"][0]))
    assert 1e10 * s0 == pytest.approx(t["mu_s"][0], rel=1e-12)
    e.close()


def _records(e, first, n, seed):
    pix = torch.empty(n, dtype=torch.int32, device="cuda")
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    sas.sas_trace_records(e.h, first, n, seed, pix, w)
    torch.cuda.synchronize()
    return pix.cpu().numpy().astype(np.int64), w.cpu().numpy()


@pytest.mark.parametrize("name", ["sphere_fp64", "core_shell_py", "cylinder_cap", "ellipsoid_iso",
                                  "triaxial_fp64", "parallelepiped"])
def test_records_parity(name):
    inst, m = CASES[name]
    e = sas.Experiment(inst, m, stream=torch.cuda.current_stream())
    n = 6007
    for first in (0, 123456789):
        pix, w = _records(e, first, n, seed=13)
        po, wo = oracle.records(inst, m, n, seed=13, first=first)
        assert np.array_equal(pix, po)
        rel, absf = _tol(m)
        scale = np.max(np.abs(wo))
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


def test_trace_parity_core_shell():
    inst, m = CASES["core_shell_py"]
    n = 300001
    e = sas.Experiment(inst, m, stream=torch.cuda.current_stream())
    e.trace(n, seed=4)
    d = e.read()
    ref = oracle.trace(inst, m, n, seed=4)
    _check_detector(d, ref, n)
    # the beam is visibly depleted: mu_s l ~ 0.06 for this sample
    assert d["trans"] / n < 0.96
    e.close()


def test_batch_with_and_without_self_attenuation():
    inst = W.instrument(nx=64, ny=64)
    cs = W.core_shell_config()["model"]
    models = [_att(cs), cs, _att(W.Model(kind=W.CYLINDER, radius=20.0, length=200.0, poly=0.1, n_poly=6,
                                         sigma_orient=0.25, n_gamma=6, n_psi=8)),
              _att(W.Model(kind=W.SPHERE, radius=30.0, poly=0.2, n_poly=10))]
    counts = np.array([30001, 30001, 20000, 25000], dtype=np.uint64)
    b = sas.sas_create_batch(inst, models, counts, stream=torch.cuda.current_stream())
    sas.sas_trace_batch(b, seed=9)
    npix = inst.nx * inst.ny
    for k, m in enumerate(models):
        d = sas.sas_read_batch_detector(b, k, npix)
        ref = oracle.trace(inst, m, int(counts[k]), seed=9, exp_id=k)
        _check_detector(d, ref, int(counts[k]))
    sas.sas_destroy_batch(b)


def test_refusals():
    inst = W.instrument()
    ev = _att(W.Model(kind=W.SPHERE, radius=30.0, poly=0.2, poly_dist=W.GAUSSIAN, n_poly=8,
                      sampling=W.PER_EVENT))
    with pytest.raises(sas.SasError):
        sas.Experiment(inst, ev, stream=torch.cuda.current_stream())
    bad = W.Model(**{**W.core_shell_config()["model"].as_dict(), "self_attenuation": 2})
    with pytest.raises(sas.SasError):
        sas.Experiment(inst, bad, stream=torch.cuda.current_stream())
    npix = inst.nx * inst.ny
    sw = torch.zeros(npix, dtype=torch.float64, device="cuda")
    cnt = torch.zeros(npix, dtype=torch.int64, device="cuda")
    tr = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(sas.SasError):
        sas.sas_trace_batch_static(inst, [_att(W.core_shell_config()["model"])], [1000], 1, sw, sw, cnt, tr)
