"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (FP32 path):
  * model evaluations: |gpu - oracle| <= 1e-5 |oracle| + 1e-7 dSigma(0)
  * per-neutron weights (records): same form, scale = largest weight
  * pixel choice and per-bin counts: bit-exact (integer arithmetic on the
    same Philox words)
  * total detected weight: relative 1e-4; every bin within 3 sigma of its
    counting error (and, stronger, within 1e-4 relative where it is not tiny)
FP64 path: 1e-10 relative.
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
    torch.cuda.init()
    yield


def _exp(inst, model):
    return sas.Experiment(inst, model, stream=torch.cuda.current_stream())


# ----------------------------------------------------------------- models

def _model_cases():
    cs = W.core_shell_config()["model"]
    cyl = W.cylinder_config()["model"]
    cases = {
        "sphere_mono": W.Model(kind=W.SPHERE, radius=50.0, sld=2e-6, volume_fraction=0.01),
        "sphere_poly": W.Model(kind=W.SPHERE, radius=80.0, sld=2e-6, volume_fraction=0.01,
                               poly=0.3, n_poly=40),
        "core_shell_py": cs,
        "core_shell_nopy": W.Model(**{**cs.as_dict(), "sq_kind": W.SQ_NONE}),
        "cylinder_oriented": W.Model(kind=W.CYLINDER, radius=120.0, length=200.0, sld=1e-6,
                                     volume_fraction=0.01, axis_theta=math.radians(60),
                                     axis_phi=math.radians(60)),
        "cylinder_cfg": cyl,
        "cylinder_iso": W.Model(kind=W.CYLINDER, radius=30.0, length=150.0, sld=1e-6,
                                volume_fraction=0.01, poly=0.1, n_poly=20, isotropic=1,
                                n_gamma=40, n_psi=40),
        "ellipsoid": W.Model(kind=W.ELLIPSOID, radius=30.0, radius_polar=90.0, sld=3e-6,
                             volume_fraction=0.02, poly=0.15, n_poly=24,
                             sigma_orient=math.radians(20), axis_theta=1.0, axis_phi=0.3,
                             n_gamma=24, n_psi=24),
    }
    return cases


CASES = _model_cases()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", [W.FP32, W.FP64])
def test_eval_model_parity(name, precision):
    m = W.Model(**{**CASES[name].as_dict(), "precision": precision})
    heavy = m.kind in (W.CYLINDER, W.ELLIPSOID) and m.n_gamma * m.n_psi > 1000
    n = 601 if heavy else 5003            # several blocks and a ragged tail
    q = W.random_q(n, 0.25, seed=17 + precision)
    q[0] = 0.0                            # Q = 0 exactly
    q[1] = [1e-6, 0.0, 0.0]
    dt = torch.float32 if precision == W.FP32 else torch.float64
    qd = torch.tensor(q, dtype=dt, device="cuda").contiguous()
    out = torch.empty(n, dtype=dt, device="cuda")
    e = _exp(W.instrument(), m)
    sas.sas_eval_model(e.h, qd, n, out)
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    ref = oracle.dsigma(m, qd.double().cpu().numpy())
    p0 = oracle.dsigma(m, np.zeros((1, 3)))[0]
    if precision == W.FP32:
        tol = 1e-5 * np.abs(ref) + 1e-7 * p0
    else:
        tol = 1e-10 * np.abs(ref) + 1e-13 * p0
    bad = np.abs(got - ref) > tol
    assert not bad.any(), (name, int(bad.sum()), q[bad][:3], got[bad][:3], ref[bad][:3])
    e.close()


def test_core_shell_series_switch_and_extreme_arguments():
    """The FP32 core-shell node loop switches from the small-x series to the
    closed form at x = q r = 1.5 for each radius: Q on both sides of the
    switch of every core and outer node radius, tiny Q, and Q up to 2 / A
    (x up to about 150, far beyond the detector's range)."""
    m = CASES["core_shell_py"]
    prep = oracle.Prepared(m)
    radii = np.concatenate([prep.poly_r, prep.poly_r + m.thickness])
    qs = np.concatenate([1.5 / radii * (1 - 3e-7), 1.5 / radii * (1 + 3e-7),
                         np.logspace(-7, -2, 40), np.linspace(0.3, 2.0, 60)])
    rng = np.random.default_rng(3)
    d = rng.normal(size=(len(qs), 3))
    q = d / np.linalg.norm(d, axis=1)[:, None] * qs[:, None]
    qd = torch.tensor(q, dtype=torch.float32, device="cuda").contiguous()
    out = torch.empty(len(q), dtype=torch.float32, device="cuda")
    e = _exp(W.instrument(), m)
    sas.sas_eval_model(e.h, qd, len(q), out)
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    ref = oracle.dsigma(prep, qd.double().cpu().numpy())
    p0 = oracle.dsigma(prep, np.zeros((1, 3)))[0]
    bad = np.abs(got - ref) > 1e-5 * np.abs(ref) + 1e-7 * p0
    assert not bad.any(), (int(bad.sum()), qs[bad][:3], got[bad][:3], ref[bad][:3])
    near = np.abs(ref) > 1e-3 * p0
    assert np.max(np.abs(got - ref)[near] / np.abs(ref)[near]) < 1e-5
    e.close()


EXTREME = {
    "sphere_r200": W.Model(kind=W.SPHERE, radius=200.0, sld=2e-6, volume_fraction=0.01, poly=0.1, n_poly=20),
    "core_shell_thick": W.Model(kind=W.CORE_SHELL, radius=150.0, thickness=60.0, sld=1e-6, sld_shell=3e-6,
                                sld_solvent=6e-6, volume_fraction=0.05, poly=0.1, n_poly=20),
    "cylinder_long": W.Model(kind=W.CYLINDER, radius=40.0, length=2000.0, sld=1e-6, volume_fraction=0.01,
                             poly=0.1, n_poly=12, sigma_orient=math.radians(10), axis_theta=1.0, axis_phi=0.5,
                             n_gamma=12, n_psi=12),
    "ellipsoid_big": W.Model(kind=W.ELLIPSOID, radius=150.0, radius_polar=300.0, sld=2e-6, volume_fraction=0.01,
                             poly=0.1, n_poly=12, sigma_orient=0.2, n_gamma=10, n_psi=10),
    "parallelepiped_big": W.Model(kind=W.PARALLELEPIPED, radius=60.0, radius_b=120.0, radius_polar=400.0,
                                  sld=2e-6, volume_fraction=0.01, poly=0.1, n_poly=8, isotropic=W.UNIFORM_ANGLES,
                                  n_gamma=6, n_psi=6, n_rot=6),
}


@pytest.mark.parametrize("name", list(EXTREME))
def test_fp32_large_arguments(name):
    """FP32 evaluations where q r reaches a few hundred (large particles,
    |Q| up to 0.5 1/A), where the special-function unit's argument scaling
    loses the most: same tolerance as the other evaluations."""
    m = EXTREME[name]
    n = 3001
    q = W.random_q(n, 0.5, seed=29)
    qd = torch.tensor(q, dtype=torch.float32, device="cuda").contiguous()
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    e = _exp(W.instrument(), m)
    sas.sas_eval_model(e.h, qd, n, out)
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    prep = oracle.Prepared(m)
    ref = oracle.dsigma(prep, qd.double().cpu().numpy())
    p0 = oracle.dsigma(prep, np.zeros((1, 3)))[0]
    bad = np.abs(got - ref) > 1e-5 * np.abs(ref) + 1e-7 * p0
    assert not bad.any(), (name, int(bad.sum()), got[bad][:3], ref[bad][:3])
    e.close()


# ----------------------------------------------------------- per-neutron

def _records(e, first, n, seed):
    pix = torch.empty(n, dtype=torch.int32, device="cuda")
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    sas.sas_trace_records(e.h, first, n, seed, pix, w)
    torch.cuda.synchronize()
    return pix.cpu().numpy().astype(np.int64), w.cpu().numpy()


RECORD_CASES = {
    "sphere_fp64": (W.sphere_config()["instrument"],
                    W.Model(**{**W.sphere_config()["model"].as_dict()})),
    "sphere_fp32": (W.instrument(), W.Model(kind=W.SPHERE, radius=50.0, sld=2e-6,
                                            volume_fraction=0.01)),
    "core_shell": (W.instrument(), W.core_shell_config()["model"]),
    "cylinder_small_grid": (W.instrument(nx=256, ny=256),
                            W.Model(**{**W.cylinder_config()["model"].as_dict(),
                                       "n_gamma": 16, "n_psi": 16})),
    "ellipsoid_mu": (W.Instrument(mu=50.0, nx=100, ny=60), CASES["ellipsoid"]),
    "odd_detector": (W.Instrument(nx=37, ny=5, pixel_x=0.02, pixel_y=0.05),
                     W.Model(kind=W.SPHERE, radius=40.0, poly=0.1, n_poly=10)),
}


@pytest.mark.parametrize("name", list(RECORD_CASES))
def test_records_parity(name):
    inst, m = RECORD_CASES[name]
    n = 4099
    for first in (0, 123456789, (1 << 40) + 7):
        e = _exp(inst, m)
        pix, w = _records(e, first, n, seed=1)
        po, wo = oracle.records(inst, m, n, seed=1, first=first)
        assert np.array_equal(pix, po)
        scale = np.max(np.abs(wo))
        rel = 1e-10 if m.precision == W.FP64 else 1e-5
        absf = 1e-13 if m.precision == W.FP64 else 1e-7
        err = np.abs(w - wo)
        assert np.all(err <= rel * np.abs(wo) + absf * scale), (name, first, err.max())
        e.close()


def test_full_cylinder_grid_records():
    """76x76 orientation x 40 Schulz nodes on a few neutrons of the cylinder set-up."""
    cfg = W.cylinder_config()
    e = _exp(cfg["instrument"], cfg["model"])
    n = 96
    pix, w = _records(e, 5000, n, seed=1)
    po, wo = oracle.records(cfg["instrument"], cfg["model"], n, seed=1, first=5000)
    assert np.array_equal(pix, po)
    assert np.all(np.abs(w - wo) <= 1e-5 * np.abs(wo) + 1e-7 * np.max(wo))
    e.close()


def test_experiment_id_and_seed_change_streams():
    inst, m = RECORD_CASES["sphere_fp32"]
    e = _exp(inst, m)
    p0, _ = _records(e, 0, 1000, seed=1)
    sas.sas_set_experiment_id(e.h, 5)
    p1, _ = _records(e, 0, 1000, seed=1)
    p2, w2 = _records(e, 0, 1000, seed=2)
    po, wo = oracle.records(inst, m, 1000, seed=2, exp_id=5)
    assert not np.array_equal(p0, p1) and not np.array_equal(p1, p2)
    assert np.array_equal(p2, po)
    e.close()


# ----------------------------------------------------------------- tallies

def _check_detector(d, ref, n, total_rel=1e-4, bin_rel=1e-4, exact_counts=True):
    if exact_counts:
        assert np.array_equal(d["count"].astype(np.uint64), ref["count"].astype(np.uint64))
    sw, so = d["sum_w"], ref["sum_w"]
    assert abs(sw.sum() - so.sum()) <= total_rel * abs(so.sum())
    # 3 sigma of the counting error of each bin (per incident neutron)
    var = np.maximum(ref["sum_w2"] - so ** 2 / n, 0.0)
    sig = np.sqrt(var)
    assert np.all(np.abs(sw - so) <= 3 * sig + 1e-12 * np.max(so))
    # stronger: same streams, so the bins agree to FP32 rounding
    big = so > 1e-6 * so.max()
    assert np.all(np.abs(sw - so)[big] <= bin_rel * so[big])
    assert abs(d["trans"] - ref["trans"]) <= 1e-6 * max(1.0, abs(ref["trans"]))


TRACE_CASES = {
    "sphere_fp64": (W.sphere_config()["instrument"], W.sphere_config()["model"], 300000),
    "sphere_fp32_smem": (W.instrument(), RECORD_CASES["sphere_fp32"][1], 1000003),
    "core_shell_smem": (W.instrument(), W.core_shell_config()["model"], 400000),
    "cylinder_global": (W.instrument(nx=256, ny=256), RECORD_CASES["cylinder_small_grid"][1], 20000),
    "ellipsoid_mu": (RECORD_CASES["ellipsoid_mu"][0], CASES["ellipsoid"], 30000),
    "odd_detector": (RECORD_CASES["odd_detector"][0], RECORD_CASES["odd_detector"][1], 200001),
}


@pytest.mark.parametrize("name", list(TRACE_CASES))
def test_trace_parity(name):
    inst, m, n = TRACE_CASES[name]
    e = _exp(inst, m)
    e.trace(n, seed=1)
    d = e.read()
    ref = oracle.trace(inst, m, n, seed=1)
    _check_detector(d, ref, n)
    e.close()


def test_trace_range_split_equals_whole():
    inst, m, _ = TRACE_CASES["core_shell_smem"]
    e = _exp(inst, m)
    n = 300001
    e.trace(n, seed=3)
    whole = e.read()
    sas.sas_reset_detector(e.h)
    for a, b in ((0, 77777), (77777, 200000), (200000, n)):
        e.trace_range(a, b - a, seed=3)
    parts = e.read()
    assert np.array_equal(whole["count"], parts["count"])
    assert np.allclose(whole["sum_w"], parts["sum_w"], rtol=1e-5, atol=1e-9 * whole["sum_w"].max())
    e.close()


def test_empty_and_tiny_traces():
    inst, m, _ = TRACE_CASES["core_shell_smem"]
    e = _exp(inst, m)
    e.trace(0, seed=1)
    d = e.read()
    assert d["count"].sum() == 0 and d["sum_w"].sum() == 0.0 and d["trans"] == 0.0
    for n in (1, 31, 33):
        e.trace(n, seed=9)
        d = e.read()
        ref = oracle.trace(inst, m, n, seed=9)
        assert np.array_equal(d["count"], ref["count"].astype(np.uint64))
        assert np.allclose(d["sum_w"], ref["sum_w"], rtol=1e-5, atol=1e-7 * ref["sum_w"].max())
    e.close()


def test_state_errors():
    e = sas.sas_create_experiment(sas.make_instrument(W.instrument()))
    with pytest.raises(sas.SasError) as ex:
        sas.sas_trace(e, 10, 1)
    assert ex.value.status == sas.SAS_ERR_STATE
    with pytest.raises(sas.SasError) as ex:
        sas.sas_set_model(e, W.Model(kind=7))
    assert ex.value.status == sas.SAS_ERR_ARG
    with pytest.raises(sas.SasError):
        sas.sas_read_detector(e, 10)      # wrong pixel count
    sas.sas_destroy_experiment(e)


# ------------------------------------------------- full-size configuration

def test_full_size_core_shell_properties():
    """The 1e9-neutron core-shell run in the benchmark's launch configuration:
    every history is counted once; the index range [1e9 - 4099, 1e9) agrees
    with the oracle history by history; the total weight agrees with the
    oracle's estimate from a 1e6 sample within its statistical error."""
    cfg = W.core_shell_config()
    n = cfg["n_neutrons"]
    e = _exp(cfg["instrument"], cfg["model"])
    e.trace(n, seed=1)
    d = e.read()
    assert int(d["count"].sum()) == n
    assert d["trans"] == pytest.approx(n, rel=1e-12)
    pix, w = _records(e, n - 4099, 4099, seed=1)
    po, wo = oracle.records(cfg["instrument"], cfg["model"], 4099, seed=1, first=n - 4099)
    assert np.array_equal(pix, po)
    assert np.all(np.abs(w - wo) <= 1e-5 * np.abs(wo) + 1e-7 * wo.max())
    ns = 10 ** 6
    ref = oracle.trace(cfg["instrument"], cfg["model"], ns, seed=1, first=123456789)
    mean = ref["sum_w"].sum() / ns
    sd = math.sqrt(max(ref["sum_w2"].sum() / ns - mean ** 2, 0.0) / ns)
    assert abs(d["sum_w"].sum() / n - mean) < 4 * sd
    e.close()
