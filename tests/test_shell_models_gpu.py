"""Shelled uniaxial models (core-shell cylinder, hollow cylinder, core-shell
ellipsoid, core-shell bicelle; Eq. 1 region by region) on the GPU against the FP64 oracle:
model evaluations over every form of 2 J1(x)/x, records (quadrature and
per-event draws), detectors, a batch, the self-attenuation table and the
refusals. Pixels and counts bit-exact; weights of records and detectors at
the tolerances of the other models (FP32 1e-5 relative + 1e-7 of the
largest, FP64 1e-10 + 1e-13), on contrasts of one sign.

Model evaluations bound the error by the arithmetic of a sum of terms: each
FP32 term (sinc, 2 J1(x)/x, the sphere amplitude from the special-function
unit) carries an absolute error of at most 3e-6 of its value at Q = 0, so
|dF| <= 3e-6 S with S the sum of the terms' magnitudes, and
|dP| <= 1e-5 |P| + 6e-6 sqrt(|P| P_S) + 1e-7 P_S, where P_S is the forward
scattering of the same particle with every contrast made positive (P_S =
P(0) for contrasts of one sign). Contrasts of opposite signs (a shell
against the core, or the hollow cylinder's solvent core) cancel in F, and
the bound follows S, not F. FP64: 1e-10 |P| + 1e-13 P_S."""
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
    base = dict(kind=kind, radius=20.0, thickness=6.0, thickness_face=10.0, length=120.0, radius_polar=45.0,
                sld=1.0e-6, sld_shell=3.0e-6, sld_solvent=6.0e-6, volume_fraction=0.01, poly=0.1, n_poly=12,
                axis_theta=1.2, axis_phi=0.3)
    base.update(kw)
    return W.Model(**base)


MODELS = {
    "cscyl_cap": _m(W.CORE_SHELL_CYLINDER, sigma_orient=0.25, n_gamma=8, n_psi=8),
    "cscyl_iso_fp64": _m(W.CORE_SHELL_CYLINDER, precision=W.FP64, isotropic=W.ISOTROPIC, n_gamma=8, n_psi=8),
    "hollow_fixed": _m(W.HOLLOW_CYLINDER, poly=0.2, n_poly=24),
    "hollow_angles_fp64": _m(W.HOLLOW_CYLINDER, precision=W.FP64, isotropic=W.UNIFORM_ANGLES, n_gamma=8,
                             n_psi=8),
    "csell_cap": _m(W.CORE_SHELL_ELLIPSOID, sigma_orient=0.3, n_gamma=8, n_psi=8),
    "csell_iso_fp64": _m(W.CORE_SHELL_ELLIPSOID, precision=W.FP64, isotropic=W.ISOTROPIC, n_gamma=8, n_psi=8),
    "csell_sphere_limit": _m(W.CORE_SHELL_ELLIPSOID, radius=30.0, radius_polar=30.0, thickness=8.0,
                             thickness_face=8.0, poly=0.0, n_poly=1),
    # contrasts of opposite signs: the shell against the core
    "cscyl_opposite": _m(W.CORE_SHELL_CYLINDER, sld_shell=4.0e-6, sld_solvent=2.0e-6, poly=0.0, n_poly=1),
    "csell_opposite": _m(W.CORE_SHELL_ELLIPSOID, radius=30.0, radius_polar=30.0, thickness=8.0,
                         thickness_face=8.0, sld_shell=4.0e-6, sld_solvent=2.0e-6, poly=0.0, n_poly=1),
    "csell_opposite_fp64": _m(W.CORE_SHELL_ELLIPSOID, precision=W.FP64, sld_shell=4.0e-6, sld_solvent=2.0e-6,
                              isotropic=W.ISOTROPIC, n_gamma=8, n_psi=8),
    "bicelle_cap": _m(W.CORE_SHELL_BICELLE, sld_face=2.0e-6, sigma_orient=0.25, n_gamma=8, n_psi=8),
    "bicelle_opposite_fp64": _m(W.CORE_SHELL_BICELLE, precision=W.FP64, sld=4.0e-6, sld_face=1.0e-6,
                                sld_shell=5.0e-6, sld_solvent=2.0e-6, isotropic=W.ISOTROPIC, n_gamma=8, n_psi=8),
    "bicelle_opposite": _m(W.CORE_SHELL_BICELLE, sld=4.0e-6, sld_face=1.0e-6, sld_shell=5.0e-6,
                           sld_solvent=2.0e-6, poly=0.0, n_poly=1),
    "bicelle_event": _m(W.CORE_SHELL_BICELLE, sld_face=2.0e-6, poly=0.2, poly_dist=W.GAUSSIAN, n_poly=16,
                        isotropic=W.UNIFORM_ANGLES, sampling=W.PER_EVENT),
    "cscyl_event": _m(W.CORE_SHELL_CYLINDER, poly=0.2, poly_dist=W.GAUSSIAN, n_poly=16, isotropic=W.ISOTROPIC,
                      sampling=W.PER_EVENT),
    "hollow_event_fp64": _m(W.HOLLOW_CYLINDER, precision=W.FP64, poly=0.15, poly_dist=W.GAUSSIAN, n_poly=16,
                            isotropic=W.UNIFORM_ANGLES, sampling=W.PER_EVENT),
    "csell_event": _m(W.CORE_SHELL_ELLIPSOID, poly=0.15, poly_dist=W.GAUSSIAN, n_poly=16,
                      isotropic=W.ISOTROPIC, sampling=W.PER_EVENT),
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


def _p_s(m):
    """Forward scattering of the same particle with every contrast positive."""
    d = m.as_dict()
    if m.kind == W.HOLLOW_CYLINDER:
        # the hollow cylinder's two terms are the outer cylinder and the core:
        # a core-shell cylinder with both contrasts |drho|, renormalised from
        # <V_o> to the wall volume
        dr = abs(m.sld - m.sld_solvent)
        cs = W.Model(**dict(d, kind=W.CORE_SHELL_CYLINDER, sld=2 * dr, sld_shell=dr, sld_solvent=0.0,
                            thickness_face=0.0))
        prep = oracle.Prepared(cs)
        ro = prep.poly_r + m.thickness
        vo = np.sum(prep.poly_w * ro ** 2)
        vw = np.sum(prep.poly_w * (ro ** 2 - prep.poly_r ** 2))
        return oracle.dsigma(prep, np.zeros((1, 3)))[0] * vo / vw
    if m.kind == W.CORE_SHELL_BICELLE:
        dc, df, dr = abs(m.sld - m.sld_face), abs(m.sld_face - m.sld_shell), abs(m.sld_shell - m.sld_solvent)
        pos = W.Model(**dict(d, sld=dc + df + dr, sld_face=df + dr, sld_shell=dr, sld_solvent=0.0))
        return oracle.dsigma(oracle.Prepared(pos), np.zeros((1, 3)))[0]
    d1, d2 = abs(m.sld - m.sld_shell), abs(m.sld_shell - m.sld_solvent)
    pos = W.Model(**dict(d, sld=d1 + d2, sld_shell=d2, sld_solvent=0.0))
    return oracle.dsigma(oracle.Prepared(pos), np.zeros((1, 3)))[0]


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
    ps = _p_s(m)
    assert ps >= ref[-1] * (1 - 1e-12)
    if m.precision == W.FP64:
        tol = 1e-10 * np.abs(ref) + 1e-13 * ps
    else:
        tol = 1e-5 * np.abs(ref) + 6e-6 * np.sqrt(np.abs(ref) * ps) + 1e-7 * ps
    err = np.abs(got - ref)
    assert np.all(err <= tol), (name, np.max(err / tol))
    e.close()


def _records(e, first, n, seed):
    pix = torch.empty(n, dtype=torch.int32, device="cuda")
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    sas.sas_trace_records(e.h, first, n, seed, pix, w)
    torch.cuda.synchronize()
    return pix.cpu().numpy().astype(np.int64), w.cpu().numpy()


@pytest.mark.parametrize("name", ["cscyl_cap", "cscyl_iso_fp64", "hollow_fixed", "hollow_angles_fp64",
                                  "csell_cap", "csell_iso_fp64", "cscyl_event", "hollow_event_fp64",
                                  "csell_event", "bicelle_cap", "bicelle_opposite_fp64", "bicelle_event"])
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


@pytest.mark.parametrize("name", ["cscyl_cap", "hollow_fixed", "csell_cap", "csell_event", "bicelle_cap"])
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
    m = W.Model(**{**MODELS["cscyl_cap"].as_dict(), "self_attenuation": 1})
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


@pytest.mark.parametrize("kind,bad", [(W.CORE_SHELL_CYLINDER, dict(thickness=-1.0)),
                                      (W.CORE_SHELL_CYLINDER, dict(thickness_face=-1.0)),
                                      (W.CORE_SHELL_CYLINDER, dict(length=0.0)),
                                      (W.HOLLOW_CYLINDER, dict(thickness=0.0)),
                                      (W.CORE_SHELL_ELLIPSOID, dict(radius_polar=0.0)),
                                      (W.CORE_SHELL_ELLIPSOID, dict(thickness_face=float("nan"))),
                                      (W.CORE_SHELL_BICELLE, dict(sld_face=float("inf")))])
def test_refusals(kind, bad):
    m = _m(kind, **bad)
    with pytest.raises(sas.SasError):
        sas.Experiment(W.instrument(), m, stream=torch.cuda.current_stream())
