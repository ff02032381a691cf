"""Shape-independent laws (dSigma/dOmega = f_scale f(|Q|)) on the GPU
against the FP64 oracle: evaluations of every law in FP32 and FP64, records,
a traced detector, and the refusals.

Evaluation tolerance. The laws that stay within a few decades of their
largest value over the whole grid and have no zeros (power law, Lorentzian,
Debye-Anderson-Brumberger, Teubner-Strey) are held to the relative part of
T1 alone (FP32 1e-5, FP64 1e-10): an absolute floor taken from their
largest value would exceed most of the values themselves (the power law
spans 14 decades from |Q| = 1e-4 to 1). The laws with a finite forward
value whose tails fall below FP32's range (Guinier, Gaussian coil) or
vanish away from a peak (Gaussian peak), and the fractals whose building
blocks' sphere factor has zeros on the grid, keep T1's absolute part, 1e-7
of their forward (peak) value, the same rule as the form factors' 1e-7
P(0). The fractals of 2 A blocks (no zero below |Q| = 1, five decades at
most) and the spinodal peak (no zero for |Q| > 0) are held to the relative
part."""
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


# laws held to the relative tolerance alone (no zeros, no underflow on the grid)
RELATIVE_ONLY = {"lorentz", "dab", "power_law", "teubner_strey", "peak_lorentz", "two_power_law",
                 "guinier_porod", "guinier_porod_rod", "gauss_lorentz_gel", "poly_coil", "star",
                 "mass_fractal", "fractal", "spinodal", "excluded_volume", "excluded_volume_swollen"}

LAWS = {
    "guinier": (W.GUINIER, (40.0, 0.0, 0.0)),
    "coil": (W.GAUSS_COIL, (35.0, 0.0, 0.0)),
    "lorentz": (W.LORENTZ, (25.0, 0.0, 0.0)),
    "dab": (W.DAB, (60.0, 0.0, 0.0)),
    "power_law": (W.POWER_LAW, (3.6, 0.0, 0.0)),
    "gauss_peak": (W.GAUSS_PEAK, (0.05, 0.008, 0.0)),
    "teubner_strey": (W.TEUBNER_STREY, (1.0, -120.0, 1.0e4)),
    "peak_lorentz": (W.PEAK_LORENTZ, (0.05, 0.01, 0.0)),
    "two_power_law": (W.TWO_POWER_LAW, (0.03, 1.7, 3.9)),
    "guinier_porod": (W.GUINIER_POROD, (40.0, 0.0, 4.0)),
    "guinier_porod_rod": (W.GUINIER_POROD, (30.0, 1.0, 3.5)),
    "gauss_lorentz_gel": (W.GAUSS_LORENTZ_GEL, (80.0, 25.0, 0.3)),
    "poly_coil": (W.POLY_GAUSS_COIL, (50.0, 0.5, 0.0)),
    "star": (W.STAR_POLYMER, (40.0, 6.0, 0.0)),
    # building blocks of 2 A: no zero of the sphere factor below |Q| = 1 (relative only)
    "mass_fractal": (W.MASS_FRACTAL, (2.0, 2.0, 100.0)),
    "mass_fractal_blocks": (W.MASS_FRACTAL, (25.0, 2.6, 300.0)),
    "fractal": (W.FRACTAL, (2.0, 2.1, 120.0)),
    "spinodal": (W.SPINODAL, (0.03, 3.0, 0.0)),
    "excluded_volume": (W.POLYMER_EXCL_VOLUME, (40.0, 5.0 / 3.0, 0.0)),
    "excluded_volume_swollen": (W.POLYMER_EXCL_VOLUME, (25.0, 4.5, 0.0)),
    "linear_pearls": (W.LINEAR_PEARLS, (20.0, 10.0, 8.0)),
    "linear_pearls_long": (W.LINEAR_PEARLS, (6.0, 4.0, 60.0)),
}


def _m(name, precision):
    fn, p = LAWS[name]
    return W.Model(kind=W.SHAPE_INDEPENDENT, precision=precision, function=fn, f_scale=0.37, f_p0=p[0],
                   f_p1=p[1], f_p2=p[2])


@pytest.mark.parametrize("precision", [W.FP32, W.FP64])
@pytest.mark.parametrize("name", list(LAWS))
def test_law_parity(name, precision):
    m = _m(name, precision)
    rng = np.random.default_rng(9)
    d = rng.normal(size=(3000, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    qm = np.concatenate([rng.uniform(1e-4, 0.02, 1000), rng.uniform(0.02, 0.2, 1500), rng.uniform(0.2, 1.0, 500)])
    q = d * qm[:, None]
    e = sas.Experiment(W.instrument(), m, stream=torch.cuda.current_stream())
    dt = torch.float64 if precision == W.FP64 else torch.float32
    out = torch.empty(len(q), dtype=dt, device="cuda")
    sas.sas_eval_model(e.h, torch.tensor(q, dtype=dt, device="cuda"), len(q), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    # the oracle at the Q the device saw (FP32 inputs rounded first)
    qd = torch.tensor(q, dtype=dt).double().numpy()
    ref = oracle.dsigma(oracle.Prepared(m), qd)
    rel, ab = (1e-10, 1e-13) if precision == W.FP64 else (1e-5, 1e-7)
    if name in RELATIVE_ONLY:
        ab = 0.0
    err = np.abs(got - ref)
    assert np.all(err <= rel * np.abs(ref) + ab * ref.max()), \
        (name, np.max(err / (rel * np.abs(ref) + ab * ref.max())))
    e.close()


def _records(e, first, n, seed):
    pix = torch.empty(n, dtype=torch.int32, device="cuda")
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    sas.sas_trace_records(e.h, first, n, seed, pix, w)
    torch.cuda.synchronize()
    return pix.cpu().numpy().astype(np.int64), w.cpu().numpy()


@pytest.mark.parametrize("name,precision", [("coil", W.FP32), ("dab", W.FP64), ("teubner_strey", W.FP32),
                                            ("poly_coil", W.FP32), ("star", W.FP64), ("guinier_porod", W.FP32),
                                            ("fractal", W.FP32), ("spinodal", W.FP64),
                                            ("excluded_volume", W.FP32), ("linear_pearls", W.FP32)])
def test_records_and_trace(name, precision):
    m = _m(name, precision)
    inst = W.instrument(nx=64, ny=64)
    e = sas.Experiment(inst, m, stream=torch.cuda.current_stream())
    n = 5001
    pix, w = _records(e, 7, n, seed=2)
    po, wo = oracle.records(inst, m, n, seed=2, first=7)
    assert np.array_equal(pix, po)
    rel, ab = (1e-10, 1e-13) if precision == W.FP64 else (1e-5, 1e-7)
    assert np.all(np.abs(w - wo) <= rel * np.abs(wo) + ab * np.max(wo))
    nt = 100003
    e.trace(nt, seed=5)
    d = e.read()
    ref = oracle.trace(inst, m, nt, seed=5)
    assert np.array_equal(d["count"].ravel(), ref["count"].ravel().astype(np.uint64))
    so = ref["sum_w"].ravel()
    big = so > 1e-6 * so.max()
    assert np.all(np.abs(d["sum_w"].ravel() - so)[big] <= 1e-4 * so[big])
    e.close()


@pytest.mark.parametrize("bad", [dict(function=16), dict(f_p0=0.0), dict(f_scale=-1.0),
                                 dict(function=W.MASS_FRACTAL, f_p0=10.0, f_p1=1.0, f_p2=50.0),
                                 dict(function=W.FRACTAL, f_p0=0.0, f_p1=2.0, f_p2=50.0),
                                 dict(function=W.SPINODAL, f_p0=0.03, f_p1=0.0),
                                 dict(function=W.POLYMER_EXCL_VOLUME, f_p0=30.0, f_p1=1.0),
                                 dict(function=W.LINEAR_PEARLS, f_p0=10.0, f_p1=2.0, f_p2=2.5),
                                 dict(sampling=W.PER_EVENT), dict(self_attenuation=1),
                                 dict(sq_kind=W.SQ_HARD_SPHERE_PY, sq_radius=10.0, sq_fraction=0.1)])
def test_refusals(bad):
    m = W.Model(**{**_m("guinier", W.FP32).as_dict(), **bad})
    with pytest.raises(sas.SasError):
        sas.Experiment(W.instrument(), m, stream=torch.cuda.current_stream())
    ts = W.Model(**{**_m("teubner_strey", W.FP32).as_dict(), "f_p1": -300.0})   # a2 + c1 Q^2 + c2 Q^4 < 0 somewhere
    with pytest.raises(sas.SasError):
        sas.Experiment(W.instrument(), ts, stream=torch.cuda.current_stream())
    inst = W.instrument(nx=32, ny=32)
    with pytest.raises(sas.SasError):
        sas.sas_create_batch(inst, [_m("guinier", W.FP32)], np.array([1000], np.uint64),
                             stream=torch.cuda.current_stream())
