"""Pins of the oracle's per-event sampling estimator (Sec. II.B).

The paper draws, for every scattering event, the polydisperse radius from a
Gaussian (redrawing non-positive values) and the particle axis from uniform
angles theta ~ U[0, pi], phi ~ U[0, 2 pi]. The oracle samples the restricted
Gaussian by inversion. These tests pin:

* erfcinv against scipy;
* the radius draw against scipy's truncated-normal quantile function;
* the quadrature nodes of the same distributions against closed forms;
* the axis draws against their definitions;
* the invariant of the method: the per-event estimator averages to the
  quadrature estimator over matching distributions, at fixed Q and over
  whole traced detectors (same histories, per-pixel z-scores).
"""
import math

import numpy as np
import pytest

import oracle
import sas_workloads as W

sp = pytest.importorskip("scipy.special")
st = pytest.importorskip("scipy.stats")


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def _word(u):
    """A 32-bit word whose uniform ((x >> 9) + 0.5) 2^-23 is closest to u."""
    k = np.clip(np.floor(np.asarray(u) * 8388608.0), 0, 8388607).astype(np.int64)
    return (k << 9), (k + 0.5) / 8388608.0


def test_erfcinv_matches_scipy():
    ys = np.concatenate([np.logspace(-300, -1, 60), np.linspace(0.05, 1.0, 40)])
    got = np.array([oracle.erfcinv(y) for y in ys])
    ref = sp.erfcinv(ys)
    assert np.all(np.abs(got - ref) <= 1e-13 * np.abs(ref) + 1e-15)


@pytest.mark.parametrize("p", [0.05, 0.1, 0.3, 0.6])
def test_event_radius_is_restricted_gaussian_quantile(p):
    R = 37.0
    words, u = _word(np.concatenate([np.linspace(0.0, 1.0, 400), [1e-7, 1 - 1e-7]]))
    got = np.array([oracle.event_radius(R, p, int(x)) for x in words])
    ref = st.truncnorm.ppf(u, a=-1.0 / p, b=np.inf, loc=R, scale=p * R)
    assert np.all(got > 0.0)
    assert np.all(np.abs(got - ref) <= 1e-10 * R), np.max(np.abs(got - ref))


def test_event_radius_monodisperse_and_median():
    assert oracle.event_radius(20.0, 0.0, 12345) == 20.0
    w, u = _word(0.5)
    assert abs(u - 0.5) < 1e-7
    # with the restriction negligible (p small) the median is the mean
    assert oracle.event_radius(20.0, 0.05, int(w)) == pytest.approx(20.0, abs=2e-6)


@pytest.mark.parametrize("p", [0.1, 0.3])
def test_gaussian_nodes_moments(p):
    R = 50.0
    r, w = oracle.gaussian_nodes(R, p, 48)
    assert w.sum() == pytest.approx(1.0, abs=1e-14) and np.all(r >= 0)
    dist = st.truncnorm(a=-1.0 / p, b=np.inf, loc=R, scale=p * R)
    for k in range(1, 7):
        assert np.dot(w, r ** k) == pytest.approx(dist.moment(k), rel=1e-9), k


def test_uniform_angle_nodes_closed_forms():
    c, w = oracle.uniform_angle_nodes(40, 40)
    assert w.sum() == pytest.approx(1.0, abs=1e-14)
    assert np.allclose(np.linalg.norm(c, axis=1), 1.0)
    # theta uniform on [0, pi]: <cos^2 theta> = 1/2 (1/3 on the sphere); phi uniform
    assert np.dot(w, c[:, 2] ** 2) == pytest.approx(0.5, abs=1e-12)
    assert np.dot(w, c[:, 0] ** 2) == pytest.approx(0.25, abs=1e-12)
    assert np.dot(w, c[:, 1] ** 2) == pytest.approx(0.25, abs=1e-12)
    assert abs(np.dot(w, c[:, 2])) < 1e-12
    # <|cos theta|> = 2/pi for theta uniform on [0, pi]
    assert np.dot(w, np.abs(c[:, 2])) == pytest.approx(2.0 / math.pi, abs=2e-3)


def test_event_axis_definitions():
    wa, ua = _word(np.linspace(0.01, 0.99, 13))
    wb, ub = _word(np.linspace(0.97, 0.02, 13))
    for xa, xb, a, b in zip(wa, wb, ua, ub):
        c2 = oracle.event_axis(2, 0.0, 0.0, int(xa), int(xb))
        assert math.acos(max(-1.0, min(1.0, c2[2]))) == pytest.approx(math.pi * a, abs=1e-9)
        assert math.atan2(c2[1], c2[0]) % (2 * math.pi) == pytest.approx(2 * math.pi * b, abs=1e-9)
        c1 = oracle.event_axis(1, 0.0, 0.0, int(xa), int(xb))
        assert c1[2] == pytest.approx(1.0 - 2.0 * a, abs=1e-15)
        assert np.linalg.norm(c1) == pytest.approx(1.0, abs=1e-14)
    c0 = oracle.event_axis(0, 0.7, 1.1, 0, 0)
    assert np.allclose(c0, [math.sin(0.7) * math.cos(1.1), math.sin(0.7) * math.sin(1.1), math.cos(0.7)])


def _pair(kind, iso=W.UNIFORM_ANGLES, **kw):
    base = dict(kind=kind, radius=30.0, sld=2e-6, sld_solvent=0.0, volume_fraction=0.01, poly=0.2,
                poly_dist=W.GAUSSIAN, n_poly=48, isotropic=iso, n_gamma=48, n_psi=48)
    if kind == W.CORE_SHELL:
        base.update(thickness=8.0, sld=1e-6, sld_shell=3e-6, sld_solvent=6e-6)
    if kind == W.CYLINDER:
        base.update(radius=15.0, length=200.0)
    if kind == W.ELLIPSOID:
        base.update(radius=25.0, radius_polar=60.0)
    base.update(kw)
    quad = W.Model(**base, sampling=W.QUADRATURE)
    event = W.Model(**base, sampling=W.PER_EVENT)
    return quad, event


@pytest.mark.parametrize("kind,iso", [(W.SPHERE, 0), (W.CORE_SHELL, 0), (W.CYLINDER, W.UNIFORM_ANGLES),
                                      (W.CYLINDER, W.ISOTROPIC), (W.ELLIPSOID, W.UNIFORM_ANGLES)])
def test_per_event_expectation_equals_quadrature(kind, iso):
    """E over the per-event draws = the quadrature over the same laws."""
    quad, event = _pair(kind, iso)
    n = 120000
    for qv in ([0.012, 0.004, 0.0], [0.0, 0.03, 0.002], [0.05, -0.02, 0.01]):
        q = np.tile(np.array(qv, dtype=np.float64), (n, 1))
        d = oracle.dsigma_event(event, q, seed=7, first=1000)
        ref = oracle.dsigma(oracle.Prepared(quad), q[:1])[0]
        z = (d.mean() - ref) / (d.std() / math.sqrt(n))
        assert abs(z) < 4.0, (kind, iso, qv, d.mean(), ref, z)
        assert d.std() > 0.0


def test_per_event_without_spread_is_the_quadrature():
    """No polydispersity and a fixed axis: every draw is the same node."""
    quad, event = _pair(W.CYLINDER, iso=W.CAP, poly=0.0, sigma_orient=0.0, axis_theta=1.1, axis_phi=0.3)
    q = np.random.default_rng(2).normal(size=(50, 3)) * 0.02
    d = oracle.dsigma_event(event, q, seed=1)
    ref = oracle.dsigma(oracle.Prepared(quad), q)
    assert np.allclose(d, ref, rtol=1e-13, atol=0)


def test_per_event_trace_matches_quadrature_trace():
    """Same histories, two estimators: identical pixels, and per-pixel sums
    of the per-history differences consistent with zero."""
    inst = W.Instrument(nx=12, ny=12, pixel_x=0.02, pixel_y=0.02, det_distance=3.0)
    quad, event = _pair(W.CYLINDER, W.UNIFORM_ANGLES, n_poly=24, n_gamma=24, n_psi=24)
    n = 60000
    pq, wq = oracle.records(inst, quad, n, seed=5)
    pe, we = oracle.records(inst, event, n, seed=5)
    assert np.array_equal(pq, pe)
    ok = pq >= 0
    npix = inst.nx * inst.ny
    d = we[ok] - wq[ok]
    s1 = np.bincount(pq[ok], weights=d, minlength=npix)
    s2 = np.bincount(pq[ok], weights=d * d, minlength=npix)
    m = s2 > 0
    z = s1[m] / np.sqrt(s2[m])
    assert np.max(np.abs(z)) < 4.5
    assert np.mean(z * z) < 1.6
    tq = oracle.trace(inst, quad, n, seed=5)
    te = oracle.trace(inst, event, n, seed=5)
    assert np.array_equal(tq["count"], te["count"])
    assert te["trans"] == pytest.approx(tq["trans"], rel=1e-13)
