"""Pins of the oracle's shape-independent models (the isotropic group G):
dSigma/dOmega = f_scale f(|Q|).

* the Gaussian coil against a brute-force Gaussian chain: the mean of
  exp(-Q^2 b^2 |i - j| / 6) over all pairs of N segments, Rg^2 = N b^2 / 6,
  converges to Debye's function as 1/N;
* the coil's series and closed form meet at their switch; the coil and the
  Guinier law share the small-Q slope -Rg^2/3;
* the Debye-Anderson-Brumberger form is the Lorentzian squared; the
  Lorentzian halves at Q = 1/xi; Teubner-Strey with c2 = 0 is a
  Lorentzian; the power law scales as 2^-m per octave; the Gaussian peak
  has its maximum at Q0 and its half width at half maximum sigma sqrt(2 ln 2);
* every form depends on |Q| only.
"""
import math

import numpy as np
import pytest

import oracle
import sas_workloads as W


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def _m(function, **kw):
    return W.Model(kind=W.SHAPE_INDEPENDENT, function=function, f_scale=kw.pop("f_scale", 2.5), **kw)


def _p(m, qs):
    qs = np.atleast_1d(np.asarray(qs, dtype=np.float64))
    return oracle.dsigma(oracle.Prepared(m), np.stack([qs, np.zeros_like(qs), np.zeros_like(qs)], axis=1))


def test_coil_against_a_discrete_gaussian_chain():
    rg = 40.0
    m = _m(W.GAUSS_COIL, f_p0=rg, f_scale=1.0)
    n = 200000
    b2 = 6.0 * rg * rg / n
    k = np.arange(1, n, dtype=np.float64)
    for q in (0.005, 0.02, 0.05, 0.1):
        x = math.exp(-q * q * b2 / 6.0)
        pair = (n + 2.0 * np.sum((n - k) * x ** k)) / (n * n)
        assert _p(m, q)[0] == pytest.approx(pair, rel=2e-5), q


def test_coil_series_meets_closed_form_and_guinier_slope():
    rg = 30.0
    coil, gui = _m(W.GAUSS_COIL, f_p0=rg), _m(W.GUINIER, f_p0=rg)
    us = math.sqrt(1e-3) / rg
    lo, hi = _p(coil, [us * (1 - 1e-9), us * (1 + 1e-9)])
    assert lo == pytest.approx(hi, rel=1e-10)
    for q in (1e-4, 5e-4, 1e-3):
        u = (q * rg) ** 2
        c, g = _p(coil, q)[0] / 2.5, _p(gui, q)[0] / 2.5
        assert abs(c - (1 - u / 3)) < 0.1 * u * u and abs(g - (1 - u / 3)) < 0.1 * u * u
        assert abs(c - g) <= (1 / 12 - 1 / 18) * u * u * 1.01 + 1e-15


def test_lorentzian_family():
    xi = 25.0
    lor, dab = _m(W.LORENTZ, f_p0=xi), _m(W.DAB, f_p0=xi)
    qs = np.linspace(0.0, 0.4, 41)
    assert np.allclose(_p(dab, qs) * 2.5, _p(lor, qs) ** 2, rtol=1e-14)
    assert _p(lor, 1.0 / xi)[0] == pytest.approx(1.25, rel=1e-14)
    ts = _m(W.TEUBNER_STREY, f_p0=0.5, f_p1=0.5 * xi * xi, f_p2=0.0, f_scale=1.0)
    assert np.allclose(_p(ts, qs), 2.0 * _p(lor, qs) / 2.5, rtol=1e-14)


def test_power_law_and_gaussian_peak():
    pw = _m(W.POWER_LAW, f_p0=3.7)
    for q in (0.01, 0.1):
        assert _p(pw, 2 * q)[0] / _p(pw, q)[0] == pytest.approx(2 ** -3.7, rel=1e-13)
    q0, sig = 0.08, 0.01
    pk = _m(W.GAUSS_PEAK, f_p0=q0, f_p1=sig)
    assert _p(pk, q0)[0] == pytest.approx(2.5, rel=1e-15)
    hw = sig * math.sqrt(2 * math.log(2))
    assert np.allclose(_p(pk, [q0 - hw, q0 + hw]), 1.25, rtol=1e-12)


@pytest.mark.parametrize("function,params", [(W.GUINIER, (30.0,)), (W.GAUSS_COIL, (30.0,)), (W.DAB, (20.0,)),
                                             (W.TEUBNER_STREY, (1.0, -200.0, 2e4))])
def test_isotropy(function, params):
    m = _m(function, **{f"f_p{i}": v for i, v in enumerate(params)})
    d = np.random.default_rng(4).normal(size=(30, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    prep = oracle.Prepared(m)
    for q in (0.01, 0.07):
        v = oracle.dsigma(prep, q * d)
        assert np.max(np.abs(v / v[0] - 1)) < 1e-13
