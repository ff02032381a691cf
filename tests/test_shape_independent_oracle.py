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
* every form depends on |Q| only;
* the fractal factor of the mass fractal and of Teixeira's aggregate is
  the normalised three-dimensional transform of r^(D - 3) exp(-r / xi),
  integrated numerically (scipy's QAWF Fourier quadrature), times the
  sphere factor (scipy's spherical Bessel j1); Teixeira's S(0) =
  1 + Gamma(D + 1) (xi / R0)^D;
* the spinodal peak has its maximum 1 at Qmax and slopes 2 and -g in
  log-log below and above it;
* the chain with excluded volume is Hammouda's integral
  2 int_0^1 (1 - x) exp(-U x^(2 nu)) dx (scipy's adaptive quadrature), is
  Debye's function at nu = 1/2, has the Guinier slope -Rg^2/3 and the
  log-log slope -1/nu at large Q;
* linear pearls: the isotropic average of |sum_j exp(i Q.r_j)|^2 of the
  chain by Gauss-Legendre quadrature over the angle to the chain's axis,
  times the sphere factor; one pearl is the sphere.
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
                                             (W.TEUBNER_STREY, (1.0, -200.0, 2e4)),
                                             (W.MASS_FRACTAL, (12.0, 2.3, 150.0)),
                                             (W.FRACTAL, (5.0, 2.1, 120.0)), (W.SPINODAL, (0.03, 3.0))])
def test_isotropy(function, params):
    m = _m(function, **{f"f_p{i}": v for i, v in enumerate(params)})
    d = np.random.default_rng(4).normal(size=(30, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    prep = oracle.Prepared(m)
    for q in (0.01, 0.07):
        v = oracle.dsigma(prep, q * d)
        assert np.max(np.abs(v / v[0] - 1)) < 1e-13


# ---- the further laws of group G: peak Lorentz, two power laws, Guinier-Porod,
# Gauss-Lorentz gel, polydisperse Gaussian coil, star polymer

def test_peak_lorentz_maximum_and_half_width():
    q0, b = 0.05, 0.01
    m = _m(W.PEAK_LORENTZ, f_p0=q0, f_p1=b, f_scale=1.0)
    assert _p(m, q0)[0] == pytest.approx(1.0, rel=1e-15)
    lo, hi = _p(m, [q0 - b, q0 + b])
    assert lo == pytest.approx(0.5, rel=1e-12) and hi == pytest.approx(0.5, rel=1e-12)
    qs = np.linspace(0.001, 0.099, 37)
    assert np.allclose(_p(m, qs), _p(m, 2 * q0 - qs), rtol=1e-12)    # symmetric about q0


def _loglog_slope(m, q, h=1e-6):
    a, b = _p(m, [q * (1 - h), q * (1 + h)])
    return (math.log(b) - math.log(a)) / (math.log(1 + h) - math.log(1 - h))


def test_two_power_law_continuity_and_slopes():
    qc, m1, m2 = 0.03, 1.7, 3.9
    m = _m(W.TWO_POWER_LAW, f_p0=qc, f_p1=m1, f_p2=m2, f_scale=1.0)
    lo, hi = _p(m, [qc * (1 - 1e-12), qc * (1 + 1e-12)])
    assert lo == pytest.approx(hi, rel=1e-9)
    assert _p(m, qc)[0] == pytest.approx(qc ** -m1, rel=1e-13)
    assert _loglog_slope(m, 0.01) == pytest.approx(-m1, rel=1e-6)
    assert _loglog_slope(m, 0.1) == pytest.approx(-m2, rel=1e-6)


@pytest.mark.parametrize("s", [0.0, 1.0, 2.0])
def test_guinier_porod_is_smooth_at_its_join(s):
    rg, mp = 40.0, 4.0
    m = _m(W.GUINIER_POROD, f_p0=rg, f_p1=s, f_p2=mp, f_scale=1.0)
    q1 = math.sqrt((mp - s) * (3 - s) / 2) / rg
    lo, hi = _p(m, [q1 * (1 - 1e-12), q1 * (1 + 1e-12)])
    assert lo == pytest.approx(hi, rel=1e-9)                     # the value joins
    # and the slope: -s - 2 q^2 Rg^2 / (3 - s) reaches -m at q1
    assert _loglog_slope(m, q1 * (1 - 1e-4)) == pytest.approx(-mp, rel=2e-3)
    assert _loglog_slope(m, q1 * 1.5) == pytest.approx(-mp, rel=1e-6)
    if s == 0.0:                                                 # Guinier at small q
        q = 1e-3
        assert _p(m, q)[0] == pytest.approx(math.exp(-(q * rg) ** 2 / 3), rel=1e-14)


def test_gauss_lorentz_gel_limits():
    xi_g, xi_l, r = 80.0, 25.0, 0.3
    m = _m(W.GAUSS_LORENTZ_GEL, f_p0=xi_g, f_p1=xi_l, f_p2=r, f_scale=1.0)
    assert _p(m, 0.0)[0] == pytest.approx(1.0 + r, rel=1e-15)
    q = 0.04
    assert _p(m, q)[0] == pytest.approx(math.exp(-0.5 * (q * xi_g) ** 2) + r / (1 + (q * xi_l) ** 2), rel=1e-14)
    g0 = _m(W.GAUSS_LORENTZ_GEL, f_p0=xi_g, f_p1=xi_l, f_p2=0.0, f_scale=1.0)
    lz = _m(W.LORENTZ, f_p0=xi_l, f_scale=r)
    qs = np.array([0.01, 0.03, 0.08])
    assert np.allclose(_p(m, qs), _p(g0, qs) + _p(lz, qs), rtol=1e-13)


def test_poly_coil_against_a_schulz_zimm_average_of_chains():
    """The closed form against its definition: Debye's function of chains
    whose length N is Schulz-Zimm distributed (number density ~ N^z
    e^-(z+1) N / N_n, Mw/Mn = 1 + U, U = 1/(z+1)), each weighted by N^2,
    integrated numerically; Rg is the z-average radius of gyration, so the
    number-average chain has Rg_n^2 = Rg^2 / (1 + 2U)."""
    from scipy import integrate, special
    rg = 50.0
    for U in (0.1, 0.5, 1.0):
        z = 1.0 / U - 1.0
        m = _m(W.POLY_GAUSS_COIL, f_p0=rg, f_p1=U, f_scale=1.0)
        rgn2 = rg * rg / (1 + 2 * U)
        for q in (0.002, 0.01, 0.03, 0.1):
            def debye(u):
                return 2 * (math.expm1(-u) + u) / (u * u) if u > 1e-6 else 1 - u / 3

            def w(n):   # N in units of N_n
                return n ** (z + 2) * math.exp(-(z + 1) * n)
            num = integrate.quad(lambda n: w(n) * debye(q * q * rgn2 * n), 0, np.inf, limit=400)[0]
            den = math.exp(special.gammaln(z + 3) - (z + 3) * math.log(z + 1))
            assert _p(m, q)[0] == pytest.approx(num / den, rel=1e-8), (U, q)
    mono = _m(W.GAUSS_COIL, f_p0=rg, f_scale=1.0)
    zero = _m(W.POLY_GAUSS_COIL, f_p0=rg, f_p1=0.0, f_scale=1.0)
    qs = np.array([1e-4, 1e-2, 0.05, 0.2])
    assert np.allclose(_p(zero, qs), _p(mono, qs), rtol=1e-12)


def test_poly_coil_moment_series_at_small_q():
    """Debye's function as its power series sum_k 2 (-u)^k / (k + 2)!,
    averaged term by term over the same N^2-weighted Schulz-Zimm chains:
    <N^k> / N_n^k = prod_{j<k} (1 + (2 + j) U). At u = Q^2 Rg_n^2 <= 0.03 forty
    terms give the average to rounding, so the closed form and its series
    branch must both agree to 1e-12 across their switch (cancellation or a
    truncated series near it shows up here first)."""
    rg = 50.0
    for U in (0.1, 0.5, 1.0, 4.0):
        m = _m(W.POLY_GAUSS_COIL, f_p0=rg, f_p1=U, f_scale=1.0)
        rgn2 = rg * rg / (1 + 2 * U)
        xs = np.logspace(-7, math.log10(0.03), 57)
        qs = np.sqrt(xs / rgn2)
        got = _p(m, qs)
        for x, g in zip(xs, got):
            s, mom, fact = 0.0, 1.0, 2.0
            for k in range(40):
                s += 2.0 * (-x) ** k * mom / fact
                mom *= 1.0 + (2 + k) * U
                fact *= k + 3
            assert g == pytest.approx(s, rel=1e-12, abs=0.0), (U, x)


def test_star_polymer_against_a_discrete_gaussian_star():
    """f arms of n Gaussian segments from one centre: the mean over all pairs
    of exp(-Q^2 b^2 d / 6), d the number of segments between them along the
    star (|i - j| on one arm, i + j across arms), with Rg^2 of the star
    = (3f - 2) / f x n b^2 / 6; the closed form is the continuous limit
    (corrections of order 1/n). Two arms make one chain: the Gaussian coil."""
    rg = 40.0
    n = 4000
    i = np.arange(1, n + 1, dtype=np.float64)
    for fa in (3, 6):
        b2 = 6.0 * rg * rg * fa / ((3 * fa - 2) * n)
        m = _m(W.STAR_POLYMER, f_p0=rg, f_p1=float(fa), f_scale=1.0)
        for q in (0.005, 0.02, 0.06):
            x = math.exp(-q * q * b2 / 6.0)
            k = np.arange(1, n, dtype=np.float64)
            same = n + 2.0 * np.sum((n - k) * x ** k)            # pairs on one arm
            s1 = np.sum(x ** i)
            cross = s1 * s1                                     # pairs on two different arms
            pair = (fa * same + fa * (fa - 1) * cross) / (fa * n) ** 2
            assert _p(m, q)[0] == pytest.approx(pair, rel=2e-3), (fa, q)
    two = _m(W.STAR_POLYMER, f_p0=rg, f_p1=2.0, f_scale=1.0)
    one = _m(W.STAR_POLYMER, f_p0=rg, f_p1=1.0, f_scale=1.0)
    coil = _m(W.GAUSS_COIL, f_p0=rg, f_scale=1.0)
    qs = np.array([1e-3, 0.01, 0.05, 0.2])
    assert np.allclose(_p(two, qs), _p(coil, qs), rtol=1e-12)
    assert np.allclose(_p(one, qs), _p(coil, qs), rtol=1e-12)


# ---- fractals (mass fractal, Teixeira's aggregate) and the spinodal peak

def _fractal_transform(q, d, xi):
    """(1 / Gamma(D) xi^D) int_0^inf r^(D-1) exp(-r / xi) sin(q r) / (q r) dr,
    the normalised 3D transform of r^(D-3) exp(-r / xi), by QAWF."""
    from scipy import integrate
    # [0, xi] by plain adaptive quadrature (the integrand ~ q r^(D-1) at 0),
    # the tail by the Fourier quadrature
    head, _ = integrate.quad(lambda r: r ** (d - 2.0) * math.exp(-r / xi) * math.sin(q * r), 0.0, xi, limit=400,
                             epsabs=0.0, epsrel=1e-10)
    tail, _ = integrate.quad(lambda r: r ** (d - 2.0) * math.exp(-r / xi), xi, np.inf, weight="sin", wvar=q,
                             limlst=200)
    return (head + tail) / (q * math.gamma(d) * xi ** d)


def _sphere_p(x):
    from scipy.special import spherical_jn
    return (3.0 * spherical_jn(1, x) / x) ** 2


@pytest.mark.parametrize("d", [1.5, 2.0, 2.6, 3.0])
def test_mass_fractal_is_the_transform_of_its_correlation(d):
    xi = 37.0
    pure = _m(W.MASS_FRACTAL, f_p0=0.0, f_p1=d, f_p2=xi, f_scale=1.0)
    qs = np.array([0.3, 2.0, 15.0, 90.0]) / xi
    got = _p(pure, qs)
    ref = np.array([_fractal_transform(q, d, xi) for q in qs])
    assert np.allclose(got, ref, rtol=1e-8, atol=0), (got, ref)
    assert abs(_p(pure, 1e-9)[0] - 1.0) < 1e-12
    r = 14.0                                                       # with building blocks of radius r
    blocks = _m(W.MASS_FRACTAL, f_p0=r, f_p1=d, f_p2=xi, f_scale=1.0)
    assert np.allclose(_p(blocks, qs), ref * _sphere_p(qs * r), rtol=1e-8, atol=0)


@pytest.mark.parametrize("d,xi,r0", [(1.8, 90.0, 6.0), (2.5, 200.0, 12.0)])
def test_fractal_aggregate_against_its_pair_correlation(d, xi, r0):
    """S(Q) = 1 + (D / R0^D) int r^(D-1) exp(-r / xi) sin(Q r) / (Q r) dr
    (Teixeira's pair correlation of the aggregate), times the sphere factor
    of the building blocks."""
    m = _m(W.FRACTAL, f_p0=r0, f_p1=d, f_p2=xi, f_scale=1.0)
    qs = np.array([0.001, 0.01, 0.05, 0.2])
    s_ref = 1.0 + d / r0 ** d * math.gamma(d) * xi ** d * np.array([_fractal_transform(q, d, xi) for q in qs])
    assert np.allclose(_p(m, qs), s_ref * _sphere_p(qs * r0), rtol=1e-8, atol=0)
    assert _p(m, 1e-9)[0] == pytest.approx(1.0 + math.gamma(d + 1.0) * (xi / r0) ** d, rel=1e-9)


@pytest.mark.parametrize("g", [2.0, 3.0, 4.0])
def test_spinodal_peak(g):
    qmax = 0.031
    m = _m(W.SPINODAL, f_p0=qmax, f_p1=g, f_scale=1.0)
    assert abs(_p(m, qmax)[0] - 1.0) < 1e-14
    grid = qmax * np.linspace(0.5, 1.5, 2001)
    v = _p(m, grid)
    assert abs(grid[np.argmax(v)] - qmax) <= qmax * 5e-4 and v.max() <= 1.0 + 1e-14
    lo = _p(m, [1e-6 * qmax, 2e-6 * qmax])
    assert lo[1] / lo[0] == pytest.approx(4.0, rel=1e-5)            # Q^2 below the peak
    hi = _p(m, [1e4 * qmax, 2e4 * qmax])
    assert math.log2(hi[0] / hi[1]) == pytest.approx(g, rel=1e-4)   # Q^-g above it


# ---- the chain with excluded volume (Hammouda)

def _pev(rg, m, qs):
    return _p(_m(W.POLYMER_EXCL_VOLUME, f_p0=rg, f_p1=m, f_scale=1.0), qs)


@pytest.mark.parametrize("m", [5.0 / 3.0, 2.5, 3.0, 4.5])
def test_excluded_volume_chain_is_hammoudas_integral(m):
    from scipy import integrate
    rg, nu = 40.0, 1.0 / m
    qs = np.array([1e-4, 0.01, 0.05, 0.2, 1.0])
    got = _pev(rg, m, qs)
    for q, g in zip(qs, got):
        u = q * q * rg * rg * (2 * nu + 1) * (2 * nu + 2) / 6.0
        # x = y^p, p = 1 / (2 nu): the exponent becomes -u y, the layer where it
        # falls has width 1/u in y
        p = 0.5 / nu
        pts = [c / u for c in (0.1, 1.0, 10.0, 100.0) if c / u < 1.0] or None
        ref, _ = integrate.quad(lambda y: 2.0 * (1.0 - y ** p) * math.exp(-u * y) * p * y ** (p - 1.0), 0.0, 1.0,
                                epsabs=0.0, epsrel=1e-13, limit=2000, points=pts)
        assert g == pytest.approx(ref, rel=1e-10), (m, q)


def test_excluded_volume_chain_limits():
    rg = 35.0
    qs = np.array([0.003, 0.02, 0.1, 0.4])
    u = (qs * rg) ** 2                                              # nu = 1/2: Debye's function of (Q Rg)^2
    assert np.allclose(_pev(rg, 2.0, qs), 2.0 * (np.exp(-u) - 1.0 + u) / u ** 2, rtol=1e-12, atol=0)
    for m in (5.0 / 3.0, 3.0):
        q = 1e-4                                                    # Guinier: 1 - Q^2 Rg^2 / 3
        assert (1.0 - _pev(rg, m, q)[0]) / (q * q * rg * rg / 3.0) == pytest.approx(1.0, rel=1e-4)
        hi = _pev(rg, m, [20.0, 40.0])                              # Q^-m far beyond 1/Rg, up to the
        assert math.log2(hi[0] / hi[1]) == pytest.approx(m, rel=1e-4)   # second term's U^(-m/2) ~ 1e-5


# ---- linear pearls

@pytest.mark.parametrize("n,r,sep", [(2, 20.0, 0.0), (7, 15.0, 12.0), (30, 8.0, 3.0)])
def test_linear_pearls_is_the_orientation_average_of_the_chain(n, r, sep):
    d = 2 * r + sep
    m = _m(W.LINEAR_PEARLS, f_p0=r, f_p1=sep, f_p2=float(n), f_scale=1.0)
    qs = np.array([1e-3, 0.01, 0.03, 0.1, 0.3])
    x, w = np.polynomial.legendre.leggauss(400)                 # cos of the angle between Q and the axis
    z = d * np.arange(n)
    ref = []
    for q in qs:
        amp = np.exp(1j * q * np.outer(x, z)).sum(axis=1)       # sum over the pearls at each angle
        ref.append(0.5 * np.dot(w, np.abs(amp) ** 2) / n ** 2 * _sphere_p(q * r))
    assert np.allclose(_p(m, qs), ref, rtol=1e-10, atol=0)
    assert abs(_p(m, 1e-9)[0] - 1.0) < 1e-12


def test_one_pearl_is_the_sphere():
    m = _m(W.LINEAR_PEARLS, f_p0=25.0, f_p1=5.0, f_p2=1.0, f_scale=1.0)
    qs = np.array([0.01, 0.1, 0.3])
    assert np.allclose(_p(m, qs), _sphere_p(qs * 25.0), rtol=1e-12, atol=0)
