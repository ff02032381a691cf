"""Pins of the oracle's scattering attenuation (single scattering).

The particles deplete the beam inside the sample at the rate of their total
scattering cross section per unit volume,

    Sigma_s(lambda) = integral over all directions of dSigma/dOmega(Q) dOmega,
    Q = k (k_f - z),  k = 2 pi / lambda,

and the trace then attenuates with mu + Sigma_s(lambda). The oracle takes the
integral by a fixed product rule in (|Q|, phi). These tests pin it to facts
that do not come from that rule:

* large k, sphere: Sigma_s -> (3/2) lambda^2 R phi drho^2. Since
  integral_0^inf Q V P(Q) dQ = 4 pi integral gamma_0(r) dr with the sphere's
  characteristic function gamma_0(r) = 1 - 3r/(4R) + r^3/(16 R^3), whose
  integral is 3R/4; the finite upper limit 2k removes the Porod tail,
  a relative 1/(2kR)^2;
* small k (Guinier over the Ewald sphere): <Q_i Q_j> over all directions
  is k^2 (delta_ij / 3 + z_i z_j), so with P = 1 - sum_e (Q.e)^2 s_e^2 the
  cross section is 4 pi I(0) [1 - k^2 sum_e (1/3 + e_z^2) s_e^2] to second
  order; this pins the direction of the Ewald sphere (the z term) for a
  cylinder along and across the beam and for a rotated parallelepiped;
* large k, oriented particles: the Ewald sphere flattens to the plane
  normal to the beam and, by the projection-slice theorem, Sigma_s ->
  lambda^2 phi drho^2 (1/V) integral t(x, y)^2 dx dy with t the thickness
  along the beam: 16 R / (3 pi) for a cylinder across the beam, 2c for a
  parallelepiped with its edge 2c along it;
* conservation (the check that multiple scattering is off): with the
  sample's own scattering as the only attenuation and no attenuation after
  the scattering point, transmitted + once-scattered weight over all
  directions is exactly 1; that is Sigma_s = the integral of dSigma/dOmega
  over the sphere, checked here against an importance-sampled Monte Carlo
  integral of the same cross section (independent of the rule);
* the Chebyshev table of the trace against direct evaluations.
"""
import math

import numpy as np
import pytest

import oracle
import sas_workloads as W


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


@pytest.mark.parametrize("lam,R", [(6.0, 50.0), (2.0, 50.0), (6.0, 30.0)])
def test_sphere_large_k_closed_form(lam, R):
    phi, drho = 0.01, 2e-6
    m = W.Model(kind=W.SPHERE, radius=R, sld=drho, volume_fraction=phi)
    k = 2 * math.pi / lam
    ref = 1.5 * lam ** 2 * R * phi * drho ** 2 * (1.0 - 1.0 / (2 * k * R) ** 2)
    assert oracle.sigma_s(m, lam) == pytest.approx(ref, rel=2e-5)


def _guinier(i0, k, axes):
    """4 pi I(0) [1 - k^2 sum_e (1/3 + e_z^2) s_e^2] for P = 1 - sum_e (Q.e)^2 s_e^2."""
    return 4 * math.pi * i0 * (1.0 - k * k * sum((1.0 / 3.0 + e[2] ** 2) * s2 for e, s2 in axes))


def test_sphere_small_k_series():
    R, phi, drho = 10.0, 0.01, 2e-6
    m = W.Model(kind=W.SPHERE, radius=R, sld=drho, volume_fraction=phi)
    V = 4 / 3 * math.pi * R ** 3
    i0 = phi * drho ** 2 * V
    for lam in (400.0, 800.0):
        k = 2 * math.pi / lam
        # P = 1 - x^2/5 + 3 x^4/175; <Q^2> = 2 k^2, <Q^4> = 16 k^4 / 3
        ref = 4 * math.pi * i0 * (1 - 2 * (k * R) ** 2 / 5 + 16 * (k * R) ** 4 / 175)
        assert oracle.sigma_s(m, lam) == pytest.approx(ref, rel=1e-6)


@pytest.mark.parametrize("theta,phi_ax", [(0.0, 0.0), (0.5 * math.pi, 0.0), (1.0, 0.7)])
def test_cylinder_small_k_ewald_direction(theta, phi_ax):
    R, L, phi, drho = 10.0, 40.0, 0.01, 2e-6
    m = W.Model(kind=W.CYLINDER, radius=R, length=L, sld=drho, volume_fraction=phi,
                axis_theta=theta, axis_phi=phi_ax)
    n = np.array([math.sin(theta) * math.cos(phi_ax), math.sin(theta) * math.sin(phi_ax), math.cos(theta)])
    i0 = phi * drho ** 2 * math.pi * R * R * L
    lam = 4000.0
    k = 2 * math.pi / lam
    # P = 1 - (Q.n)^2 L^2/12 - |Q x n|^2 R^2/4; |Q x n|^2 = sum over two axes normal to n
    e1 = np.cross(n, [1.0, 0.0, 0.0] if abs(n[0]) < 0.9 else [0.0, 1.0, 0.0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(n, e1)
    ref = _guinier(i0, k, [(n, L * L / 12), (e1, R * R / 4), (e2, R * R / 4)])
    assert oracle.sigma_s(m, lam) == pytest.approx(ref, rel=1e-6)


def test_parallelepiped_small_k_rotated_frame():
    a, b, c, phi, drho = 6.0, 10.0, 16.0, 0.01, 2e-6
    th, ph, ps = 0.9, 0.4, 1.2
    m = W.Model(kind=W.PARALLELEPIPED, radius=a, radius_b=b, radius_polar=c, sld=drho, volume_fraction=phi,
                axis_theta=th, axis_phi=ph, axis_psi=ps)
    f = oracle.frame(th, ph, ps)
    i0 = phi * drho ** 2 * 8 * a * b * c
    lam = 4000.0
    k = 2 * math.pi / lam
    # sinc(Q.e s)^2 = 1 - (Q.e)^2 s^2 / 3
    ref = _guinier(i0, k, [(f[0], a * a / 3), (f[1], b * b / 3), (f[2], c * c / 3)])
    assert oracle.sigma_s(m, lam) == pytest.approx(ref, rel=1e-6)


def test_flat_ewald_limit_projection_slice():
    phi, drho = 0.01, 2e-6
    R, L = 20.0, 400.0
    cyl = W.Model(kind=W.CYLINDER, radius=R, length=L, sld=drho, volume_fraction=phi,
                  axis_theta=0.5 * math.pi, axis_phi=0.3)
    lam = 0.5
    assert oracle.sigma_s(cyl, lam) == pytest.approx(lam ** 2 * phi * drho ** 2 * 16 * R / (3 * math.pi), rel=3e-3)
    # the parallelepiped's sinc streaks reach far out, where the Ewald sphere
    # leaves the plane: the limit is approached like sqrt(lambda)
    ppd = W.Model(kind=W.PARALLELEPIPED, radius=30.0, radius_b=40.0, radius_polar=5.0, sld=drho,
                  volume_fraction=phi, axis_theta=0.0, axis_phi=0.0)
    lam = 0.25
    assert oracle.sigma_s(ppd, lam) == pytest.approx(lam ** 2 * phi * drho ** 2 * 2 * 5.0, rel=1e-2)


def _mc_sigma(model, lam, q0, n, seed):
    """Importance-sampled integral of dSigma/dOmega over all directions:
    |Q| from p(Q) = 2 q0^2 Q / (Q^2 + q0^2)^2 restricted to [0, 2k] (by
    inversion), phi uniform, weight (Q / k^2) f 2 pi / p."""
    rng = np.random.default_rng(seed)
    k = 2 * math.pi / lam
    umax = (2 * k) ** 2 / ((2 * k) ** 2 + q0 * q0)
    u = rng.uniform(0.0, umax, size=n)
    Q = q0 * np.sqrt(u / (1.0 - u))
    ph = rng.uniform(0.0, 2 * math.pi, size=n)
    st = np.sqrt(np.maximum(1 - Q * Q / (4 * k * k), 0.0))
    qv = np.stack([Q * st * np.cos(ph), Q * st * np.sin(ph), -Q * Q / (2 * k)], axis=1)
    f = oracle.dsigma(oracle.Prepared(model), qv)
    p = 2 * q0 * q0 * Q / (Q * Q + q0 * q0) ** 2 / umax
    g = Q / (k * k) * f * 2 * math.pi / p
    return g.mean(), g.std() / math.sqrt(n)


@pytest.mark.parametrize("name", ["core_shell_py", "cylinder_spread", "triaxial"])
def test_conservation_against_monte_carlo(name):
    if name == "core_shell_py":
        m = W.core_shell_config()["model"]
        q0 = 1.0 / 50.0
    elif name == "cylinder_spread":
        m = W.Model(kind=W.CYLINDER, radius=20.0, length=200.0, sld=2e-6, volume_fraction=0.01, poly=0.1,
                    n_poly=6, sigma_orient=math.radians(15.0), axis_theta=0.5 * math.pi, n_gamma=6, n_psi=8)
        q0 = 1.0 / 40.0
    else:
        m = W.Model(kind=W.TRIAXIAL_ELLIPSOID, radius=15.0, radius_b=25.0, radius_polar=40.0, sld=2e-6,
                    volume_fraction=0.01, axis_theta=0.8, axis_phi=0.2, axis_psi=0.5)
        q0 = 1.0 / 25.0
    lam = 6.0
    est, err = _mc_sigma(m, lam, q0, 200000, seed=3)
    s = oracle.sigma_s(m, lam)
    assert abs(est - s) < 5 * err, (est, s, err)
    assert err < 0.01 * s


def test_chebyshev_table_against_direct():
    inst = W.instrument()
    m = W.core_shell_config()["model"]
    lam, mu, c = oracle.att_table(inst, m)
    lmin, lmax = inst.lambda0 * (1 - inst.dlambda_rel), inst.lambda0 * (1 + inst.dlambda_rel)
    assert len(lam) == 8 and lam.min() > lmin and lam.max() < lmax
    assert np.allclose(mu, [1e10 * oracle.sigma_s(m, x, lmin) for x in lam], rtol=1e-13)
    xs = np.linspace(lmin, lmax, 41)
    got = oracle.att_eval(inst, m, xs)
    ref = np.array([1e10 * oracle.sigma_s(m, x, lmin) for x in xs])
    assert np.all(np.abs(got / ref - 1) < 1e-5)
    # at the nodes the interpolant is exact
    assert np.allclose(oracle.att_eval(inst, m, lam), mu, rtol=1e-12)
    # no spread: one node at lambda0
    mono = W.Instrument(dlambda_rel=0.0)
    lam1, mu1, _ = oracle.att_table(mono, m)
    assert len(lam1) == 1 and lam1[0] == mono.lambda0
    assert mu1[0] == pytest.approx(1e10 * oracle.sigma_s(m, mono.lambda0), rel=1e-14)


def test_trace_uses_the_attenuation():
    """Transmitted weight: exp(-(mu + mu_s(lambda)) l) per history; with the
    table on, each history's weight is the plain one times
    exp(-mu_s(lambda) (s + l_out)) <= 1, and the transmitted sum drops."""
    inst = W.instrument(nx=16, ny=16, pixel_x=0.02, pixel_y=0.02)
    m = W.core_shell_config()["model"]
    on = W.Model(**{**m.as_dict(), "self_attenuation": 1})
    n = 20000
    p0, w0 = oracle.records(inst, m, n, seed=2)
    p1, w1 = oracle.records(inst, on, n, seed=2)
    assert np.array_equal(p0, p1)
    ok = p0 >= 0
    r = w1[ok] / w0[ok]
    mu_max = oracle.att_table(inst, m)[1].max()
    # paths inside a 1 mm slab: at most a few mm for these small angles
    assert np.all(r <= 1.0) and np.all(r >= math.exp(-mu_max * 0.01))
    t0 = oracle.trace(inst, m, n, seed=2)["trans"]
    t1 = oracle.trace(inst, on, n, seed=2)["trans"]
    mu0 = oracle.att_eval(inst, m, [inst.lambda0])[0]
    assert t0 == pytest.approx(n, rel=1e-12)
    assert t1 / n == pytest.approx(math.exp(-mu0 * inst.sample_thickness), rel=2e-3)


def test_panels_sum_to_the_total():
    m = W.Model(kind=W.CYLINDER, radius=20.0, length=300.0, sld=2e-6, volume_fraction=0.01, poly=0.1, n_poly=4,
                sigma_orient=0.2, n_gamma=4, n_psi=4)
    n = oracle.sigma_s_npanels(m, 5.4)
    parts = [oracle.sigma_s_panel(m, 6.0, 5.4, i) for i in range(n)]
    assert math.isnan(oracle.sigma_s_panel(m, 6.0, 5.4, n))
    assert sum(parts) == pytest.approx(oracle.sigma_s(m, 6.0, 5.4), rel=1e-13)
    assert all(p > 0 for p in parts)
