"""Pins of the oracle's shelled uniaxial models: the core-shell cylinder
(core r x L, shell t around it and t_f on the end faces), the hollow
cylinder (a tube of wall material between r and r + t, solvent inside),
the core-shell ellipsoid of revolution (core radii r, r_p; shell t at the
equator and t_p at the poles) and the core-shell bicelle (core r x L, face
layers t_f of the core's radius, a rim t around both over L + 2 t_f).

* reductions to the plain models: no shell, a shell of the core's density,
  a hollow cylinder as a core-shell cylinder with a solvent core, the
  core-shell ellipsoid with r_p = r, t_p = t as the core-shell sphere, the
  bicelle with faces of the rim's density as the core-shell cylinder;
* fixed axes against Eq. 1 integrated over the body by brute force: for the
  cylinders, disjoint (rho, z) rectangles of each density with the azimuth
  in closed form (2 pi J0) and Gauss-Legendre in rho and z; for the
  ellipsoids, Gauss-Legendre over the mapped unit ball;
* the per-event mean equals the quadrature over the same laws.
"""
import math

import numpy as np
import pytest

import oracle
import sas_workloads as W

sp = pytest.importorskip("scipy.special")


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def _q(n, seed, scale=0.06):
    return np.random.default_rng(seed).normal(size=(n, 3)) * scale


def _rect(qz, qp, r0, r1, z0, z1, n=48):
    """Integral of exp(i Q.x) over the ring r0 <= rho <= r1, z0 <= z <= z1
    about the axis (the real part; the bodies here are symmetric in z)."""
    x, w = np.polynomial.legendre.leggauss(n)
    rho = 0.5 * (r0 + r1) + 0.5 * (r1 - r0) * x
    wr = 0.5 * (r1 - r0) * w
    z = 0.5 * (z0 + z1) + 0.5 * (z1 - z0) * x
    wz = 0.5 * (z1 - z0) * w
    return np.sum(wr * rho * 2.0 * math.pi * sp.j0(qp * rho)) * np.sum(wz * np.cos(qz * z))


def _cs_cylinder_F(qz, qp, r, t, L, tf, rho_c, rho_s, rho_v):
    h = 0.5 * L
    F = (rho_c - rho_v) * _rect(qz, qp, 0.0, r, -h, h)
    F += (rho_s - rho_v) * _rect(qz, qp, r, r + t, -h, h)                # side wall
    F += (rho_s - rho_v) * 2.0 * _rect(qz, qp, 0.0, r + t, h, h + tf)    # both end faces (cos is even)
    return F


def _ball_F(q_local, a, c, n=40):
    """Integral of exp(i Q.x) over the ellipsoid of revolution with radii
    (a, a, c) about z, by Gauss-Legendre over the mapped unit ball."""
    x, w = np.polynomial.legendre.leggauss(n)
    rr = 0.5 * (x + 1.0)
    wr = 0.5 * w * rr ** 2
    ph = math.pi * (x + 1.0)
    R, CT, PH = np.meshgrid(rr, x, ph, indexing="ij")
    ST = np.sqrt(1 - CT ** 2)
    W3 = np.einsum("i,j,k->ijk", wr, w, math.pi * w) * a * a * c
    arg = q_local[0] * a * R * ST * np.cos(PH) + q_local[1] * a * R * ST * np.sin(PH) + q_local[2] * c * R * CT
    return np.sum(W3 * np.cos(arg))


def _axis_parts(q, th, ph):
    c = oracle.axis_from_angles(th, ph)[0]
    qz = float(q @ c)
    return qz, float(np.linalg.norm(q - qz * c))


def _m(kind, **kw):
    base = dict(kind=kind, sld=1.0, sld_solvent=0.0, volume_fraction=1.0, axis_theta=1.1, axis_phi=0.6)
    base.update(kw)
    return W.Model(**base)


def test_core_shell_cylinder_reductions():
    q = _q(40, 1)
    # no shell: the plain cylinder of the core's contrast, polydisperse too
    a = _m(W.CORE_SHELL_CYLINDER, radius=20.0, length=120.0, sld=2.0, sld_shell=5.0, sld_solvent=0.5,
           poly=0.15, n_poly=12, sigma_orient=0.3, n_gamma=8, n_psi=8)
    b = _m(W.CYLINDER, radius=20.0, length=120.0, sld=2.0, sld_solvent=0.5, poly=0.15, n_poly=12,
           sigma_orient=0.3, n_gamma=8, n_psi=8)
    assert np.allclose(oracle.dsigma(oracle.Prepared(a), q), oracle.dsigma(oracle.Prepared(b), q), rtol=1e-12)
    # a shell of the core's density: one cylinder of the outer sizes
    a = _m(W.CORE_SHELL_CYLINDER, radius=20.0, thickness=5.0, thickness_face=8.0, length=120.0, sld=2.0,
           sld_shell=2.0, sld_solvent=0.5)
    b = _m(W.CYLINDER, radius=25.0, length=136.0, sld=2.0, sld_solvent=0.5)
    assert np.allclose(oracle.dsigma(oracle.Prepared(a), q), oracle.dsigma(oracle.Prepared(b), q), rtol=1e-12)


def test_hollow_cylinder_is_a_core_shell_cylinder_with_a_solvent_core():
    q = _q(40, 2)
    r, t, L = 15.0, 6.0, 90.0
    h = _m(W.HOLLOW_CYLINDER, radius=r, thickness=t, length=L, sld=3.0, sld_solvent=1.0)
    cs = _m(W.CORE_SHELL_CYLINDER, radius=r, thickness=t, length=L, sld=1.0, sld_shell=3.0, sld_solvent=1.0)
    # the hollow cylinder is normalised by its wall volume, the core-shell one by the outer volume
    ratio = ((r + t) ** 2) / ((r + t) ** 2 - r ** 2)
    assert np.allclose(oracle.dsigma(oracle.Prepared(h), q), ratio * oracle.dsigma(oracle.Prepared(cs), q),
                       rtol=1e-12)


def test_core_shell_ellipsoid_reductions():
    q = _q(40, 3)
    # r_p = r and t_p = t: the core-shell sphere (monodisperse: the ellipsoid keeps r_p fixed)
    a = _m(W.CORE_SHELL_ELLIPSOID, radius=30.0, radius_polar=30.0, thickness=8.0, thickness_face=8.0, sld=1.0,
           sld_shell=3.0, sld_solvent=2.0)
    b = _m(W.CORE_SHELL, radius=30.0, thickness=8.0, sld=1.0, sld_shell=3.0, sld_solvent=2.0)
    assert np.allclose(oracle.dsigma(oracle.Prepared(a), q), oracle.dsigma(oracle.Prepared(b), q), rtol=1e-12)
    # no shell: the plain ellipsoid, polydisperse too
    a = _m(W.CORE_SHELL_ELLIPSOID, radius=20.0, radius_polar=50.0, sld=2.0, sld_shell=7.0, poly=0.1, n_poly=10,
           isotropic=W.ISOTROPIC, n_gamma=10, n_psi=10)
    b = _m(W.ELLIPSOID, radius=20.0, radius_polar=50.0, sld=2.0, poly=0.1, n_poly=10, isotropic=W.ISOTROPIC,
           n_gamma=10, n_psi=10)
    assert np.allclose(oracle.dsigma(oracle.Prepared(a), q), oracle.dsigma(oracle.Prepared(b), q), rtol=1e-12)
    # a shell of the core's density: the ellipsoid of the outer radii
    a = _m(W.CORE_SHELL_ELLIPSOID, radius=20.0, radius_polar=50.0, thickness=4.0, thickness_face=9.0, sld=2.0,
           sld_shell=2.0)
    b = _m(W.ELLIPSOID, radius=24.0, radius_polar=59.0, sld=2.0)
    assert np.allclose(oracle.dsigma(oracle.Prepared(a), q), oracle.dsigma(oracle.Prepared(b), q), rtol=1e-12)


@pytest.mark.parametrize("kind", [W.CORE_SHELL_CYLINDER, W.HOLLOW_CYLINDER])
def test_cylinders_against_eq1_rectangles(kind):
    r, t, L, tf = 18.0, 6.0, 100.0, 9.0
    rc, rs, rv = 1.5, 4.0, 0.5
    if kind == W.CORE_SHELL_CYLINDER:
        m = _m(kind, radius=r, thickness=t, length=L, thickness_face=tf, sld=rc, sld_shell=rs, sld_solvent=rv)
        V = math.pi * (r + t) ** 2 * (L + 2 * tf)
    else:
        m = _m(kind, radius=r, thickness=t, length=L, sld=rs, sld_solvent=rv)
        V = math.pi * ((r + t) ** 2 - r ** 2) * L
    prep = oracle.Prepared(m)
    for q in _q(10, 4):
        qz, qp = _axis_parts(q, 1.1, 0.6)
        if kind == W.CORE_SHELL_CYLINDER:
            F = _cs_cylinder_F(qz, qp, r, t, L, tf, rc, rs, rv)
        else:
            F = (rs - rv) * _rect(qz, qp, r, r + t, -0.5 * L, 0.5 * L)
        ds = oracle.dsigma(prep, q[None, :])[0]
        assert ds * V == pytest.approx(F * F, rel=1e-9, abs=1e-12 * V * V), q


def test_bicelle_reductions():
    q = _q(40, 6)
    kw = dict(radius=18.0, thickness=5.0, thickness_face=7.0, length=80.0, sld_solvent=0.5, poly=0.1, n_poly=10,
              sigma_orient=0.3, n_gamma=8, n_psi=8)
    # faces of the rim's density: the core-shell cylinder
    a = _m(W.CORE_SHELL_BICELLE, sld=2.0, sld_shell=3.0, sld_face=3.0, **kw)
    b = _m(W.CORE_SHELL_CYLINDER, sld=2.0, sld_shell=3.0, **kw)
    assert np.allclose(oracle.dsigma(oracle.Prepared(a), q), oracle.dsigma(oracle.Prepared(b), q), rtol=1e-12)
    # one density throughout: the plain cylinder of the outer sizes (monodisperse)
    mono = dict(kw, poly=0.0, n_poly=1)
    a = _m(W.CORE_SHELL_BICELLE, sld=2.0, sld_shell=2.0, sld_face=2.0, **mono)
    b = _m(W.CYLINDER, radius=23.0, length=94.0, sld=2.0, sld_solvent=0.5, sigma_orient=0.3, n_gamma=8, n_psi=8)
    assert np.allclose(oracle.dsigma(oracle.Prepared(a), q), oracle.dsigma(oracle.Prepared(b), q), rtol=1e-12)


def test_bicelle_against_eq1_rectangles():
    r, t, L, tf = 18.0, 6.0, 90.0, 8.0
    rc, rr, rf, rv = 1.5, 4.0, 2.5, 0.5
    m = _m(W.CORE_SHELL_BICELLE, radius=r, thickness=t, length=L, thickness_face=tf, sld=rc, sld_shell=rr,
           sld_face=rf, sld_solvent=rv)
    V = math.pi * (r + t) ** 2 * (L + 2 * tf)
    prep = oracle.Prepared(m)
    h = 0.5 * L
    for q in _q(10, 7):
        qz, qp = _axis_parts(q, 1.1, 0.6)
        F = (rc - rv) * _rect(qz, qp, 0.0, r, -h, h)
        F += (rf - rv) * 2.0 * _rect(qz, qp, 0.0, r, h, h + tf)          # face layers
        F += (rr - rv) * _rect(qz, qp, r, r + t, -h - tf, h + tf)         # rim over the full length
        ds = oracle.dsigma(prep, q[None, :])[0]
        assert ds * V == pytest.approx(F * F, rel=1e-9, abs=1e-12 * V * V), q


def test_core_shell_ellipsoid_against_eq1_ball():
    r, rp, t, tp = 15.0, 40.0, 5.0, 9.0
    rc, rs, rv = 1.0, 3.5, 0.5
    m = _m(W.CORE_SHELL_ELLIPSOID, radius=r, radius_polar=rp, thickness=t, thickness_face=tp, sld=rc,
           sld_shell=rs, sld_solvent=rv)
    V = 4.0 / 3.0 * math.pi * (r + t) ** 2 * (rp + tp)
    prep = oracle.Prepared(m)
    n, e_t, e_p = oracle.axis_from_angles(1.1, 0.6)
    for q in _q(8, 5):
        ql = np.array([q @ e_t, q @ e_p, q @ n])
        F = (rc - rs) * _ball_F(ql, r, rp) + (rs - rv) * _ball_F(ql, r + t, rp + tp)
        ds = oracle.dsigma(prep, q[None, :])[0]
        assert ds * V == pytest.approx(F * F, rel=1e-9, abs=1e-12 * V * V), q


@pytest.mark.parametrize("kind", [W.CORE_SHELL_CYLINDER, W.HOLLOW_CYLINDER, W.CORE_SHELL_ELLIPSOID,
                                  W.CORE_SHELL_BICELLE])
def test_per_event_draws_average_to_the_quadrature(kind):
    base = dict(kind=kind, radius=12.0, thickness=4.0, thickness_face=6.0, length=60.0, radius_polar=30.0,
                sld=1e-6, sld_shell=3e-6, sld_face=2e-6, sld_solvent=0.0, volume_fraction=0.01, poly=0.15,
                poly_dist=W.GAUSSIAN, n_poly=32, isotropic=W.ISOTROPIC, n_gamma=32, n_psi=32)
    quad = W.Model(**base, sampling=W.QUADRATURE)
    ev = W.Model(**base, sampling=W.PER_EVENT)
    n = 400000
    for qv in ([0.03, 0.01, 0.0], [0.0, 0.06, 0.02]):
        q = np.tile(np.array(qv), (n, 1))
        d = oracle.dsigma_event(ev, q, seed=5, first=17)
        ref = oracle.dsigma(oracle.Prepared(quad), q[:1])[0]
        z = (d.mean() - ref) / (d.std() / math.sqrt(n))
        assert abs(z) < 4.0, (kind, qv, z)
