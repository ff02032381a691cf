"""Pins of the oracle's capped cylinder and barbell: a cylinder of radius r
and length L with spherical end caps of radius R >= r. The caps are the
parts of two spheres beyond the end faces; the capped cylinder has the
spheres' centres inside the cylinder, h = sqrt(R^2 - r^2) from each face,
the barbell outside it, h beyond each face. The oracle sums Eq. 1 over disk
slices normal to the axis, the cap integral by Gauss-Legendre.

* volume: the forward scattering |F(0)|^2 = V^2 against the textbook
  spherical-cap volume pi H^2 (3R - H) / 3, H = R -+ h;
* reductions: R = r and L = 0 is the sphere of radius r; with R = r the two
  models are the same body; R >> r leaves the plain cylinder;
* fixed axes against an independent evaluation of Eq. 1: cylindrical shells
  about the axis, the z integral and the azimuth in closed form (2 J0), the
  shell radius by Gauss-Legendre in s = sqrt(R^2 - rho^2);
* the isotropic average's Guinier radius from the shell integral.
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


def _model(kind, r, R, L, **kw):
    base = dict(kind=kind, radius=r, radius_polar=R, length=L, sld=1.0, sld_solvent=0.0, volume_fraction=1.0,
                n_cap=24)
    base.update(kw)
    return W.Model(**base)


def _cap_volume(kind, r, R):
    h = math.sqrt(R * R - r * r)
    H = R - h if kind == W.CAPPED_CYLINDER else R + h
    return math.pi * H * H * (3.0 * R - H) / 3.0


def _volume(kind, r, R, L):
    return math.pi * r * r * L + 2.0 * _cap_volume(kind, r, R)


def _zc(kind, r, R, L):
    h = math.sqrt(R * R - r * r)
    return 0.5 * L - h if kind == W.CAPPED_CYLINDER else 0.5 * L + h


def _shell_F(kind, r, R, L, qz, qp, n=96):
    """F(Q) = integral of exp(i Q.x) over the body, sliced into cylindrical
    shells about the axis. A shell of radius rho meets the body in z
    intervals with end points fixed by the spheres: for rho <= r the single
    interval |z| <= z_c + s, s = sqrt(R^2 - rho^2) (the cylinder joined to
    both caps); for r < rho <= R (barbell only) the two sphere chords
    |z -+ z_c| <= s. The z integral of exp(i q_z z) and the azimuthal one,
    2 pi J0(q_p rho), are closed forms; rho dRho = -s ds."""
    zc = _zc(kind, r, R, L)
    h = math.sqrt(R * R - r * r)
    x, w = np.polynomial.legendre.leggauss(n)

    def zint(half):                      # integral over |z| <= half of exp(i q_z z)
        return 2.0 * half * np.sinc(qz * half / math.pi)

    s = 0.5 * (R + h) + 0.5 * (R - h) * x
    ws = 0.5 * (R - h) * w
    rho = np.sqrt(np.maximum(R * R - s * s, 0.0))
    F = np.sum(ws * s * 2.0 * math.pi * sp.j0(qp * rho) * zint(zc + s))
    if kind == W.BARBELL and h > 0.0:
        s = 0.5 * h * (x + 1.0)
        ws = 0.5 * h * w
        rho = np.sqrt(R * R - s * s)
        F += np.sum(ws * s * 2.0 * math.pi * sp.j0(qp * rho) * 2.0 * math.cos(qz * zc) * zint(s))
    return F


def _shell_rg2(kind, r, R, L, n=96):
    """Radius of gyration squared, the same shells: <rho^2 + z^2> over the body."""
    zc = _zc(kind, r, R, L)
    h = math.sqrt(R * R - r * r)
    x, w = np.polynomial.legendre.leggauss(n)
    s = 0.5 * (R + h) + 0.5 * (R - h) * x
    ws = 0.5 * (R - h) * w
    rho2 = np.maximum(R * R - s * s, 0.0)
    Z = zc + s
    V = np.sum(ws * s * 2.0 * math.pi * 2.0 * Z)
    M = np.sum(ws * s * 2.0 * math.pi * (rho2 * 2.0 * Z + 2.0 * Z ** 3 / 3.0))
    if kind == W.BARBELL and h > 0.0:
        s = 0.5 * h * (x + 1.0)
        ws = 0.5 * h * w
        rho2 = R * R - s * s
        V += np.sum(ws * s * 2.0 * math.pi * 2.0 * 2.0 * s)
        # two chords [zc - s, zc + s] and mirror: integral of z^2 = 2 (2 s zc^2 + 2 s^3 / 3)
        M += np.sum(ws * s * 2.0 * math.pi * (rho2 * 4.0 * s + 2.0 * (2.0 * s * zc * zc + 2.0 * s ** 3 / 3.0)))
    return M / V, V


@pytest.mark.parametrize("kind", [W.CAPPED_CYLINDER, W.BARBELL])
@pytest.mark.parametrize("r,R,L", [(20.0, 25.0, 100.0), (10.0, 30.0, 80.0), (15.0, 15.0, 40.0)])
def test_forward_scattering_is_the_cap_volume(kind, r, R, L):
    V = _volume(kind, r, R, L)
    m = _model(kind, r, R, L)
    p0 = oracle.dsigma(oracle.Prepared(m), np.zeros((1, 3)))[0]     # (phi / V) V^2 with phi = drho = 1
    assert p0 == pytest.approx(V, rel=1e-12)
    # the shells agree on the volume
    assert _shell_rg2(kind, r, R, L)[1] == pytest.approx(V, rel=1e-10)


def test_reductions():
    q = np.random.default_rng(2).normal(size=(30, 3)) * 0.08
    for kind in (W.CAPPED_CYLINDER, W.BARBELL):
        # R = r and L = 0: two hemispheres, the sphere of radius r
        m = _model(kind, 30.0, 30.0, 0.0, axis_theta=0.7, axis_phi=1.9, n_cap=40)
        sph = W.Model(kind=W.SPHERE, radius=30.0, sld=1.0, volume_fraction=1.0)
        assert np.allclose(oracle.dsigma(oracle.Prepared(m), q), oracle.dsigma(oracle.Prepared(sph), q),
                           rtol=1e-10, atol=1e-12 * 4 / 3 * math.pi * 30.0 ** 3)
    # R = r: capped cylinder and barbell are the same spherocylinder
    a = _model(W.CAPPED_CYLINDER, 20.0, 20.0, 90.0, sigma_orient=0.3, n_gamma=8, n_psi=8, poly=0.1, n_poly=6)
    b = _model(W.BARBELL, 20.0, 20.0, 90.0, sigma_orient=0.3, n_gamma=8, n_psi=8, poly=0.1, n_poly=6)
    assert np.allclose(oracle.dsigma(oracle.Prepared(a), q), oracle.dsigma(oracle.Prepared(b), q), rtol=1e-13)
    # R >> r: the caps are lenses of height r^2 / 2R, the plain cylinder is left
    cap = _model(W.CAPPED_CYLINDER, 20.0, 2.0e6, 100.0, axis_theta=1.0, axis_phi=0.3)
    cyl = W.Model(kind=W.CYLINDER, radius=20.0, length=100.0, sld=1.0, volume_fraction=1.0, axis_theta=1.0,
                  axis_phi=0.3)
    # |F| differs by at most the caps' volume (|exp(i Q.x)| = 1 over them)
    Vcap, Vcyl = _volume(W.CAPPED_CYLINDER, 20.0, 2.0e6, 100.0), math.pi * 400.0 * 100.0
    Fa = np.sqrt(oracle.dsigma(oracle.Prepared(cap), q) * Vcap)
    Fb = np.sqrt(oracle.dsigma(oracle.Prepared(cyl), q) * Vcyl)
    assert 0.0 < Vcap - Vcyl < 1e-5 * Vcyl
    assert np.all(np.abs(Fa - Fb) <= (Vcap - Vcyl) * (1 + 1e-6) + 1e-9 * Vcyl)


@pytest.mark.parametrize("kind", [W.CAPPED_CYLINDER, W.BARBELL])
@pytest.mark.parametrize("r,R,L", [(20.0, 25.0, 100.0), (10.0, 30.0, 60.0)])
def test_fixed_axis_against_eq1_shells(kind, r, R, L):
    th, ph = 1.1, 0.6
    m = _model(kind, r, R, L, axis_theta=th, axis_phi=ph)
    c = oracle.axis_from_angles(th, ph)[0]
    V = _volume(kind, r, R, L)
    prep = oracle.Prepared(m)
    rng = np.random.default_rng(7)
    for q in rng.normal(size=(10, 3)) * 0.06:
        qz = float(q @ c)
        qp = float(np.linalg.norm(q - qz * c))
        F = _shell_F(kind, r, R, L, qz, qp)
        ds = oracle.dsigma(prep, q[None, :])[0]
        assert ds * V == pytest.approx(F * F, rel=1e-9, abs=1e-12 * V * V), (q, ds * V, F * F)


@pytest.mark.parametrize("kind", [W.CAPPED_CYLINDER, W.BARBELL])
def test_isotropic_guinier(kind):
    r, R, L = 12.0, 20.0, 60.0
    m = _model(kind, r, R, L, isotropic=W.ISOTROPIC, n_gamma=32, n_psi=8)
    prep = oracle.Prepared(m)
    rg2, V = _shell_rg2(kind, r, R, L)
    p0 = oracle.dsigma(prep, np.zeros((1, 3)))[0]
    for qm in (0.001, 0.002):
        p = oracle.dsigma(prep, np.array([[0.0, qm, 0.0]]))[0] / p0
        assert abs(p - (1.0 - qm * qm * rg2 / 3.0)) < 0.1 * (qm * qm * rg2) ** 2


def test_polydisperse_scales_every_size():
    """One polydisperse factor scales r, R and L: a node's volume is V(r_i / r)^3."""
    r, R, L = 20.0, 25.0, 100.0
    m = _model(W.BARBELL, r, R, L, poly=0.2, n_poly=16)
    prep = oracle.Prepared(m)
    V = _volume(W.BARBELL, r, R, L)
    s = prep.poly_r / r
    v2 = np.sum(prep.poly_w * (V * s ** 3) ** 2)
    v1 = np.sum(prep.poly_w * V * s ** 3)
    assert oracle.dsigma(prep, np.zeros((1, 3)))[0] == pytest.approx(v2 / v1, rel=1e-12)


@pytest.mark.parametrize("kind,iso", [(W.CAPPED_CYLINDER, W.ISOTROPIC), (W.BARBELL, W.UNIFORM_ANGLES)])
def test_per_event_draws_average_to_the_quadrature(kind, iso):
    """The per-event estimator (one Gaussian radius and one axis drawn per
    history, Sec. II.B) has the quadrature over the same laws as its mean."""
    base = dict(kind=kind, radius=12.0, radius_polar=18.0, length=50.0, sld=2e-6, volume_fraction=0.01,
                poly=0.15, poly_dist=W.GAUSSIAN, n_poly=32, isotropic=iso, n_gamma=32, n_psi=32, n_cap=16)
    quad = W.Model(**base, sampling=W.QUADRATURE)
    ev = W.Model(**base, sampling=W.PER_EVENT)
    n = 400000   # |F|^2 of one drawn elongated body is heavy-tailed; the z test wants many draws
    for qv in ([0.03, 0.01, 0.0], [0.0, 0.06, 0.02]):
        q = np.tile(np.array(qv), (n, 1))
        d = oracle.dsigma_event(ev, q, seed=5, first=17)
        ref = oracle.dsigma(oracle.Prepared(quad), q[:1])[0]
        z = (d.mean() - ref) / (d.std() / math.sqrt(n))
        assert abs(z) < 4.0, (kind, iso, qv, z)
