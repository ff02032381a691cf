"""Pins of the oracle's particles without a symmetry axis (Sec. II.B):
triaxial ellipsoid (semi-axes a, b, c) and rectangular parallelepiped
(half-edges a, b, c), oriented by three angles (theta, phi of the C axis,
psi about it).

* the frame: orthonormal, right-handed, C along (theta, phi), psi a
  rotation about C;
* reductions: a = b gives the ellipsoid of revolution (any psi), a = b = c
  the sphere;
* fixed frames against a brute-force evaluation of Eq. 1 (the volume
  integral of exp(-i Q.r)) by Gauss-Legendre quadrature over the body;
* the isotropic average of the parallelepiped: Guinier radius
  Rg^2 = (a^2 + b^2 + c^2)/3 and independence of the direction of Q;
* the per-event estimator (all three angles drawn) averages to the
  quadrature over the same laws;
* the elliptical cylinder (semi-axes a, b, length L along C) with a = b is
  the cylinder; it and the hollow rectangular prism (walls t thick) against
  brute-force volume integrals (a mapped disk times the axis; six disjoint
  wall boxes); their per-event means equal the quadrature.
"""
import math

import numpy as np
import pytest

import oracle
import sas_workloads as W


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def _word(u):
    k = int(min(max(math.floor(u * 8388608.0), 0), 8388607))
    return k << 9, (k + 0.5) / 8388608.0


def test_frame_definition():
    for th, ph, ps in [(0.3, 1.1, 0.0), (2.5, -0.7, 1.9), (1.5707963, 3.0, 4.0)]:
        f = oracle.frame(th, ph, ps)
        assert np.allclose(f @ f.T, np.eye(3), atol=1e-14)
        assert np.linalg.det(f) == pytest.approx(1.0, abs=1e-14)
        assert np.allclose(f[2], [math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        f0 = oracle.frame(th, ph, 0.0)
        assert np.allclose(f[0], math.cos(ps) * f0[0] + math.sin(ps) * f0[1], atol=1e-14)
        assert np.allclose(f[1], -math.sin(ps) * f0[0] + math.cos(ps) * f0[1], atol=1e-14)
        assert np.allclose(f, oracle.frame_from_angles(th, ph, ps), atol=1e-15)


def test_event_frame_definitions():
    wa, ua = _word(0.37)
    wb, ub = _word(0.81)
    wc, uc = _word(0.12)
    assert np.allclose(oracle.event_frame(2, 0, 0, 0, wa, wb, wc),
                       oracle.frame(math.pi * ua, 2 * math.pi * ub, 2 * math.pi * uc), atol=1e-14)
    assert np.allclose(oracle.event_frame(1, 0, 0, 0, wa, wb, wc),
                       oracle.frame(math.acos(1 - 2 * ua), 2 * math.pi * ub, 2 * math.pi * uc), atol=1e-14)
    assert np.allclose(oracle.event_frame(0, 0.4, 0.5, 0.6, wa, wb, wc), oracle.frame(0.4, 0.5, 0.6))


def _q(n, seed, scale=0.05):
    return np.random.default_rng(seed).normal(size=(n, 3)) * scale


def test_triaxial_reduces_to_ellipsoid_of_revolution_and_sphere():
    q = _q(40, 1)
    base = dict(sld=2e-6, volume_fraction=0.01, poly=0.1, n_poly=12)
    # monodisperse: the 3-axis models scale all sizes with the polydisperse
    # factor, the ellipsoid of revolution only its equatorial radius
    mono = dict(base, poly=0.0, n_poly=1)
    for psi in (0.0, 0.9):
        tri = W.Model(kind=W.TRIAXIAL_ELLIPSOID, radius=25.0, radius_b=25.0, radius_polar=60.0,
                      axis_theta=1.0, axis_phi=0.4, axis_psi=psi, sigma_orient=0.3, n_gamma=10, n_psi=10, **mono)
        rev = W.Model(kind=W.ELLIPSOID, radius=25.0, radius_polar=60.0, axis_theta=1.0, axis_phi=0.4,
                      sigma_orient=0.3, n_gamma=10, n_psi=10, **mono)
        assert np.allclose(oracle.dsigma(oracle.Prepared(tri), q), oracle.dsigma(oracle.Prepared(rev), q),
                           rtol=1e-12, atol=0)
    sph = W.Model(kind=W.SPHERE, radius=30.0, **base)
    tri = W.Model(kind=W.TRIAXIAL_ELLIPSOID, radius=30.0, radius_b=30.0, radius_polar=30.0, axis_theta=0.7,
                  axis_phi=2.0, axis_psi=1.3, **base)
    assert np.allclose(oracle.dsigma(oracle.Prepared(tri), q), oracle.dsigma(oracle.Prepared(sph), q),
                       rtol=1e-12, atol=0)


def _brute_F2(kind, a, b, c, frame, q, n=28):
    """|integral over the body of exp(-i Q.r) dV|^2 by Gauss-Legendre."""
    x, w = np.polynomial.legendre.leggauss(n)
    qa, qb, qc = frame @ q
    if kind == W.PARALLELEPIPED:
        u, v, t = np.meshgrid(a * x, b * x, c * x, indexing="ij")
        W3 = np.einsum("i,j,k->ijk", w, w, w) * a * b * c
        re = np.sum(W3 * np.cos(qa * u + qb * v + qc * t))
        im = np.sum(W3 * np.sin(qa * u + qb * v + qc * t))
    else:
        # unit ball in spherical coordinates, mapped by (a, b, c)
        rr = 0.5 * (x + 1.0)
        wr = 0.5 * w * rr ** 2
        ct = x
        ph = math.pi * (x + 1.0)
        wp = math.pi * w
        R, CT, PH = np.meshgrid(rr, ct, ph, indexing="ij")
        ST = np.sqrt(1 - CT ** 2)
        X, Y, Z = R * ST * np.cos(PH), R * ST * np.sin(PH), R * CT
        W3 = np.einsum("i,j,k->ijk", wr, w, wp) * a * b * c
        arg = qa * a * X + qb * b * Y + qc * c * Z
        re = np.sum(W3 * np.cos(arg))
        im = np.sum(W3 * np.sin(arg))
    return re * re + im * im


@pytest.mark.parametrize("kind", [W.TRIAXIAL_ELLIPSOID, W.PARALLELEPIPED])
def test_fixed_frame_against_eq1_volume_integral(kind):
    a, b, c = 12.0, 20.0, 35.0
    th, ph, ps = 1.1, 0.6, 0.8
    m = W.Model(kind=kind, radius=a, radius_b=b, radius_polar=c, sld=1.0, sld_solvent=0.0, volume_fraction=1.0,
                axis_theta=th, axis_phi=ph, axis_psi=ps)
    V = (4.0 / 3.0 * math.pi if kind == W.TRIAXIAL_ELLIPSOID else 8.0) * a * b * c
    fr = oracle.frame(th, ph, ps)
    for q in _q(8, 3, scale=0.06):
        ds = oracle.dsigma(oracle.Prepared(m), q[None, :])[0]     # (phi / V) |F|^2 with phi = 1
        assert ds * V == pytest.approx(_brute_F2(kind, a, b, c, fr, q), rel=1e-9)


def test_parallelepiped_isotropic_guinier_and_rotation_invariance():
    a, b, c = 10.0, 18.0, 30.0
    m = W.Model(kind=W.PARALLELEPIPED, radius=a, radius_b=b, radius_polar=c, sld=1.0, volume_fraction=1.0,
                isotropic=W.ISOTROPIC, n_gamma=24, n_psi=24, n_rot=24)
    prep = oracle.Prepared(m)
    rg2 = (a * a + b * b + c * c) / 3.0
    V = 8 * a * b * c
    p0 = oracle.dsigma(prep, np.zeros((1, 3)))[0]
    assert p0 == pytest.approx(V, rel=1e-12)
    for qm in (0.002, 0.004):
        p = oracle.dsigma(prep, np.array([[qm, 0.0, 0.0]]))[0] / p0
        assert abs(p - (1.0 - qm * qm * rg2 / 3.0)) < 0.1 * (qm * qm * rg2) ** 2
    dirs = _q(6, 5)
    dirs = 0.03 * dirs / np.linalg.norm(dirs, axis=1)[:, None]
    v = oracle.dsigma(prep, dirs)
    assert np.max(v) / np.min(v) - 1.0 < 1e-6


@pytest.mark.parametrize("kind", [W.TRIAXIAL_ELLIPSOID, W.PARALLELEPIPED])
@pytest.mark.parametrize("iso", [W.UNIFORM_ANGLES, W.ISOTROPIC])
def test_per_event_frames_average_to_the_quadrature(kind, iso):
    base = dict(kind=kind, radius=10.0, radius_b=16.0, radius_polar=28.0, sld=2e-6, volume_fraction=0.01,
                poly=0.15, poly_dist=W.GAUSSIAN, n_poly=32, isotropic=iso, n_gamma=24, n_psi=24, n_rot=24)
    quad = W.Model(**base, sampling=W.QUADRATURE)
    ev = W.Model(**base, sampling=W.PER_EVENT)
    n = 100000
    for qv in ([0.02, 0.01, 0.0], [0.0, 0.04, 0.02]):
        q = np.tile(np.array(qv), (n, 1))
        d = oracle.dsigma_event(ev, q, seed=3, first=50)
        ref = oracle.dsigma(oracle.Prepared(quad), q[:1])[0]
        z = (d.mean() - ref) / (d.std() / math.sqrt(n))
        assert abs(z) < 4.0, (kind, iso, qv, z)


# ------------------------------------- elliptical cylinder, hollow prism

def _brute_ellcyl_F(a, b, c, frame, q, n=40):
    """Integral of exp(-i Q.r) over the elliptical cylinder |(x/a, y/b)| <= 1,
    |z| <= c in the particle frame: the unit disk in polar coordinates
    mapped by (a, b), z by Gauss-Legendre."""
    x, w = np.polynomial.legendre.leggauss(n)
    qa, qb, qc = frame @ q
    rr = 0.5 * (x + 1.0)
    wr = 0.5 * w * rr
    ph = math.pi * (x + 1.0)
    R, PH = np.meshgrid(rr, ph, indexing="ij")
    W2 = np.outer(wr, math.pi * w) * a * b
    arg = qa * a * R * np.cos(PH) + qb * b * R * np.sin(PH)
    disk = np.sum(W2 * np.cos(arg)) + 1j * np.sum(W2 * np.sin(arg))
    z = c * x
    axial = np.sum(c * w * np.cos(qc * z)) + 1j * np.sum(c * w * np.sin(qc * z))
    return abs(disk * axial) ** 2


def _box_integral(qa, qb, qc, lo, hi, n=12):
    """Integral of exp(-i Q.r) over the box lo <= r <= hi (Gauss-Legendre)."""
    x, w = np.polynomial.legendre.leggauss(n)
    out = 1.0 + 0j
    for qk, l0, l1 in zip((qa, qb, qc), lo, hi):
        u = 0.5 * (l0 + l1) + 0.5 * (l1 - l0) * x
        out *= np.sum(0.5 * (l1 - l0) * w * np.exp(-1j * qk * u))
    return out


def _brute_hollow_prism_F(a, b, c, t, frame, q):
    """The walls as six disjoint boxes: the two C faces over the full A x B,
    the two B faces between them, the two A faces between those."""
    qa, qb, qc = frame @ q
    boxes = [((-a, -b, c - t), (a, b, c)), ((-a, -b, -c), (a, b, -c + t)),
             ((-a, b - t, -c + t), (a, b, c - t)), ((-a, -b, -c + t), (a, -b + t, c - t)),
             ((a - t, -b + t, -c + t), (a, b - t, c - t)), ((-a, -b + t, -c + t), (-a + t, b - t, c - t))]
    F = sum(_box_integral(qa, qb, qc, lo, hi) for lo, hi in boxes)
    return abs(F) ** 2


def test_elliptical_cylinder_reduces_to_the_cylinder():
    q = _q(40, 11)
    for psi in (0.0, 1.1):
        ell = W.Model(kind=W.ELLIPTICAL_CYLINDER, radius=20.0, radius_b=20.0, length=150.0, sld=2e-6,
                      volume_fraction=0.01, axis_theta=1.0, axis_phi=0.4, axis_psi=psi, sigma_orient=0.3,
                      n_gamma=10, n_psi=10)
        cyl = W.Model(kind=W.CYLINDER, radius=20.0, length=150.0, sld=2e-6, volume_fraction=0.01, axis_theta=1.0,
                      axis_phi=0.4, sigma_orient=0.3, n_gamma=10, n_psi=10)
        assert np.allclose(oracle.dsigma(oracle.Prepared(ell), q), oracle.dsigma(oracle.Prepared(cyl), q),
                           rtol=1e-12, atol=0)


@pytest.mark.parametrize("kind", [W.ELLIPTICAL_CYLINDER, W.HOLLOW_RECTANGULAR_PRISM])
def test_new_bodies_against_eq1_volume_integral(kind):
    a, b, c, t, L = 12.0, 25.0, 35.0, 4.0, 90.0
    th, ph, ps = 1.1, 0.6, 0.8
    m = W.Model(kind=kind, radius=a, radius_b=b, radius_polar=c, length=L, thickness=t, sld=1.0,
                sld_solvent=0.0, volume_fraction=1.0, axis_theta=th, axis_phi=ph, axis_psi=ps)
    if kind == W.ELLIPTICAL_CYLINDER:
        V = math.pi * a * b * L
    else:
        V = 8.0 * (a * b * c - (a - t) * (b - t) * (c - t))
    fr = oracle.frame(th, ph, ps)
    for q in _q(8, 13, scale=0.06):
        ds = oracle.dsigma(oracle.Prepared(m), q[None, :])[0]
        ref = _brute_ellcyl_F(a, b, 0.5 * L, fr, q) if kind == W.ELLIPTICAL_CYLINDER else \
            _brute_hollow_prism_F(a, b, c, t, fr, q)
        assert ds * V == pytest.approx(ref, rel=1e-9, abs=1e-12 * V * V)


@pytest.mark.parametrize("kind", [W.ELLIPTICAL_CYLINDER, W.HOLLOW_RECTANGULAR_PRISM])
def test_new_bodies_per_event_average_to_the_quadrature(kind):
    base = dict(kind=kind, radius=10.0, radius_b=16.0, radius_polar=28.0, length=60.0, thickness=3.0, sld=2e-6,
                volume_fraction=0.01, poly=0.15, poly_dist=W.GAUSSIAN, n_poly=32, isotropic=W.UNIFORM_ANGLES,
                n_gamma=24, n_psi=24, n_rot=24)
    quad = W.Model(**base, sampling=W.QUADRATURE)
    ev = W.Model(**base, sampling=W.PER_EVENT)
    n = 400000
    for qv in ([0.02, 0.01, 0.0], [0.0, 0.04, 0.02]):
        q = np.tile(np.array(qv), (n, 1))
        d = oracle.dsigma_event(ev, q, seed=3, first=50)
        ref = oracle.dsigma(oracle.Prepared(quad), q[:1])[0]
        z = (d.mean() - ref) / (d.std() / math.sqrt(n))
        assert abs(z) < 4.0, (kind, qv, z)
