"""Seeded synthetic workloads for the SANS Monte Carlo trace.

This module holds only input descriptions and seeded parameter draws. It
contains none of the method's arithmetic (no RNG stream of the trace, no
geometry, no form factor), so both the FP64 oracle and the CUDA path may use
it as their common source of inputs.

Units: instrument lengths in metres, wavelength and particle sizes in
angstrom, scattering-length densities in 1/angstrom^2, angles in radians.
The beam runs along +z; the sample front face sits at z = 0.

Workloads (the paper's KWS-1 instrument description and its measured data
set are not available, so these synthetic set-ups stand in for them; the
instrument chain follows Sec. II.A: source, collimation, sample, 2D PSD):

* ``sphere``      monodisperse sphere R=50, contrast 2e-6, phi=0.01, no S(Q),
                  128x128 detector, 1e6 neutrons, traced in FP64.
* ``core_shell``  core 40 + shell 10, SLDs (1, 3, 6)e-6 (core, shell, solvent),
                  Schulz sigma/R = 0.1 on the core radius with 40 nodes,
                  Percus-Yevick hard spheres at phi = 0.2, R_hs = 50,
                  128x128 detector, 1e9 neutrons, FP32.
* ``cylinder``    R=20, L=400, axis Gaussian (sigma 15 deg) about x (normal to
                  the beam), Schulz 0.1 on R with 40 nodes, 76x76 orientation
                  nodes, 256x256 detector, 1e9 neutrons, FP32.
* ``batched``     4096 experiments, model kind uniform over the four kinds,
                  sizes uniform in [10, 200], polydispersity uniform in
                  [0, 0.3], neutron counts log-uniform in [1e5, 1e8], 128x128
                  detector each.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

SPHERE, CORE_SHELL, CYLINDER, ELLIPSOID = 0, 1, 2, 3
TRIAXIAL_ELLIPSOID, PARALLELEPIPED = 4, 5        # no symmetry axis: sizes along A, B, C
CAPPED_CYLINDER, BARBELL = 6, 7                  # cylinder with spherical end caps (radius_polar)
CORE_SHELL_CYLINDER, HOLLOW_CYLINDER, CORE_SHELL_ELLIPSOID, CORE_SHELL_BICELLE = 8, 9, 10, 11
ELLIPTICAL_CYLINDER, HOLLOW_RECTANGULAR_PRISM = 12, 13   # no symmetry axis, like the 3-axis kinds
SHAPE_INDEPENDENT = 14                                    # dSigma/dOmega = f_scale f(|Q|), see `function`
GUINIER, GAUSS_COIL, LORENTZ, DAB, POWER_LAW, GAUSS_PEAK, TEUBNER_STREY = range(7)
PEAK_LORENTZ, TWO_POWER_LAW, GUINIER_POROD, GAUSS_LORENTZ_GEL, POLY_GAUSS_COIL, STAR_POLYMER = range(7, 13)
MASS_FRACTAL, FRACTAL, SPINODAL, POLYMER_EXCL_VOLUME, LINEAR_PEARLS = 13, 14, 15, 16, 17
MODEL_NAMES = {SPHERE: "sphere", CORE_SHELL: "core_shell", CYLINDER: "cylinder",
               ELLIPSOID: "ellipsoid", TRIAXIAL_ELLIPSOID: "triaxial_ellipsoid",
               PARALLELEPIPED: "parallelepiped", CAPPED_CYLINDER: "capped_cylinder",
               BARBELL: "barbell", CORE_SHELL_CYLINDER: "core_shell_cylinder",
               HOLLOW_CYLINDER: "hollow_cylinder", CORE_SHELL_ELLIPSOID: "core_shell_ellipsoid",
               CORE_SHELL_BICELLE: "core_shell_bicelle", ELLIPTICAL_CYLINDER: "elliptical_cylinder",
               HOLLOW_RECTANGULAR_PRISM: "hollow_rectangular_prism", SHAPE_INDEPENDENT: "shape_independent"}
SQ_NONE, SQ_HARD_SPHERE_PY, SQ_HAYTER_MSA = 0, 1, 2
FP32, FP64 = 0, 1
QUADRATURE, PER_EVENT = 0, 1              # sampling: averages over nodes / one draw per history
SCHULZ, GAUSSIAN = 0, 1                   # poly_dist of the polydisperse radius
CAP, ISOTROPIC, UNIFORM_ANGLES = 0, 1, 2  # isotropic: axis distribution of uniaxial models


@dataclass
class Instrument:
    lambda0: float = 6.0            # angstrom
    dlambda_rel: float = 0.10       # half width of the triangular spread (fraction of lambda0)
    ap1_radius: float = 4.0e-3      # m (8 mm diameter)
    ap1_z: float = -2.0             # m
    ap2_radius: float = 2.0e-3      # m (4 mm diameter)
    ap2_z: float = 0.0              # m, immediately in front of the sample
    sample_half_x: float = 5.0e-3   # m (10 mm wide)
    sample_half_y: float = 5.0e-3   # m (10 mm high)
    sample_thickness: float = 1.0e-3  # m
    mu: float = 0.0                 # 1/m, attenuation inside the sample
    det_distance: float = 5.0       # m from the sample front face
    pixel_x: float = 5.0e-3         # m
    pixel_y: float = 5.0e-3         # m
    nx: int = 128
    ny: int = 128

    def as_dict(self):
        return asdict(self)


@dataclass
class Model:
    kind: int = SPHERE
    sq_kind: int = SQ_NONE
    precision: int = FP32
    n_poly: int = 1
    n_gamma: int = 1
    n_psi: int = 1
    isotropic: int = CAP             # CAP (Gaussian about the mean axis), ISOTROPIC, UNIFORM_ANGLES
    radius: float = 50.0            # sphere R, core radius, cylinder R, ellipsoid equatorial R,
                                    # 3-axis models: semi-axis / half-edge along A
    thickness: float = 0.0          # core-shell shell thickness; hollow cylinder wall
    length: float = 0.0             # cylinder length (capped cylinder, barbell: between the end faces)
    radius_polar: float = 0.0       # ellipsoid polar radius (along the axis); 3-axis models: along C;
                                    # capped cylinder, barbell: radius of the end caps' spheres (>= radius)
    sld: float = 2.0e-6             # particle (core) SLD
    sld_shell: float = 0.0
    sld_solvent: float = 0.0
    volume_fraction: float = 0.01
    poly: float = 0.0               # Schulz relative width of the polydisperse radius
    sigma_orient: float = 0.0       # rad, Gaussian width of the axis distribution
    axis_theta: float = 0.5 * math.pi  # rad, polar angle of the mean axis from +z
    axis_phi: float = 0.0           # rad, azimuth of the mean axis
    sq_radius: float = 0.0
    sq_fraction: float = 0.0
    sampling: int = QUADRATURE      # PER_EVENT: one radius and axis drawn per history (Sec. II.B)
    poly_dist: int = SCHULZ         # GAUSSIAN: N(R, (poly R)^2) restricted to R > 0
    radial_table: int = 0           # cylinder: 1 interpolates the polydisperse radial sum from a table
    radius_b: float = 0.0           # triaxial ellipsoid semi-axis / parallelepiped half-edge along B
    axis_psi: float = 0.0           # rad, rotation of the particle frame about its C axis
    n_rot: int = 1                  # quadrature nodes in psi (uniform rotations / angles)
    self_attenuation: int = 0       # 1: attenuation mu + Sigma_s(lambda), the model's own total scattering
    n_cap: int = 16                 # capped cylinder, barbell: Gauss-Legendre nodes over each end cap
    thickness_face: float = 0.0     # core-shell cylinder: shell on the end faces; core-shell ellipsoid:
                                    # shell along the axis (thickness: radial / equatorial shell)
    sld_face: float = 0.0           # core-shell bicelle: SLD of the face layers (sld_shell is the rim's)
    function: int = GUINIER         # shape-independent: GUINIER .. LINEAR_PEARLS
    f_scale: float = 0.0            # shape-independent: dSigma/dOmega = f_scale f(|Q|), 1/angstrom
    f_p0: float = 0.0               # shape-independent parameters (Rg, xi, m, Q0 / sigma, a2 / c1 / c2)
    f_p1: float = 0.0
    f_p2: float = 0.0
    sq_charge: float = 0.0          # Hayter-Penfold S(Q): particle charge Z (elementary charges)
    sq_temperature: float = 298.15  # K
    sq_salt: float = 0.0            # mol/L of 1:1 salt
    sq_dielectric: float = 78.4     # relative permittivity of the solvent
    fuzziness: float = 0.0          # sphere: Gaussian interface width (fuzzy sphere), angstrom

    def as_dict(self):
        return asdict(self)


def instrument(nx=128, ny=128, **kw) -> Instrument:
    return Instrument(nx=nx, ny=ny, **kw)


def sphere_config():
    """Monodisperse sphere, FP64 trace, 1e6 neutrons, seed 1."""
    m = Model(kind=SPHERE, precision=FP64, radius=50.0, sld=2.0e-6, sld_solvent=0.0,
              volume_fraction=0.01, n_poly=1)
    return dict(name="sphere", instrument=instrument(), model=m, n_neutrons=10**6, seed=1)


def core_shell_config():
    """Core-shell sphere + Schulz(40) + Percus-Yevick, FP32, 1e9 neutrons, seed 1."""
    m = Model(kind=CORE_SHELL, sq_kind=SQ_HARD_SPHERE_PY, precision=FP32, radius=40.0,
              thickness=10.0, sld=1.0e-6, sld_shell=3.0e-6, sld_solvent=6.0e-6,
              volume_fraction=0.2, poly=0.1, n_poly=40, sq_radius=50.0, sq_fraction=0.2)
    return dict(name="core_shell", instrument=instrument(), model=m, n_neutrons=10**9, seed=1)


def cylinder_config():
    """Oriented polydisperse cylinder, 76x76 orientation nodes, 256x256, FP32."""
    m = Model(kind=CYLINDER, precision=FP32, radius=20.0, length=400.0, sld=2.0e-6,
              sld_solvent=0.0, volume_fraction=0.01, poly=0.1, n_poly=40,
              sigma_orient=math.radians(15.0), axis_theta=0.5 * math.pi, axis_phi=0.0,
              n_gamma=76, n_psi=76)
    return dict(name="cylinder", instrument=instrument(nx=256, ny=256), model=m,
                n_neutrons=10**9, seed=1)


def capped_cylinder_config():
    """Oriented polydisperse capped cylinder: r = 20, caps R = 25, L = 200
    angstrom, Schulz 0.1 (10 nodes), Gaussian axis spread 15 deg (16x16
    nodes), 16 slices per cap, 128x128, FP32."""
    m = Model(kind=CAPPED_CYLINDER, precision=FP32, radius=20.0, radius_polar=25.0, length=200.0,
              sld=2.0e-6, sld_solvent=0.0, volume_fraction=0.01, poly=0.1, n_poly=10,
              sigma_orient=math.radians(15.0), axis_theta=0.5 * math.pi, axis_phi=0.0,
              n_gamma=16, n_psi=16, n_cap=16)
    return dict(name="capped_cylinder", instrument=instrument(), model=m, n_neutrons=10**8, seed=1)


def barbell_config():
    """Isotropic polydisperse barbell: r = 10, bells R = 25, L = 100
    angstrom, Schulz 0.1 (10 nodes), axis uniform on the sphere (16x16
    nodes), 16 slices per bell, 128x128, FP32."""
    m = Model(kind=BARBELL, precision=FP32, radius=10.0, radius_polar=25.0, length=100.0,
              sld=2.0e-6, sld_solvent=0.0, volume_fraction=0.01, poly=0.1, n_poly=10,
              isotropic=ISOTROPIC, n_gamma=16, n_psi=16, n_cap=16)
    return dict(name="barbell", instrument=instrument(), model=m, n_neutrons=10**8, seed=1)


def shelled_configs():
    """The shelled uniaxial models at one size each: core-shell cylinder
    (r = 20, shell 5, faces 5, L = 200 A), hollow cylinder (r = 20, wall 5,
    L = 200 A), both with a Gaussian axis spread of 15 deg, and the
    core-shell ellipsoid (r = 20, r_p = 60, shells 5 A) with the axis uniform
    on the sphere, and the core-shell bicelle (r = 20, rim 5, faces 5,
    L = 200 A, face SLD 2e-6) with the cylinders' axis law; Schulz 0.1 (10
    nodes), 16x16 orientation nodes, SLDs 1, 3, 6 (x1e-6) for core, shell
    (rim) and solvent, 128x128, FP32."""
    common = dict(precision=FP32, radius=20.0, thickness=5.0, sld=1.0e-6, sld_shell=3.0e-6, sld_solvent=6.0e-6,
                  volume_fraction=0.01, poly=0.1, n_poly=10, n_gamma=16, n_psi=16)
    cyl = dict(common, length=200.0, sigma_orient=math.radians(15.0), axis_theta=0.5 * math.pi, axis_phi=0.0)
    return [dict(name="core_shell_cylinder", instrument=instrument(),
                 model=Model(kind=CORE_SHELL_CYLINDER, thickness_face=5.0, **cyl)),
            dict(name="hollow_cylinder", instrument=instrument(), model=Model(kind=HOLLOW_CYLINDER, **cyl)),
            dict(name="core_shell_ellipsoid", instrument=instrument(),
                 model=Model(kind=CORE_SHELL_ELLIPSOID, radius_polar=60.0, thickness_face=5.0,
                             isotropic=ISOTROPIC, **common)),
            dict(name="core_shell_bicelle", instrument=instrument(),
                 model=Model(kind=CORE_SHELL_BICELLE, thickness_face=5.0, **dict(cyl, sld_shell=3.0e-6),
                             sld_face=2.0e-6))]


CONFIGS = {"sphere": sphere_config, "core_shell": core_shell_config,
           "cylinder": cylinder_config}


def batched_models(n_exp=4096, seed=1, n_poly=40, n_gamma=76, n_psi=76,
                   count_range=(1e5, 1e8)):
    """Draw the batched set of experiments (numpy PCG64, seeded).

    Model kind uniform over {sphere, core-shell, cylinder, ellipsoid}; every
    size parameter uniform in [10, 200] angstrom; polydispersity uniform in
    [0, 0.3]; anisotropic particles get a Gaussian axis spread uniform in
    [0, 30] degrees about an axis uniform on the sphere; no structure factor;
    neutron counts log-uniform in ``count_range``.
    Returns (list[Model], np.ndarray[uint64] counts).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    kinds = rng.integers(0, 4, size=n_exp)
    sizes = rng.uniform(10.0, 200.0, size=(n_exp, 3))
    polys = rng.uniform(0.0, 0.3, size=n_exp)
    sig = np.radians(rng.uniform(0.0, 30.0, size=n_exp))
    cos_t = rng.uniform(-1.0, 1.0, size=n_exp)
    phis = rng.uniform(0.0, 2.0 * math.pi, size=n_exp)
    slds = rng.uniform(0.5e-6, 6.0e-6, size=(n_exp, 2))
    lo, hi = math.log(count_range[0]), math.log(count_range[1])
    counts = np.exp(rng.uniform(lo, hi, size=n_exp)).astype(np.uint64)
    models = []
    for e in range(n_exp):
        k = int(kinds[e])
        p = float(polys[e])
        npoly = n_poly if p > 0.0 else 1
        m = Model(kind=k, precision=FP32, radius=float(sizes[e, 0]), sld=float(slds[e, 0]),
                  sld_solvent=0.0, volume_fraction=0.01, poly=p, n_poly=npoly)
        if k == CORE_SHELL:
            m.thickness = float(sizes[e, 1])
            m.sld_shell = float(slds[e, 1])
            m.sld_solvent = 0.0
        if k in (CYLINDER, ELLIPSOID):
            if k == CYLINDER:
                m.length = float(sizes[e, 1])
            else:
                m.radius_polar = float(sizes[e, 1])
            m.sigma_orient = float(sig[e])
            m.axis_theta = float(math.acos(cos_t[e]))
            m.axis_phi = float(phis[e])
            if m.sigma_orient > 0.0:
                m.n_gamma, m.n_psi = n_gamma, n_psi
        models.append(m)
    return models, counts


def random_q(n, qmax, seed):
    """Uniform random scattering vectors in a ball of radius qmax (1/angstrom)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    r = qmax * rng.uniform(0.0, 1.0, size=n) ** (1.0 / 3.0)
    return v * r[:, None]


def surrogate_box(n_fourier=12, n_buckets=32):
    """Training box of the learned surrogate around the cylinder workload:
    R in [15, 25], L in [300, 500] angstrom, sigma_orient in [10, 20] deg,
    sigma_poly in [0.05, 0.15] (n_buckets values), |Q| <= 0.25 1/angstrom,
    with the cylinder workload's quadrature (40 Schulz nodes, 76 x 76
    orientation nodes)."""
    return dict(q_max=0.25, r_min=15.0, r_max=25.0, l_min=300.0, l_max=500.0,
                sigma_orient_min=math.radians(10.0), sigma_orient_max=math.radians(20.0),
                poly_min=0.05, poly_max=0.15, n_poly=40, n_gamma=76, n_psi=76,
                n_buckets=n_buckets, n_fourier=n_fourier, model=CYLINDER)


def batched_surrogate_box(n_fourier=12, n_buckets=64):
    """Training box of the learned surrogate for the cylinders of the batched
    workload: R and L in [10, 200] angstrom, sigma_orient in [0.01, 30] deg,
    sigma_poly in [2e-5, 0.3] (n_buckets values), |Q| <= 0.115 1/angstrom
    (the corner of the 128 x 128 detector seen from the edge of the sample
    at the shortest wavelength, with the beam divergence, reaches 0.110),
    with the batched quadrature (40 Schulz nodes, 76 x 76 orientation
    nodes). The lower edges sit just below the smallest spreads the 4096
    draws hold (0.014 deg, 2.7e-5), so that every drawn cylinder is
    covered; the library needs both spreads > 0."""
    return dict(q_max=0.115, r_min=10.0, r_max=200.0, l_min=10.0, l_max=200.0,
                sigma_orient_min=math.radians(0.01), sigma_orient_max=math.radians(30.0),
                poly_min=2e-5, poly_max=0.3, n_poly=40, n_gamma=76, n_psi=76,
                n_buckets=n_buckets, n_fourier=n_fourier, model=CYLINDER)


def batched_ellipsoid_surrogate_box(n_fourier=12, n_buckets=64):
    """Training box of the learned surrogate for the ellipsoids of the
    batched workload: equatorial semi-axis R and polar semi-axis R_p in
    [10, 200] angstrom (the box's length L = 2 R_p in [20, 400]), the other
    ranges and the quadrature as for the batched cylinders."""
    return dict(batched_surrogate_box(n_fourier, n_buckets), l_min=20.0, l_max=400.0, model=ELLIPSOID)
