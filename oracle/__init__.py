"""FP64 CPU oracle of the SANS Monte Carlo trace.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only users. Nothing in the CUDA
library imports, links or calls this package, and this package imports
nothing from the CUDA library.

The C part (``sas_oracle.c``) traces neutrons in double precision; this
module builds it with gcc, loads it with ctypes and computes the quadrature
nodes it consumes:

* Schulz polydispersity: the Schulz density of mean rbar and relative width
  p, f(r) ~ r^z exp(-(z+1) r / rbar) with z = 1/p^2 - 1, becomes the
  generalised Laguerre weight x^z e^-x under x = (z+1) r / rbar, so an
  n-point generalised Gauss-Laguerre rule (alpha = z) gives nodes
  r_i = rbar x_i / (z+1); it is exact for <r^k> with k <= 2n-1.
  (The paper samples a Gaussian per event, Sec. II.B; the Schulz rule with a
  fixed node count is the reading used here for the polydisperse workloads.)
* Orientation: the particle axis is spread about a mean axis n with density
  proportional to exp(-gamma^2 / (2 sigma^2)) on the unit sphere (gamma is the
  angle from n, psi the azimuth about n), truncated at gamma = min(3 sigma, pi),
  integrated by Gauss-Legendre in gamma (with the sin(gamma) area element)
  and Gauss-Legendre in psi over [0, 2 pi). The axis of node (gamma, psi) is
  cos(gamma) n + sin(gamma) (cos(psi) e_theta + sin(psi) e_phi), with e_theta,
  e_phi the spherical unit vectors at n. Isotropic: gamma over [0, pi], flat.
  Orientation angles theta, phi of the axis follow Sec. II.A (Eq. 7).

Both rules use the Golub-Welsch construction (eigen-decomposition of the
Jacobi matrix of the orthogonal polynomials) with numpy's symmetric
eigensolver.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sas_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsas_oracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, FP64, OpenMP). Returns the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Instrument(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "lambda0", "dlambda_rel", "ap1_radius", "ap1_z", "ap2_radius", "ap2_z",
        "sample_half_x", "sample_half_y", "sample_thickness", "mu", "det_distance",
        "pixel_x", "pixel_y")] + [("nx", ctypes.c_int64), ("ny", ctypes.c_int64)]


_DP = ctypes.POINTER(ctypes.c_double)


class _Model(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int64), ("sq_kind", ctypes.c_int64),
                ("n_poly", ctypes.c_int64), ("n_orient", ctypes.c_int64)] + \
               [(n, ctypes.c_double) for n in (
                   "radius", "thickness", "length", "radius_polar", "sld", "sld_shell",
                   "sld_solvent", "volume_fraction", "sq_radius", "sq_fraction")] + \
               [("poly_r", _DP), ("poly_w", _DP), ("orient_c", _DP), ("orient_w", _DP)] + \
               [("event", ctypes.c_int64), ("orient_mode", ctypes.c_int64), ("poly", ctypes.c_double),
                ("axis_theta", ctypes.c_double), ("axis_phi", ctypes.c_double),
                ("radius_b", ctypes.c_double), ("axis_psi", ctypes.c_double),
                ("self_att", ctypes.c_int64), ("n_cap", ctypes.c_int64), ("thickness_face", ctypes.c_double),
                ("sld_face", ctypes.c_double), ("function", ctypes.c_int64)] + \
               [(n, ctypes.c_double) for n in ("f_scale", "f_p0", "f_p1", "f_p2")] + \
               [("sq_tab", _DP), ("sq_n", ctypes.c_int64), ("sq_dq", ctypes.c_double),
                ("fuzz", ctypes.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            L.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
            for f in ("oracle_sphere_f", "oracle_cyl_a", "oracle_sinc"):
                getattr(L, f).argtypes = [ctypes.c_double]
                getattr(L, f).restype = ctypes.c_double
            L.oracle_sq_py.argtypes = [ctypes.c_double] * 3
            L.oracle_sq_py.restype = ctypes.c_double
            L.oracle_dsigma.argtypes = [ctypes.POINTER(_Model), _DP]
            L.oracle_dsigma.restype = ctypes.c_double
            L.oracle_dsigma_many.argtypes = [ctypes.POINTER(_Model), _DP, ctypes.c_int64, _DP]
            L.oracle_trace.argtypes = [ctypes.POINTER(_Instrument), ctypes.POINTER(_Model),
                                       ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                       ctypes.c_uint64, _DP, _DP,
                                       ctypes.POINTER(ctypes.c_uint64), _DP, ctypes.c_int]
            L.oracle_records.argtypes = [ctypes.POINTER(_Instrument), ctypes.POINTER(_Model),
                                         ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                         ctypes.c_uint64, ctypes.POINTER(ctypes.c_int64), _DP]
            L.oracle_geometry_records.argtypes = [ctypes.POINTER(_Instrument), ctypes.c_uint64,
                                                  ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64,
                                                  ctypes.POINTER(ctypes.c_int64), _DP, _DP, _DP]
            L.oracle_erfcinv.argtypes = [ctypes.c_double]
            L.oracle_erfcinv.restype = ctypes.c_double
            L.oracle_event_radius.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_uint32]
            L.oracle_event_radius.restype = ctypes.c_double
            L.oracle_event_axis.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_uint32,
                                            ctypes.c_uint32, _DP]
            L.oracle_dsigma_event_many.argtypes = [ctypes.POINTER(_Model), _DP, ctypes.c_uint64, ctypes.c_uint32,
                                                   ctypes.c_uint64, ctypes.c_int64, _DP]
            L.oracle_frame.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, _DP]
            L.oracle_event_frame.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _DP]
            L.oracle_num_threads.restype = ctypes.c_int
            L.oracle_sample_lambda.argtypes = [ctypes.c_double] * 3
            L.oracle_sample_lambda.restype = ctypes.c_double
            L.oracle_model_extent.argtypes = [ctypes.POINTER(_Model)]
            L.oracle_model_extent.restype = ctypes.c_double
            L.oracle_sigma_s.argtypes = [ctypes.POINTER(_Model), ctypes.c_double, ctypes.c_double]
            L.oracle_sigma_s.restype = ctypes.c_double
            L.oracle_sigma_s_panel.argtypes = [ctypes.POINTER(_Model), ctypes.c_double, ctypes.c_double,
                                               ctypes.c_int]
            L.oracle_sigma_s_panel.restype = ctypes.c_double
            L.oracle_sigma_s_npanels.argtypes = [ctypes.POINTER(_Model), ctypes.c_double]
            L.oracle_sigma_s_npanels.restype = ctypes.c_int
            L.oracle_att_table.argtypes = [ctypes.POINTER(_Instrument), ctypes.POINTER(_Model), _DP, _DP, _DP]
            L.oracle_att_table.restype = ctypes.c_int
            L.oracle_att_eval.argtypes = [ctypes.POINTER(_Instrument), ctypes.POINTER(_Model), _DP,
                                          ctypes.c_int64, _DP]
            _lib = L
    return _lib


# ------------------------------------------------------------- quadrature

def gauss_legendre(n: int):
    """n-point Gauss-Legendre rule on [-1, 1] by Golub-Welsch."""
    if n == 1:
        return np.array([0.0]), np.array([2.0])
    k = np.arange(1, n, dtype=np.float64)
    off = k / np.sqrt(4.0 * k * k - 1.0)
    J = np.diag(off, 1) + np.diag(off, -1)
    x, V = np.linalg.eigh(J)
    w = 2.0 * V[0, :] ** 2
    return x, w


def gauss_laguerre_gen(n: int, alpha: float):
    """n-point generalised Gauss-Laguerre rule for x^alpha e^-x on (0, inf),
    weights normalised to sum 1, by Golub-Welsch."""
    k = np.arange(n, dtype=np.float64)
    diag = 2.0 * k + alpha + 1.0
    kk = np.arange(1, n, dtype=np.float64)
    off = np.sqrt(kk * (kk + alpha))
    J = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    x, V = np.linalg.eigh(J)
    w = V[0, :] ** 2
    return x, w / w.sum()


def schulz_nodes(mean: float, p: float, n: int):
    """Nodes and normalised weights of the Schulz distribution of mean `mean`
    and relative standard deviation p; p == 0 or n == 1 gives the mean."""
    if p <= 0.0 or n <= 1:
        return np.array([float(mean)]), np.array([1.0])
    z = 1.0 / (p * p) - 1.0
    x, w = gauss_laguerre_gen(n, z)
    return mean * x / (z + 1.0), w


def gaussian_nodes(mean: float, p: float, n: int):
    """Nodes and normalised weights of the Gaussian N(mean, (p mean)^2)
    restricted to positive values (Sec. II.B): Gauss-Legendre on
    [max(0, mean (1 - 8p)), mean (1 + 8p)] weighted by the density; the
    mass beyond 8 sigma is below 1e-15. p == 0 or n == 1 gives the mean."""
    if p <= 0.0 or n <= 1:
        return np.array([float(mean)]), np.array([1.0])
    a, b = max(0.0, mean * (1.0 - 8.0 * p)), mean * (1.0 + 8.0 * p)
    x, w = gauss_legendre(n)
    r = 0.5 * (b - a) * (x + 1.0) + a
    wr = 0.5 * (b - a) * w * np.exp(-0.5 * ((r - mean) / (p * mean)) ** 2)
    return r, wr / wr.sum()


def radius_nodes(m):
    """Nodes of the polydisperse radius for the model's distribution
    (poly_dist 0: Schulz, 1: Gaussian restricted to r > 0)."""
    if int(m.get("poly_dist", 0)) == 1:
        return gaussian_nodes(m["radius"], m["poly"], int(m["n_poly"]))
    return schulz_nodes(m["radius"], m["poly"], int(m["n_poly"]))


def uniform_angle_nodes(n_theta, n_phi):
    """Axis nodes for theta ~ U[0, pi], phi ~ U[0, 2 pi] (Sec. II.B; uniform
    in the angles, so not uniform on the sphere): Gauss-Legendre in both."""
    xt, wt = gauss_legendre(n_theta)
    xp, wp = gauss_legendre(n_phi)
    th = 0.5 * math.pi * (xt + 1.0)
    ph = math.pi * (xp + 1.0)
    T, P = np.meshgrid(th, ph, indexing="ij")
    c = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], axis=-1)
    W = np.outer(wt, wp).reshape(-1)
    return c.reshape(-1, 3), W / W.sum()


def frame_from_angles(theta, phi, psi):
    """Particle frame rows (A, B, C): C along (theta, phi); A, B the unit
    vectors e_theta, e_phi of C rotated by psi about C (Sec. II.B)."""
    st, ct, sp, cp = math.sin(theta), math.cos(theta), math.sin(phi), math.cos(phi)
    et = np.array([ct * cp, ct * sp, -st])
    ep = np.array([-sp, cp, 0.0])
    A = math.cos(psi) * et + math.sin(psi) * ep
    B = -math.sin(psi) * et + math.cos(psi) * ep
    C = np.array([st * cp, st * sp, ct])
    return np.stack([A, B, C])


def _rotation_taking(u, v):
    """Rotation matrix of the smallest rotation taking unit u to unit v."""
    k = np.cross(u, v)
    s, c = np.linalg.norm(k), float(np.dot(u, v))
    if s < 1e-15:
        return np.eye(3)
    k = k / s
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + s * K + (1.0 - c) * (K @ K)


def frame_nodes(m):
    """Orientation nodes of a particle without a symmetry axis: frames
    [n][3][3] (rows A, B, C) and normalised weights. isotropic 0: the
    Gaussian cap of the C axis about (axis_theta, axis_phi) (as for the
    uniaxial models), the mean frame carried along by the smallest rotation
    taking its C to the node's; 1: uniform rotations (Gauss-Legendre in
    cos theta, phi and psi); 2: theta, phi and psi uniform (Sec. II.B)."""
    iso = int(m["isotropic"])
    ng, npsi, nr = int(m["n_gamma"]), int(m["n_psi"]), int(m.get("n_rot", 1))
    if iso == 0:
        F0 = frame_from_angles(m["axis_theta"], m["axis_phi"], m.get("axis_psi", 0.0))
        c, w = orientation_nodes(m["axis_theta"], m["axis_phi"], m["sigma_orient"], ng, npsi, False)
        frames = np.stack([(_rotation_taking(F0[2], ci) @ F0.T).T for ci in c])
        return frames, w
    xt, wt = gauss_legendre(ng)
    xp, wp = gauss_legendre(npsi)
    xr, wr = gauss_legendre(nr)
    if iso == 1:
        th = np.arccos(np.clip(xt, -1.0, 1.0))            # cos theta uniform on [-1, 1]
    else:
        th = 0.5 * math.pi * (xt + 1.0)
    ph = math.pi * (xp + 1.0)
    ps = math.pi * (xr + 1.0)
    frames, w = [], []
    for i, t in enumerate(th):
        for j, f in enumerate(ph):
            for k, q in enumerate(ps):
                frames.append(frame_from_angles(t, f, q))
                w.append(wt[i] * wp[j] * wr[k])
    w = np.array(w)
    return np.stack(frames), w / w.sum()


def axis_from_angles(theta: float, phi: float):
    n = np.array([math.sin(theta) * math.cos(phi), math.sin(theta) * math.sin(phi),
                  math.cos(theta)])
    e_t = np.array([math.cos(theta) * math.cos(phi), math.cos(theta) * math.sin(phi),
                    -math.sin(theta)])
    e_p = np.array([-math.sin(phi), math.cos(phi), 0.0])
    return n, e_t, e_p


def orientation_nodes(theta, phi, sigma, n_gamma, n_psi, isotropic=False):
    """Axis unit vectors [n,3] and normalised weights [n] of the orientation
    distribution (see the module docstring)."""
    n, e_t, e_p = axis_from_angles(theta, phi)
    if not isotropic and (sigma <= 0.0 or n_gamma * n_psi <= 1):
        return n[None, :].copy(), np.array([1.0])
    gmax = math.pi if isotropic else min(3.0 * sigma, math.pi)
    xg, wg = gauss_legendre(n_gamma)
    xp, wp = gauss_legendre(n_psi)
    gam = 0.5 * gmax * (xg + 1.0)
    wgam = 0.5 * gmax * wg * np.sin(gam)
    if not isotropic:
        wgam = wgam * np.exp(-gam * gam / (2.0 * sigma * sigma))
    psi = math.pi * (xp + 1.0)
    wpsi = math.pi * wp
    G, P = np.meshgrid(gam, psi, indexing="ij")
    W = np.outer(wgam, wpsi)
    c = (np.cos(G)[..., None] * n + np.sin(G)[..., None] *
         (np.cos(P)[..., None] * e_t + np.sin(P)[..., None] * e_p))
    W = W.reshape(-1)
    return c.reshape(-1, 3), W / W.sum()


# ----------------------------------------------------------- marshalling

class Prepared:
    """A model bound to its quadrature tables (keeps the arrays alive)."""

    def __init__(self, model):
        m = model if isinstance(model, dict) else model.as_dict()
        self.m = m
        kind = int(m["kind"])
        self.poly_r, self.poly_w = radius_nodes(m)
        iso = int(m["isotropic"])
        if kind in (4, 5, 12, 13):
            fr, self.orient_w = frame_nodes(m)
            self.orient_c = fr.reshape(-1, 9)
        elif kind in (2, 3, 6, 7, 8, 9, 10, 11) and iso == 2:
            self.orient_c, self.orient_w = uniform_angle_nodes(int(m["n_gamma"]), int(m["n_psi"]))
        elif kind in (2, 3, 6, 7, 8, 9, 10, 11):
            self.orient_c, self.orient_w = orientation_nodes(
                m["axis_theta"], m["axis_phi"], m["sigma_orient"], int(m["n_gamma"]),
                int(m["n_psi"]), bool(iso))
        else:
            self.orient_c, self.orient_w = np.zeros((1, 3)), np.ones(1)
        self.poly_r = np.ascontiguousarray(self.poly_r, dtype=np.float64)
        self.poly_w = np.ascontiguousarray(self.poly_w, dtype=np.float64)
        self.orient_c = np.ascontiguousarray(self.orient_c, dtype=np.float64)
        self.orient_w = np.ascontiguousarray(self.orient_w, dtype=np.float64)
        # Hayter-Penfold S(Q): solved here (oracle/msa.py), tabulated at
        # Q sigma' steps of 0.02 to 1 / angstrom for the C side
        self.sq_tab = np.zeros(2)
        sq_n, sq_dq = 0, 0.0
        if int(m["sq_kind"]) == 2:
            from . import msa
            self.msa = msa.Solution(m["sq_radius"], m["sq_fraction"], m.get("sq_charge", 0.0),
                                    m.get("sq_temperature", 298.15), m.get("sq_salt", 0.0),
                                    m.get("sq_dielectric", 78.4))
            sig = self.msa.sigma * self.msa.s
            sq_n = int(math.ceil(1.0 * sig / 0.02)) + 3
            sq_dq, S, D = self.msa.table(0.02 / sig * (sq_n - 1), sq_n)
            self.sq_tab = np.ascontiguousarray(np.stack([S, D], axis=1).reshape(-1))
        self.c = _Model(kind=kind, sq_kind=int(m["sq_kind"]), n_poly=len(self.poly_r),
                        n_orient=len(self.orient_w), radius=m["radius"],
                        thickness=m["thickness"], length=m["length"],
                        radius_polar=m["radius_polar"], sld=m["sld"],
                        sld_shell=m["sld_shell"], sld_solvent=m["sld_solvent"],
                        volume_fraction=m["volume_fraction"], sq_radius=m["sq_radius"],
                        sq_fraction=m["sq_fraction"],
                        poly_r=self.poly_r.ctypes.data_as(_DP),
                        poly_w=self.poly_w.ctypes.data_as(_DP),
                        orient_c=self.orient_c.ctypes.data_as(_DP),
                        orient_w=self.orient_w.ctypes.data_as(_DP),
                        event=int(m.get("sampling", 0)), orient_mode=iso, poly=float(m["poly"]),
                        axis_theta=float(m["axis_theta"]), axis_phi=float(m["axis_phi"]),
                        radius_b=float(m.get("radius_b", 0.0)), axis_psi=float(m.get("axis_psi", 0.0)),
                        self_att=int(m.get("self_attenuation", 0)), n_cap=int(m.get("n_cap", 16)),
                        thickness_face=float(m.get("thickness_face", 0.0)),
                        sld_face=float(m.get("sld_face", 0.0)), function=int(m.get("function", 0)),
                        f_scale=float(m.get("f_scale", 0.0)), f_p0=float(m.get("f_p0", 0.0)),
                        f_p1=float(m.get("f_p1", 0.0)), f_p2=float(m.get("f_p2", 0.0)),
                        sq_tab=self.sq_tab.ctypes.data_as(_DP), sq_n=sq_n, sq_dq=sq_dq,
                        fuzz=float(m.get("fuzziness", 0.0)))


def _inst(instrument):
    d = instrument if isinstance(instrument, dict) else instrument.as_dict()
    return _Instrument(**{k: (int(v) if k in ("nx", "ny") else float(v)) for k, v in d.items()})


# ------------------------------------------------------------- public API

def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, k, o)
    return list(o)


def sphere_f(x):
    return lib().oracle_sphere_f(float(x))


def cyl_a(x):
    return lib().oracle_cyl_a(float(x))


def sinc(x):
    return lib().oracle_sinc(float(x))


def sq_py(q, radius, phi):
    return lib().oracle_sq_py(float(q), float(radius), float(phi))


def dsigma(model, q_xyz):
    """dSigma/dOmega in 1/angstrom at scattering vectors q_xyz [n,3] (1/angstrom)."""
    prep = model if isinstance(model, Prepared) else Prepared(model)
    q = np.ascontiguousarray(np.asarray(q_xyz, dtype=np.float64).reshape(-1, 3))
    out = np.empty(q.shape[0], dtype=np.float64)
    lib().oracle_dsigma_many(ctypes.byref(prep.c), q.ctypes.data_as(_DP), q.shape[0],
                             out.ctypes.data_as(_DP))
    return out


def trace(instrument, model, n, seed, first=0, exp_id=0, threads=0):
    """Trace neutrons [first, first+n). Returns dict(sum_w, sum_w2, count, trans)
    with detector arrays of shape (ny, nx)."""
    inst = _inst(instrument)
    prep = model if isinstance(model, Prepared) else Prepared(model)
    npix = inst.nx * inst.ny
    sw = np.zeros(npix)
    sw2 = np.zeros(npix)
    cnt = np.zeros(npix, dtype=np.uint64)
    tr = ctypes.c_double(0.0)
    lib().oracle_trace(ctypes.byref(inst), ctypes.byref(prep.c), int(seed), int(exp_id),
                       int(first), int(n), sw.ctypes.data_as(_DP), sw2.ctypes.data_as(_DP),
                       cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), ctypes.byref(tr),
                       int(threads))
    shp = (inst.ny, inst.nx)
    return dict(sum_w=sw.reshape(shp), sum_w2=sw2.reshape(shp), count=cnt.reshape(shp),
                trans=tr.value)


def records(instrument, model, n, seed, first=0, exp_id=0):
    """Per-neutron (pixel, weight); pixel -1 marks a history that missed."""
    inst = _inst(instrument)
    prep = model if isinstance(model, Prepared) else Prepared(model)
    pix = np.empty(n, dtype=np.int64)
    w = np.empty(n, dtype=np.float64)
    lib().oracle_records(ctypes.byref(inst), ctypes.byref(prep.c), int(seed), int(exp_id),
                         int(first), int(n), pix.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                         w.ctypes.data_as(_DP))
    return pix, w


def geometry_records(instrument, n, seed, first=0, exp_id=0):
    """Per-neutron geometry: pixel (-1 on a miss), Q [n][3] (1/angstrom), the
    prefactor with weight = prefactor * dSigma/dOmega(Q) (dSigma/dOmega in
    1/angstrom), and the transmitted weight."""
    inst = _inst(instrument)
    pix = np.empty(n, dtype=np.int64)
    q = np.empty((n, 3), dtype=np.float64)
    pref = np.empty(n, dtype=np.float64)
    wt = np.empty(n, dtype=np.float64)
    lib().oracle_geometry_records(ctypes.byref(inst), int(seed), int(exp_id), int(first), int(n),
                                  pix.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                  q.ctypes.data_as(_DP), pref.ctypes.data_as(_DP), wt.ctypes.data_as(_DP))
    return dict(pixel=pix, q=q, pref=pref, trans=wt)


def frame(theta, phi, psi):
    f = np.empty(9)
    lib().oracle_frame(float(theta), float(phi), float(psi), f.ctypes.data_as(_DP))
    return f.reshape(3, 3)


def event_frame(mode, theta, phi, psi, wa, wb, wc):
    f = np.empty(9)
    lib().oracle_event_frame(int(mode), float(theta), float(phi), float(psi), int(wa) & 0xFFFFFFFF,
                             int(wb) & 0xFFFFFFFF, int(wc) & 0xFFFFFFFF, f.ctypes.data_as(_DP))
    return f.reshape(3, 3)


def erfcinv(y):
    return lib().oracle_erfcinv(float(y))


def event_radius(mean, p, word):
    """Radius drawn by the per-event estimator from the 32-bit Philox word."""
    return lib().oracle_event_radius(float(mean), float(p), int(word) & 0xFFFFFFFF)


def event_axis(mode, theta, phi, word_a, word_b):
    c = np.empty(3)
    lib().oracle_event_axis(int(mode), float(theta), float(phi), int(word_a) & 0xFFFFFFFF,
                            int(word_b) & 0xFFFFFFFF, c.ctypes.data_as(_DP))
    return c


def dsigma_event(model, q, seed, first=0, exp_id=0):
    """Per-event estimates of dSigma/dOmega (1/angstrom) at q [n][3]; row i
    uses the draws of neutron index first + i."""
    prep = model if isinstance(model, Prepared) else Prepared(model)
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1, 3)
    out = np.empty(len(q))
    lib().oracle_dsigma_event_many(ctypes.byref(prep.c), q.ctypes.data_as(_DP), int(seed), int(exp_id),
                                   int(first), len(q), out.ctypes.data_as(_DP))
    return out


def sample_lambda(lambda0, drel, u):
    return lib().oracle_sample_lambda(float(lambda0), float(drel), float(u))


def num_threads():
    return lib().oracle_num_threads()


def model_extent(model):
    """Largest extent of the particle (angstrom) over its polydisperse nodes."""
    prep = model if isinstance(model, Prepared) else Prepared(model)
    return lib().oracle_model_extent(ctypes.byref(prep.c))


def sigma_s(model, lam, lam_min=None):
    """Total scattering cross section per unit volume Sigma_s(lambda) in
    1/angstrom: dSigma/dOmega integrated over all directions for a neutron
    along +z, by the rule built at lam_min (default lam)."""
    prep = model if isinstance(model, Prepared) else Prepared(model)
    return lib().oracle_sigma_s(ctypes.byref(prep.c), float(lam), float(lam if lam_min is None else lam_min))


def sigma_s_panel(model, lam, lam_min, i):
    """The share of |Q| panel i of the rule in Sigma_s(lam) (1/angstrom)."""
    prep = model if isinstance(model, Prepared) else Prepared(model)
    return lib().oracle_sigma_s_panel(ctypes.byref(prep.c), float(lam), float(lam_min), int(i))


def sigma_s_npanels(model, lam_min):
    prep = model if isinstance(model, Prepared) else Prepared(model)
    return lib().oracle_sigma_s_npanels(ctypes.byref(prep.c), float(lam_min))


def _att_model(model):
    m = model if isinstance(model, dict) else model.as_dict()
    return Prepared(dict(m, self_attenuation=1))


def att_table(instrument, model):
    """The trace's attenuation table for the instrument's wavelength band:
    (lambda nodes, mu_s at the nodes in 1/m, Chebyshev coefficients)."""
    lam, mu, c = np.zeros(8), np.zeros(8), np.zeros(8)
    prep = _att_model(model)   # keeps the node arrays alive during the call
    n = lib().oracle_att_table(ctypes.byref(_inst(instrument)), ctypes.byref(prep.c),
                               lam.ctypes.data_as(_DP), mu.ctypes.data_as(_DP), c.ctypes.data_as(_DP))
    return lam[:n], mu[:n], c[:n]


def att_eval(instrument, model, lam):
    """mu_s(lambda) in 1/m from the trace's table at the wavelengths lam."""
    lam = np.ascontiguousarray(np.atleast_1d(lam), dtype=np.float64)
    out = np.empty(len(lam))
    prep = _att_model(model)
    lib().oracle_att_eval(ctypes.byref(_inst(instrument)), ctypes.byref(prep.c),
                          lam.ctypes.data_as(_DP), len(lam), out.ctypes.data_as(_DP))
    return out
