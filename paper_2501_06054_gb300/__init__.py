"""Python binding of libsas, the GB300 SANS Monte Carlo trace library.

Argument marshalling only (ctypes): every step of the trace runs in the
library's CUDA kernels. The functions carry the C ABI's names (include/sas.h);
device buffers are passed as torch CUDA tensors (or raw integer addresses),
host buffers as numpy arrays owned by the caller.

If the compiled library is missing and cannot be built, importing the
library raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

SAS_OK, SAS_ERR_ARG, SAS_ERR_CUDA, SAS_ERR_OOM, SAS_ERR_STATE = 0, 1, 2, 3, 4
SAS_ERR_TIMEOUT, SAS_ERR_OUT_OF_BOX, SAS_ERR_NUMERIC = 5, 6, 7
SAS_SPHERE, SAS_CORE_SHELL, SAS_CYLINDER, SAS_ELLIPSOID = 0, 1, 2, 3
SAS_SQ_NONE, SAS_SQ_HARD_SPHERE_PY = 0, 1
SAS_FP32, SAS_FP64 = 0, 1


class SasError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libsas error {status}: {msg}")
        self.status = status


class sas_instrument(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "lambda0", "dlambda_rel", "ap1_radius", "ap1_z", "ap2_radius", "ap2_z",
        "sample_half_x", "sample_half_y", "sample_thickness", "mu", "det_distance",
        "pixel_x", "pixel_y")] + [("nx", ctypes.c_int64), ("ny", ctypes.c_int64)]


class sas_model_desc(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "kind", "sq_kind", "precision", "n_poly", "n_gamma", "n_psi", "isotropic")] + \
               [(n, ctypes.c_double) for n in (
                   "radius", "thickness", "length", "radius_polar", "sld", "sld_shell",
                   "sld_solvent", "volume_fraction", "poly", "sigma_orient", "axis_theta",
                   "axis_phi", "sq_radius", "sq_fraction")] + \
               [(n, ctypes.c_int64) for n in ("sampling", "poly_dist", "radial_table")] + \
               [("radius_b", ctypes.c_double), ("axis_psi", ctypes.c_double), ("n_rot", ctypes.c_int64),
                ("self_attenuation", ctypes.c_int64), ("n_cap", ctypes.c_int64),
                ("thickness_face", ctypes.c_double), ("sld_face", ctypes.c_double),
                ("function", ctypes.c_int64)] + \
               [(n, ctypes.c_double) for n in ("f_scale", "f_p0", "f_p1", "f_p2", "sq_charge",
                                               "sq_temperature", "sq_salt", "sq_dielectric", "fuzziness")]


class sas_launch_config(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in (
        "block", "tally", "agg", "ctas_per_sm", "stage_orient", "order_q")]


class sas_batch_config(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("use_hist", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("target_item_flop", ctypes.c_double)]


class sas_surrogate_box(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "q_max", "r_min", "r_max", "l_min", "l_max", "sigma_orient_min", "sigma_orient_max",
        "poly_min", "poly_max")] + [(n, ctypes.c_int32) for n in (
            "n_poly", "n_gamma", "n_psi", "n_buckets", "n_fourier", "model")]


_lib = None
_lock = threading.Lock()
_vp = ctypes.c_void_p
_u64 = ctypes.c_uint64
_dp = ctypes.POINTER(ctypes.c_double)

_SIGS = {
    "sas_create_experiment": [ctypes.POINTER(sas_instrument), _vp, ctypes.POINTER(_vp)],
    "sas_set_model": [_vp, ctypes.POINTER(sas_model_desc)],
    "sas_set_experiment_id": [_vp, ctypes.c_uint32],
    "sas_set_stream": [_vp, _vp],
    "sas_trace": [_vp, _u64, _u64],
    "sas_trace_range": [_vp, _u64, _u64, _u64],
    "sas_reset_detector": [_vp],
    "sas_read_detector": [_vp, _vp, _vp, _vp, ctypes.c_size_t, _vp],
    "sas_detector_device": [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                            ctypes.POINTER(_vp)],
    "sas_eval_model": [_vp, _vp, ctypes.c_size_t, _vp],
    "sas_trace_records": [_vp, _u64, _u64, _u64, _vp, _vp],
    "sas_attenuation_table": [_vp, ctypes.POINTER(ctypes.c_int), _dp, _dp, _dp, _dp],
    "sas_total_cross_section": [_vp, ctypes.c_double, _dp, _dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
    "sas_sync": [_vp],
    "sas_destroy_experiment": [_vp],
    "sas_device_info": [ctypes.POINTER(ctypes.c_int)] * 4,
    "sas_gauss_legendre": [ctypes.c_int, _dp, _dp],
    "sas_schulz_nodes": [ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp, _dp],
    "sas_orientation_nodes": [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                              ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.POINTER(ctypes.c_int)],
    "sas_py_series": [ctypes.c_double, _dp, _dp, ctypes.c_int],
    "sas_cylinder_radial_table": [_dp, _dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                  _dp, _dp, _dp],
    "sas_hayter_msa_table": [ctypes.c_double] * 7 + [ctypes.c_int, _dp, _dp, ctypes.POINTER(ctypes.c_int),
                                                      _dp, _dp, _dp, _dp],
    "sas_get_launch_config": [_vp, ctypes.POINTER(sas_launch_config)],
    "sas_set_launch_config": [_vp, ctypes.POINTER(sas_launch_config)],
    "sas_autotune": [_vp, _u64, _u64, ctypes.POINTER(sas_launch_config), _dp],
    "sas_create_batch": [_vp, _vp, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(_vp)],
    "sas_trace_batch": [_vp, _u64],
    "sas_read_batch_detector": [_vp, ctypes.c_size_t, _vp, _vp, _vp, ctypes.c_size_t, _vp],
    "sas_batch_detector_device": [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                  ctypes.POINTER(_vp), ctypes.POINTER(_vp)],
    "sas_batch_set_config": [_vp, ctypes.POINTER(sas_batch_config)],
    "sas_batch_get_config": [_vp, ctypes.POINTER(sas_batch_config)],
    "sas_batch_info": [_vp, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_int),
                       ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_uint64)],
    "sas_batch_autotune": [_vp, _u64, ctypes.POINTER(sas_batch_config), _dp],
    "sas_destroy_batch": [_vp],
    "sas_create_surrogate": [ctypes.POINTER(sas_surrogate_box), _u64, _vp, ctypes.POINTER(_vp)],
    "sas_surrogate_generate": [_vp, _u64, _u64],
    "sas_surrogate_dataset": [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_u64)],
    "sas_surrogate_exact": [_vp, _vp, ctypes.c_size_t, _vp],
    "sas_surrogate_eval": [_vp, _vp, ctypes.c_size_t, _vp],
    "sas_surrogate_grad": [_vp, _vp, _vp, ctypes.c_uint32, _vp, ctypes.c_size_t],
    "sas_surrogate_train": [_vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double, ctypes.c_uint32],
    "sas_surrogate_get_params": [_vp, _vp, ctypes.c_size_t],
    "sas_surrogate_set_params": [_vp, _vp, ctypes.c_size_t],
    "sas_surrogate_info": [_vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_uint32)],
    "sas_surrogate_test_stall": [_vp, _u64],
    "sas_destroy_surrogate": [_vp],
    "sas_attach_surrogate": [_vp, _vp],
    "sas_batch_attach_surrogate": [_vp, _vp],
    "sas_surrogate_fallbacks": [_vp, _vp, ctypes.POINTER(_u64)],
    "sas_batch_surrogate_share": [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64)],
    "sas_trace_batch_static": [_vp, _vp, _vp, ctypes.c_size_t, _u64, _vp, _vp, _vp, _vp, _vp],
}

# extra entry points added by later modules of the library register here
EXTRA_SIGS = {}


def library_path():
    return _build.LIB


def lib():
    """Load libsas.so (building it in-tree first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path, mode=ctypes.RTLD_GLOBAL)
            for name, args in {**_SIGS, **EXTRA_SIGS}.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = ctypes.c_int
            L.sas_last_error.restype = ctypes.c_char_p
            L.sas_last_error.argtypes = []
            _lib = L
    return _lib


def sas_last_error() -> str:
    return lib().sas_last_error().decode()


def _check(status):
    if status != SAS_OK:
        raise SasError(status, sas_last_error())


def _ptr(x):
    """Device (or host) address of a torch tensor, numpy array or integer."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_instrument(d) -> sas_instrument:
    d = d if isinstance(d, dict) else d.as_dict()
    return sas_instrument(**{k: (int(v) if k in ("nx", "ny") else float(v)) for k, v in d.items()})


def make_model(d) -> sas_model_desc:
    d = d if isinstance(d, dict) else d.as_dict()
    ints = ("kind", "sq_kind", "precision", "n_poly", "n_gamma", "n_psi", "isotropic", "sampling",
            "poly_dist", "radial_table", "n_rot", "self_attenuation", "n_cap", "function")
    return sas_model_desc(**{k: (int(v) if k in ints else float(v)) for k, v in d.items()})


# ------------------------------------------------------------ C ABI names

def sas_create_experiment(instrument, stream=None):
    inst = instrument if isinstance(instrument, sas_instrument) else make_instrument(instrument)
    h = _vp()
    _check(lib().sas_create_experiment(ctypes.byref(inst), _stream_handle(stream), ctypes.byref(h)))
    return h.value


def sas_set_model(exp, model):
    m = model if isinstance(model, sas_model_desc) else make_model(model)
    _check(lib().sas_set_model(exp, ctypes.byref(m)))


def sas_set_experiment_id(exp, exp_id):
    _check(lib().sas_set_experiment_id(exp, int(exp_id)))


def sas_set_stream(exp, stream):
    _check(lib().sas_set_stream(exp, _stream_handle(stream)))


def sas_trace(exp, n_neutrons, seed):
    _check(lib().sas_trace(exp, int(n_neutrons), int(seed)))


def sas_trace_range(exp, first, n, seed):
    _check(lib().sas_trace_range(exp, int(first), int(n), int(seed)))


def sas_reset_detector(exp):
    _check(lib().sas_reset_detector(exp))


def sas_read_detector(exp, n_pixels, sum_w=None, sum_w2=None, count=None, transmitted=True):
    """Copy the detector to host numpy buffers (allocated here if not given)."""
    sum_w = np.empty(n_pixels, np.float64) if sum_w is None else sum_w
    sum_w2 = np.empty(n_pixels, np.float64) if sum_w2 is None else sum_w2
    count = np.empty(n_pixels, np.uint64) if count is None else count
    tr = np.zeros(1, np.float64)
    _check(lib().sas_read_detector(exp, _ptr(sum_w), _ptr(sum_w2), _ptr(count), int(n_pixels),
                                   _ptr(tr) if transmitted else None))
    return dict(sum_w=sum_w, sum_w2=sum_w2, count=count, trans=float(tr[0]))


def sas_detector_device(exp):
    a, b, c, d = _vp(), _vp(), _vp(), _vp()
    _check(lib().sas_detector_device(exp, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                     ctypes.byref(d)))
    return a.value, b.value, c.value, d.value


def sas_eval_model(exp, q_xyz, n, out):
    _check(lib().sas_eval_model(exp, _ptr(q_xyz), int(n), _ptr(out)))


def sas_trace_records(exp, first, n, seed, pixel, weight):
    _check(lib().sas_trace_records(exp, int(first), int(n), int(seed), _ptr(pixel), _ptr(weight)))


def sas_attenuation_table(exp):
    """The experiment's self-attenuation table: dict(lam, mu_s (1/m), coef,
    lmin, lmax) with n points (n = 0: off)."""
    n = ctypes.c_int()
    lam, mu, c, lr = np.zeros(8), np.zeros(8), np.zeros(8), np.zeros(2)
    _check(lib().sas_attenuation_table(exp, ctypes.byref(n), lam.ctypes.data_as(_dp), mu.ctypes.data_as(_dp),
                                       c.ctypes.data_as(_dp), lr.ctypes.data_as(_dp)))
    k = n.value
    return dict(lam=lam[:k], mu_s=mu[:k], coef=c[:k], lmin=float(lr[0]), lmax=float(lr[1]))


def sas_total_cross_section(exp, lam, max_panels=4096):
    """(Sigma_s(lam) in 1/angstrom, per-panel shares) of the experiment's model."""
    sig = np.zeros(1)
    n = ctypes.c_int()
    part = np.zeros(max_panels)
    _check(lib().sas_total_cross_section(exp, float(lam), sig.ctypes.data_as(_dp), part.ctypes.data_as(_dp),
                                         int(max_panels), ctypes.byref(n)))
    return float(sig[0]), part[:min(n.value, max_panels)]


def sas_sync(exp):
    _check(lib().sas_sync(exp))


def sas_destroy_experiment(exp):
    _check(lib().sas_destroy_experiment(exp))


def sas_device_info():
    v = [ctypes.c_int() for _ in range(4)]
    _check(lib().sas_device_info(*[ctypes.byref(x) for x in v]))
    return dict(sm_count=v[0].value, smem_optin=v[1].value, cc=(v[2].value, v[3].value))


def sas_gauss_legendre(n):
    x, w = np.empty(n), np.empty(n)
    _check(lib().sas_gauss_legendre(int(n), x.ctypes.data_as(_dp), w.ctypes.data_as(_dp)))
    return x, w


def sas_cylinder_radial_table(r, w, rbar, xmax, n_points):
    """(G, D, max_err) of the cylinder radial table on the host."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    G, D, err = np.empty(n_points), np.empty(n_points), np.zeros(1)
    _check(lib().sas_cylinder_radial_table(r.ctypes.data_as(_dp), w.ctypes.data_as(_dp), len(r), float(rbar),
                                           float(xmax), int(n_points), G.ctypes.data_as(_dp),
                                           D.ctypes.data_as(_dp), err.ctypes.data_as(_dp)))
    return G, D, float(err[0])


def sas_hayter_msa_table(radius_eff, fraction, charge, temperature, salt, dielectric, q_max, n_max=65536):
    """The library's Hayter-Penfold S(Q) table on the host: dict with dq,
    S, dS_dQ (arrays), s_rescale, contact, gamma_c, kappa."""
    sd = np.empty(2 * n_max)
    dq, sr, ct, gc, ka = (np.zeros(1) for _ in range(5))
    n = ctypes.c_int(0)
    _check(lib().sas_hayter_msa_table(float(radius_eff), float(fraction), float(charge), float(temperature),
                                      float(salt), float(dielectric), float(q_max), int(n_max),
                                      dq.ctypes.data_as(_dp), sd.ctypes.data_as(_dp), ctypes.byref(n),
                                      sr.ctypes.data_as(_dp), ct.ctypes.data_as(_dp), gc.ctypes.data_as(_dp),
                                      ka.ctypes.data_as(_dp)))
    k = n.value
    return dict(dq=float(dq[0]), S=sd[0:2 * k:2].copy(), dS_dQ=sd[1:2 * k:2].copy(), s_rescale=float(sr[0]),
                contact=float(ct[0]), gamma_c=float(gc[0]), kappa=float(ka[0]))


def sas_schulz_nodes(mean, p, n):
    r, w = np.empty(n), np.empty(n)
    _check(lib().sas_schulz_nodes(float(mean), float(p), int(n), r.ctypes.data_as(_dp),
                                  w.ctypes.data_as(_dp)))
    k = 1 if (p <= 0.0 or n <= 1) else n
    return r[:k], w[:k]


def sas_orientation_nodes(theta, phi, sigma, n_gamma, n_psi, isotropic=0):
    c = np.empty((n_gamma * n_psi, 3))
    w = np.empty(n_gamma * n_psi)
    k = ctypes.c_int()
    _check(lib().sas_orientation_nodes(float(theta), float(phi), float(sigma), int(n_gamma),
                                       int(n_psi), int(isotropic), c.ctypes.data_as(_dp),
                                       w.ctypes.data_as(_dp), ctypes.byref(k)))
    return c[:k.value], w[:k.value]


def sas_py_series(phi, nser=14):
    abg = np.empty(3)
    s = np.empty(nser)
    _check(lib().sas_py_series(float(phi), abg.ctypes.data_as(_dp), s.ctypes.data_as(_dp),
                               int(nser)))
    return abg, s


def sas_get_launch_config(exp):
    c = sas_launch_config()
    _check(lib().sas_get_launch_config(exp, ctypes.byref(c)))
    return c


def sas_set_launch_config(exp, cfg):
    _check(lib().sas_set_launch_config(exp, ctypes.byref(cfg)))


def sas_autotune(exp, n_sample, seed):
    c = sas_launch_config()
    ms = ctypes.c_double()
    _check(lib().sas_autotune(exp, int(n_sample), int(seed), ctypes.byref(c), ctypes.byref(ms)))
    return c, ms.value


def sas_create_batch(instrument, models, counts, stream=None):
    inst = instrument if isinstance(instrument, sas_instrument) else make_instrument(instrument)
    arr = (sas_model_desc * len(models))(*[m if isinstance(m, sas_model_desc) else make_model(m)
                                           for m in models])
    cnt = np.ascontiguousarray(np.asarray(counts, dtype=np.uint64))
    h = _vp()
    _check(lib().sas_create_batch(ctypes.byref(inst), ctypes.cast(arr, _vp), cnt.ctypes.data,
                                  len(models), _stream_handle(stream), ctypes.byref(h)))
    return h.value


def sas_trace_batch(batch, seed):
    _check(lib().sas_trace_batch(batch, int(seed)))


def sas_read_batch_detector(batch, exp, n_pixels):
    sw = np.empty(n_pixels, np.float64)
    sw2 = np.empty(n_pixels, np.float64)
    cnt = np.empty(n_pixels, np.uint64)
    tr = np.zeros(1, np.float64)
    _check(lib().sas_read_batch_detector(batch, int(exp), sw.ctypes.data, sw2.ctypes.data,
                                         cnt.ctypes.data, int(n_pixels), tr.ctypes.data))
    return dict(sum_w=sw, sum_w2=sw2, count=cnt, trans=float(tr[0]))


def sas_batch_detector_device(batch):
    a, b, c, d = _vp(), _vp(), _vp(), _vp()
    _check(lib().sas_batch_detector_device(batch, ctypes.byref(a), ctypes.byref(b),
                                           ctypes.byref(c), ctypes.byref(d)))
    return a.value, b.value, c.value, d.value


def sas_batch_set_config(batch, cfg):
    _check(lib().sas_batch_set_config(batch, ctypes.byref(cfg)))


def sas_batch_get_config(batch):
    c = sas_batch_config()
    _check(lib().sas_batch_get_config(batch, ctypes.byref(c)))
    return c


def sas_batch_info(batch):
    n, g, sm, tot = ctypes.c_uint32(), ctypes.c_int(), ctypes.c_size_t(), ctypes.c_uint64()
    _check(lib().sas_batch_info(batch, ctypes.byref(n), ctypes.byref(g), ctypes.byref(sm),
                                ctypes.byref(tot)))
    return dict(n_items=n.value, grid=g.value, smem=sm.value, total_histories=tot.value)


def sas_batch_autotune(batch, seed):
    c = sas_batch_config()
    ms = ctypes.c_double()
    _check(lib().sas_batch_autotune(batch, int(seed), ctypes.byref(c), ctypes.byref(ms)))
    return c, ms.value


def sas_destroy_batch(batch):
    _check(lib().sas_destroy_batch(batch))


def sas_trace_batch_static(instrument, models, counts, seed, sum_w, sum_w2, count, transmitted,
                           stream=None):
    """Batched trace without device allocation: outputs are caller-owned
    device buffers ([n_exp][nx*ny] and [n_exp])."""
    inst = instrument if isinstance(instrument, sas_instrument) else make_instrument(instrument)
    arr = (sas_model_desc * len(models))(*[m if isinstance(m, sas_model_desc) else make_model(m)
                                           for m in models])
    cnt = np.ascontiguousarray(np.asarray(counts, dtype=np.uint64))
    _check(lib().sas_trace_batch_static(ctypes.byref(inst), ctypes.cast(arr, _vp), cnt.ctypes.data,
                                        len(models), int(seed), _ptr(sum_w), _ptr(sum_w2),
                                        _ptr(count), _ptr(transmitted), _stream_handle(stream)))


def make_box(d) -> sas_surrogate_box:
    ints = ("n_poly", "n_gamma", "n_psi", "n_buckets", "n_fourier", "model")
    return sas_surrogate_box(**{k: (int(v) if k in ints else float(v)) for k, v in d.items()})


def sas_create_surrogate(box, seed, stream=None):
    b = box if isinstance(box, sas_surrogate_box) else make_box(box)
    h = _vp()
    _check(lib().sas_create_surrogate(ctypes.byref(b), int(seed), _stream_handle(stream),
                                      ctypes.byref(h)))
    return h.value


def sas_surrogate_generate(s, n, seed):
    _check(lib().sas_surrogate_generate(s, int(n), int(seed)))


def sas_surrogate_dataset(s):
    r, y, n = _vp(), _vp(), _u64()
    _check(lib().sas_surrogate_dataset(s, ctypes.byref(r), ctypes.byref(y), ctypes.byref(n)))
    return r.value, y.value, n.value


def sas_surrogate_exact(s, raw, n, log_p):
    _check(lib().sas_surrogate_exact(s, _ptr(raw), int(n), _ptr(log_p)))


def sas_surrogate_eval(s, raw, n, log_p):
    _check(lib().sas_surrogate_eval(s, _ptr(raw), int(n), _ptr(log_p)))


def sas_surrogate_grad(s, raw, log_p, n, n_params):
    g = np.empty(n_params, np.float32)
    _check(lib().sas_surrogate_grad(s, _ptr(raw), _ptr(log_p), int(n), g.ctypes.data, n_params))
    return g


def sas_surrogate_train(s, n_steps, batch, lr, total_steps):
    _check(lib().sas_surrogate_train(s, int(n_steps), int(batch), float(lr), int(total_steps)))


def sas_surrogate_test_stall(s, wait_ns):
    _check(lib().sas_surrogate_test_stall(s, int(wait_ns)))


def sas_surrogate_info(s):
    n, st = ctypes.c_size_t(), ctypes.c_uint32()
    _check(lib().sas_surrogate_info(s, ctypes.byref(n), ctypes.byref(st)))
    return dict(n_params=n.value, steps_done=st.value)


def sas_surrogate_get_params(s, n_params):
    p = np.empty(n_params, np.float32)
    _check(lib().sas_surrogate_get_params(s, p.ctypes.data, n_params))
    return p


def sas_surrogate_set_params(s, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(lib().sas_surrogate_set_params(s, p.ctypes.data, p.size))


def sas_destroy_surrogate(s):
    _check(lib().sas_destroy_surrogate(s))


def sas_attach_surrogate(exp, s):
    _check(lib().sas_attach_surrogate(exp, s))


def sas_batch_attach_surrogate(batch, s):
    _check(lib().sas_batch_attach_surrogate(batch, s))


def sas_batch_surrogate_share(batch):
    """(experiments, histories) of the batch that the attached surrogate covers."""
    e, h = _u64(), _u64()
    _check(lib().sas_batch_surrogate_share(batch, ctypes.byref(e), ctypes.byref(h)))
    return int(e.value), int(h.value)


def sas_surrogate_fallbacks(exp=None, batch=None):
    c = _u64()
    _check(lib().sas_surrogate_fallbacks(exp, batch, ctypes.byref(c)))
    return c.value


# ------------------------------------------------------------ convenience

class Experiment:
    """Owns one sas_experiment handle (thin wrapper over the C ABI)."""

    def __init__(self, instrument, model=None, stream=None):
        self.inst = instrument if isinstance(instrument, sas_instrument) else make_instrument(instrument)
        self.npix = int(self.inst.nx * self.inst.ny)
        self.h = sas_create_experiment(self.inst, stream)
        if model is not None:
            self.set_model(model)

    def set_model(self, model):
        sas_set_model(self.h, model)

    def trace(self, n, seed):
        sas_trace(self.h, n, seed)

    def trace_range(self, first, n, seed):
        sas_trace_range(self.h, first, n, seed)

    def read(self):
        d = sas_read_detector(self.h, self.npix)
        shp = (int(self.inst.ny), int(self.inst.nx))
        for k in ("sum_w", "sum_w2", "count"):
            d[k] = d[k].reshape(shp)
        return d

    def sync(self):
        sas_sync(self.h)

    def close(self):
        if self.h:
            sas_destroy_experiment(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
