"""The FP32 special functions of the trace kernels, compiled for the host.

`csrc/sas_math.cuh` uses only IEEE primitives (fmaf, multiply, add, bit
moves), so the same source compiled by g++ gives the device's arithmetic
(up to the device compiler's contraction of a separate multiply and add
into one FMA). Checked here against scipy in FP64:

* 2 J1(x)/x in its forms: the degree-6 polynomial for x <= 4, the centred
  degree-7 polynomial for x <= 6, the product form with two zeros for
  x <= 8, the three-zero form for x <= 12, and the modulus-phase form
  beyond;
* sin / cos after the two-part reduction;
* the sphere amplitude g(x) = (sin x - x cos x) / x^3.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

sp = pytest.importorskip("scipy.special")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2501_06054_gb300", "csrc")

SRC = r"""
#include "sas_math.cuh"
extern "C" {
void cyl_a_r(const float* s, float* o, int n) { for (int i = 0; i < n; ++i) o[i] = sas_cyl_a_r(s[i]); }
void cyl_a_s(const float* s, float* o, int n) { for (int i = 0; i < n; ++i) o[i] = sas_cyl_a_s(s[i]); }
void cyl_a_v(const float* s, float* o, int n) { for (int i = 0; i < n; ++i) o[i] = sas_cyl_a_v(s[i]); }
void cyl_a_s3(const float* s, float* o, int n) { for (int i = 0; i < n; ++i) o[i] = sas_cyl_a_s3(s[i]); }
void cyl_a(const float* x, float* o, int n)
{
    for (int i = 0; i < n; ++i) o[i] = sas_cyl_a(x[i], 1.0f / x[i], 1.0f / sqrtf(x[i]));
}
void sincos_(const float* x, float* s, float* c, int n) { for (int i = 0; i < n; ++i) sas_sincosf(x[i], s[i], c[i]); }
void sphere_g(const float* x, float* o, int n) { for (int i = 0; i < n; ++i) o[i] = sas_sphere_g(x[i], 1.0f / x[i]); }
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    d = tmp_path_factory.mktemp("fp32host")
    src = d / "m.cpp"
    src.write_text(SRC)
    so = d / "m.so"
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-I", CSRC,
                    str(src), "-o", str(so)], check=True)
    L = ctypes.CDLL(str(so))
    return L


def _call(L, name, x, outs=1):
    x = np.ascontiguousarray(x, dtype=np.float32)
    o = [np.empty_like(x) for _ in range(outs)]
    fp = ctypes.POINTER(ctypes.c_float)
    getattr(L, name)(x.ctypes.data_as(fp), *[v.ctypes.data_as(fp) for v in o], ctypes.c_int(len(x)))
    return o[0] if outs == 1 else o


def _a(x):
    x = np.asarray(x, dtype=np.float64)
    return np.where(x > 0, 2 * sp.j1(np.maximum(x, 1e-300)) / np.maximum(x, 1e-300), 1.0)


@pytest.mark.parametrize("name,xmax,tol", [("cyl_a_r", 4.0, 4e-7), ("cyl_a_v", 6.0, 4e-7),
                                           ("cyl_a_s", 8.0, 4e-7), ("cyl_a_s3", 12.0, 4e-7)])
def test_j1_polynomial_forms(lib, name, xmax, tol):
    x = np.linspace(0.0, xmax, 20001).astype(np.float32)
    s = (x * x).astype(np.float32)
    got = _call(lib, name, s).astype(np.float64)
    ref = _a(np.sqrt(s.astype(np.float64)))
    assert np.max(np.abs(got - ref)) < tol


def test_j1_full_range(lib):
    x = np.concatenate([np.linspace(0.01, 4.0, 5000), np.linspace(4.0, 400.0, 20000)]).astype(np.float32)
    got = _call(lib, "cyl_a", x).astype(np.float64)
    ref = _a(x.astype(np.float64))
    # absolute, relative to a(0) = 1; the amplitude decays like x^-3/2
    assert np.max(np.abs(got - ref)) < 5e-7


def test_sincos_and_sphere_amplitude(lib):
    x = np.linspace(0.0, 200.0, 40001).astype(np.float32)
    s, c = _call(lib, "sincos_", x, outs=2)
    xd = x.astype(np.float64)
    assert np.max(np.abs(s - np.sin(xd))) < 2e-7 * max(1.0, 1.0)
    assert np.max(np.abs(c - np.cos(xd))) < 2e-7
    xs = x[1:]
    g = _call(lib, "sphere_g", xs).astype(np.float64)
    xd = xs.astype(np.float64)
    ref = (np.sin(xd) - xd * np.cos(xd)) / xd ** 3
    # relative to g(0) = 1/3, scaled by the amplitude's 1/x^2 envelope beyond x = 1
    env = np.minimum(1.0 / 3.0, 1.0 / np.maximum(xd, 1.0) ** 2)
    assert np.max(np.abs(g - ref) / env) < 2e-6
