"""The C ABI library (CPU only: no compute call needs a GPU here).

* libsas.so loads and exports every entry point include/sas.h declares;
* the library's host-side tables (its own Gauss-Legendre, Schulz
  generalised Gauss-Laguerre, orientation grid and Percus-Yevick series)
  agree with independent references;
* argument validation rejects bad inputs before touching the GPU.
"""
import math
import os
import re
from fractions import Fraction

import numpy as np
import pytest

import paper_2501_06054_gb300 as sas
import sas_workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "sas.h")).read()
    return sorted(set(re.findall(r"\b(sas_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    L = sas.lib()
    names = _declared()
    assert "sas_trace" in names and "sas_read_detector" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_library_is_the_in_tree_build():
    assert os.path.realpath(sas.library_path()).startswith(os.path.realpath(ROOT))
    assert os.path.exists(sas.library_path())


def test_gauss_legendre_host_table():
    for n in (1, 2, 7, 40, 76, 128):
        x, w = sas.sas_gauss_legendre(n)
        xr, wr = np.polynomial.legendre.leggauss(n)
        assert np.max(np.abs(x - xr)) < 1e-14
        assert np.max(np.abs(w - wr)) < 1e-14


@pytest.mark.parametrize("p,n", [(0.1, 40), (0.3, 40), (0.02, 40), (0.25, 7)])
def test_schulz_host_table(p, n):
    import scipy.special as spc
    rbar = 33.0
    r, w = sas.sas_schulz_nodes(rbar, p, n)
    z = 1 / p ** 2 - 1
    assert abs(w.sum() - 1) < 1e-13
    for k in range(1, 8):
        ref = rbar ** k * math.exp(spc.gammaln(z + 1 + k) - spc.gammaln(z + 1)) / (z + 1) ** k
        assert abs(np.dot(w, r ** k) / ref - 1) < 1e-10
    if z < 200:   # scipy's weights overflow for larger alpha
        xr, wr = spc.roots_genlaguerre(n, z)
        assert np.max(np.abs(r - rbar * xr / (z + 1))) < 1e-9 * rbar
        assert np.max(np.abs(w - wr / wr.sum())) < 1e-12


def test_orientation_host_table_matches_oracle_grid():
    import oracle
    for args in [(0.5 * math.pi, 0.0, math.radians(15), 76, 76, 0),
                 (0.3, 1.2, math.radians(30), 20, 24, 0),
                 (1.0, 2.0, 0.0, 76, 76, 0),
                 (0.2, 0.4, 0.0, 30, 30, 1)]:
        c, w = sas.sas_orientation_nodes(*args)
        co, wo = oracle.orientation_nodes(*args[:5], isotropic=bool(args[5]))
        assert c.shape == co.shape
        assert np.max(np.abs(c - co)) < 1e-13
        assert np.max(np.abs(w - wo)) < 1e-13


def test_py_series_exact_rationals():
    """G(A)/A series coefficients against exact rational arithmetic on the
    Taylor series of sin and cos (Fractions, no floating point)."""
    def fact(k):
        return math.factorial(k)

    def sinc(k):
        return Fraction((-1) ** ((k - 1) // 2), fact(k)) if k % 2 == 1 else Fraction(0)

    def cosc(k):
        return Fraction((-1) ** (k // 2), fact(k)) if k % 2 == 0 and k >= 0 else Fraction(0)

    def coef(poly_terms, k):
        # poly_terms: list of (c, power of A, 'sin'|'cos'|'one')
        s = Fraction(0)
        for c, pw, f in poly_terms:
            kk = k - pw
            if kk < 0:
                continue
            s += c * (sinc(kk) if f == "sin" else cosc(kk) if f == "cos" else Fraction(int(kk == 0)))
        return s

    b1 = [(1, 0, "sin"), (-1, 1, "cos")]
    b2 = [(2, 1, "sin"), (2, 0, "cos"), (-1, 2, "cos"), (-2, 0, "one")]
    b3 = [(-1, 4, "cos"), (12, 2, "cos"), (-24, 0, "cos"), (4, 3, "sin"), (-24, 1, "sin"),
          (24, 0, "one")]
    for phi in (0.05, 0.2, 0.45):
        abg, ser = sas.sas_py_series(phi, 14)
        a, b, g = abg
        d = (1 - phi) ** 4
        assert abs(a - (1 + 2 * phi) ** 2 / d) < 1e-13 * a
        assert abs(b + 6 * phi * (1 + phi / 2) ** 2 / d) < 1e-13 * abs(b)
        assert abs(g - phi * a / 2) < 1e-13 * g
        for m in range(14):
            ref = (a * float(coef(b1, 2 * m + 3)) + b * float(coef(b2, 2 * m + 4))
                   + g * float(coef(b3, 2 * m + 6)))
            assert abs(ser[m] - ref) <= 1e-13 * max(abs(ref), 1e-300) + 1e-300, (phi, m)


def _inst(**kw):
    return sas.make_instrument(W.Instrument(**kw))


@pytest.mark.parametrize("kw", [dict(lambda0=-1.0), dict(nx=0), dict(ny=5000),
                                dict(ap1_z=0.5), dict(sample_thickness=0.0),
                                dict(pixel_x=float("nan")), dict(dlambda_rel=1.5),
                                dict(mu=-1.0), dict(det_distance=1e-4)])
def test_create_experiment_rejects_bad_instrument(kw):
    with pytest.raises(sas.SasError) as e:
        sas.sas_create_experiment(_inst(**kw))
    assert e.value.status == sas.SAS_ERR_ARG
    assert len(sas.sas_last_error()) > 0


def test_null_handles_are_rejected():
    with pytest.raises(sas.SasError) as e:
        sas.sas_trace(None, 10, 1)
    assert e.value.status == sas.SAS_ERR_ARG
    with pytest.raises(sas.SasError):
        sas.sas_set_model(None, W.Model())
    sas.sas_destroy_experiment(None)   # accepted


def test_host_utilities_reject_bad_sizes():
    with pytest.raises(sas.SasError):
        sas.sas_gauss_legendre(0)
    with pytest.raises(sas.SasError):
        sas.sas_schulz_nodes(10.0, 0.1, 65)
    with pytest.raises(sas.SasError):
        sas.sas_orientation_nodes(0, 0, 0.1, 129, 2)


@pytest.mark.parametrize("name", ["sas_instrument", "sas_model_desc", "sas_launch_config",
                                  "sas_batch_config", "sas_surrogate_box"])
def test_struct_layout_matches_binding(name, tmp_path):
    """The ctypes mirror of each public struct has the C header's size and
    field offsets: a small C program compiled against include/sas.h prints
    sizeof and offsetof for every field the binding names (a field missing
    from the header fails the compile)."""
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    st = getattr(sas, name)
    fields = [f[0] for f in st._fields_]
    src = ["#include <stddef.h>", "#include <stdio.h>", '#include "sas.h"', "int main(void) {",
           f'  printf("%zu\\n", sizeof({name}));']
    src += [f'  printf("%zu\\n", offsetof({name}, {f}));' for f in fields]
    src += ["  return 0;", "}"]
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert out[0] == ctypes.sizeof(st), (name, out[0], ctypes.sizeof(st))
    for f, off in zip(fields, out[1:]):
        assert off == getattr(st, f).offset, (name, f, off, getattr(st, f).offset)
