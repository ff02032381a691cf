"""Generates sas_coeffs.h: FP32 coefficients of the device special functions.

Run once (python gen_coeffs.py > sas_coeffs.h); the output is committed.

* sin / cos on [-pi/4, pi/4]: S(t) = (sin r - r) / r^3 and
  C(t) = (cos r - 1) / r^2 as polynomials in t = r^2 (3 and 4 terms), fitted
  toward the minimax absolute error on t in [0, (1.01 pi/4)^2].
* pi/2 and pi/4 split into two FP32 parts (fl(c), fl(c - fl(c))) for the
  FMA form of Cody-Waite argument reduction.
* a(x) = 2 J1(x) / x for 0 <= x <= X1: a polynomial in s = (x / X1)^2, fitted here
  by Chebyshev-node least squares refined with Lawson iterations toward the
  minimax polynomial of the absolute error.
* a(x) for x <= 8 in product form (1 - x^2/j1^2)(1 - x^2/j2^2) h(x^2) with the
  first two zeros j1, j2 of J1 (scipy) and h a degree-8 polynomial in x^2
  fitted like the above (relative error ~1e-8); no square root, no branch
  for the cylinder workloads' arguments, and the zeros are exact factors.
* a(x) for x <= 4 as a plain degree-6 polynomial in x^2 (absolute error
  ~8e-9), the cheapest form for the small arguments of most cylinder terms.
* a(x) for x <= 6 as a degree-7 polynomial in the centred variable
  2 x^2 / 36 - 1 (absolute error ~6e-8).
* the same with the first three zeros for x <= 12 (degree 10 in the centred
  variable 2 x^2/144 - 1), used for the tail nodes of broad size
  distributions.
* x >= X1: the modulus-phase form of J1 (J1 = M cos(theta), Y1 = M sin(theta)),
  with m(u) = M sqrt(pi x / 2) and h(u) = x (theta - x + 3 pi / 4) fitted as
  polynomials in u = (X1 / x)^2; M and theta are computed from scipy's J1, Y1.
* Percus-Yevick: nothing here; its series is built per experiment on the host.
"""
import math
import sys

import numpy as np
import scipy.special as sp

X1 = 4.0


def f32(v):
    return float(np.float32(v))


def split3(c, bits=12):
    parts = []
    rem = c
    for i in range(2):
        e = math.frexp(rem)[1]
        scale = 2.0 ** (bits - e)
        p = math.floor(rem * scale + 0.5) / scale
        parts.append(p)
        rem = rem - p
    parts.append(f32(rem))
    return parts


def lawson_fit(xs, ys, basis, iters=60):
    """Weighted least squares with Lawson's weight update (approaches minimax)."""
    A = np.stack([b(xs) for b in basis], axis=1)
    w = np.ones_like(xs) / len(xs)
    best = None
    for _ in range(iters):
        sw = np.sqrt(w)
        c, *_ = np.linalg.lstsq(A * sw[:, None], ys * sw, rcond=None)
        err = np.abs(A @ c - ys)
        if best is None or err.max() < best[1]:
            best = (c, err.max())
        w = w * err
        w = w / w.sum()
    return best


def fit_small(deg):
    n = 4000
    t = 0.5 * X1 * X1 * (1 - np.cos(np.pi * (np.arange(n) + 0.5) / n))
    x = np.sqrt(t)
    y = np.where(x > 0, 2 * sp.j1(np.maximum(x, 1e-300)) / np.maximum(x, 1e-300), 1.0)
    s = t / (X1 * X1)
    basis = [lambda ss, k=k: ss ** k for k in range(deg + 1)]
    c, e = lawson_fit(s, y, basis)
    return c, e


def mod_phase(x):
    j, y = sp.j1(x), sp.y1(x)
    M = np.hypot(j, y)
    th = np.arctan2(y, j)
    ref = x - 0.75 * np.pi
    th = th + 2 * np.pi * np.round((ref - th) / (2 * np.pi))
    return M, th


def fit_large(deg_m, deg_h):
    n = 4000
    u = 0.5 * (1 - np.cos(np.pi * (np.arange(n) + 0.5) / n))
    u = np.maximum(u, 1e-6)
    x = X1 / np.sqrt(u)
    M, th = mod_phase(x)
    m = M * np.sqrt(np.pi * x / 2)
    h = x * (th - x + 0.75 * np.pi)
    basis_m = [lambda uu, k=k: uu ** k for k in range(deg_m + 1)]
    basis_h = [lambda uu, k=k: uu ** k for k in range(deg_h + 1)]
    cm, em = lawson_fit(u, m, basis_m)
    ch, eh = lawson_fit(u, h, basis_h)
    return cm, em, ch, eh


def fit_trig():
    n = 4000
    tmax = (1.01 * math.pi / 4) ** 2
    t = 0.5 * tmax * (1 - np.cos(np.pi * (np.arange(n) + 0.5) / n))
    r = np.sqrt(t)
    S = np.where(r > 1e-4, (np.sin(r) - r) / np.maximum(r, 1e-300) ** 3, -1 / 6 + t / 120)
    C = np.where(r > 1e-4, (np.cos(r) - 1) / np.maximum(t, 1e-300), -0.5 + t / 24)
    bS = [lambda tt, k=k: tt ** k for k in range(3)]
    bC = [lambda tt, k=k: tt ** k for k in range(4)]
    cS, eS = lawson_fit(t, S, bS)
    cC, eC = lawson_fit(t, C, bC)
    return cS, eS, cC, eC


def fit_product_centered(deg=10, X=12.0, nz=3):
    """As fit_product, in the centred variable v = 2 x^2 / X^2 - 1 (smaller
    coefficients, stable FP32 Horner evaluation)."""
    n = 8000
    s = 0.5 * X * X * (1 - np.cos(np.pi * (np.arange(n) + 0.5) / n))
    x = np.sqrt(s)
    j = sp.jn_zeros(1, max(nz, 1))
    a = np.where(x > 0, 2 * sp.j1(np.maximum(x, 1e-300)) / np.maximum(x, 1e-300), 1.0)
    p = np.prod([(1 - s / j[k] ** 2) for k in range(nz)], axis=0) if nz else np.ones_like(s)
    ok = np.abs(p) > 1e-6
    v = 2 * s / (X * X) - 1
    basis = [lambda vv, k=k: vv ** k for k in range(deg + 1)]
    c, e = lawson_fit(v[ok], (a / p)[ok], basis)
    return list(c), e, [1.0 / jj ** 2 for jj in j], X * X


def fit_product(deg=8, X=8.0, nz=2):
    n = 8000
    s = 0.5 * X * X * (1 - np.cos(np.pi * (np.arange(n) + 0.5) / n))
    x = np.sqrt(s)
    j = sp.jn_zeros(1, max(nz, 1))
    a = np.where(x > 0, 2 * sp.j1(np.maximum(x, 1e-300)) / np.maximum(x, 1e-300), 1.0)
    p = np.prod([(1 - s / j[k] ** 2) for k in range(nz)], axis=0) if nz else np.ones_like(s)
    ok = np.abs(p) > 1e-6
    u = s / (X * X)
    basis = [lambda uu, k=k: uu ** k for k in range(deg + 1)]
    c, e = lawson_fit(u[ok], (a / p)[ok], basis)
    cs = [ci / (X * X) ** k for k, ci in enumerate(c)]   # coefficients in s = x^2
    if nz == 2:
        return cs, e, 1.0 / j[0] ** 2, 1.0 / j[1] ** 2, X * X
    if nz == 0:
        return cs, e, X * X
    return cs, e, [1.0 / jj ** 2 for jj in j], X * X


def split2(c):
    hi = f32(c)
    return [hi, f32(c - hi)]


def main():
    out = sys.stdout
    cs, es = fit_small(7)
    cm, em, ch, eh = fit_large(5, 5)
    cS, eS, cC, eC = fit_trig()
    cP, eP, iz1, iz2, smax = fit_product()
    cQ, eQ, izq, smaxq = fit_product_centered(deg=10, X=12.0, nz=3)
    cR, eR, smaxr = fit_product(deg=6, X=4.0, nz=0)
    cV, eV, _, smaxv = fit_product_centered(deg=7, X=6.0, nz=0)
    p2 = split2(math.pi / 2)
    p4 = split2(math.pi / 4)
    w = out.write
    w("/* Generated by gen_coeffs.py -- FP32 coefficients of the device special\n")
    w(" * functions (own fits, see the generator's docstring). Do not edit. */\n")
    w("#pragma once\n\n")
    w(f"#define SAS_J1_X1 {X1!r}f\n")
    w(f"/* fit errors (FP64): small {es:.3e}, modulus {em:.3e}, phase {eh:.3e}, "
      f"S {eS:.3e}, C {eC:.3e} */\n")
    w("#define SAS_PIO2_1 %.9ef\n#define SAS_PIO2_2 %.9ef\n" % tuple(p2))
    w("#define SAS_PIO4_1 %.9ef\n#define SAS_PIO4_2 %.9ef\n" % tuple(p4))
    w(f"/* 2 J1(x)/x = (1 - s z1)(1 - s z2) h(s), s = x^2 <= {smax:g}; fit error of h {eP:.3e} */\n")
    w("#define SAS_J1P_SMAX %.9ef\n#define SAS_J1P_Z1 %.9ef\n#define SAS_J1P_Z2 %.9ef\n" % (smax, iz1, iz2))
    w(f"#define SAS_J1P_C_N {len(cP)}\n")
    w("#define SAS_J1P_C {" + ", ".join("%.9ef" % v for v in cP) + "}\n")
    w(f"/* 2 J1(x)/x = (1 - s z1)(1 - s z2)(1 - s z3) g(2 s / {smaxq:g} - 1), s <= {smaxq:g}; fit error of g {eQ:.3e} */\n")
    w("#define SAS_J1Q_SMAX %.9ef\n#define SAS_J1Q_Z1 %.9ef\n#define SAS_J1Q_Z2 %.9ef\n#define SAS_J1Q_Z3 %.9ef\n"
      % (smaxq, izq[0], izq[1], izq[2]))
    w(f"#define SAS_J1Q_C_N {len(cQ)}\n")
    w("#define SAS_J1Q_C {" + ", ".join("%.9ef" % v for v in cQ) + "}\n")
    w(f"/* 2 J1(x)/x = r(s), s = x^2 <= {smaxr:g}; fit error {eR:.3e} */\n")
    w("#define SAS_J1R_SMAX %.9ef\n" % smaxr)
    w(f"#define SAS_J1R_C_N {len(cR)}\n")
    w("#define SAS_J1R_C {" + ", ".join("%.9ef" % v for v in cR) + "}\n")
    w(f"/* 2 J1(x)/x = v(2 s / {smaxv:g} - 1), s = x^2 <= {smaxv:g}; fit error {eV:.3e} */\n")
    w("#define SAS_J1V_SMAX %.9ef\n" % smaxv)
    w(f"#define SAS_J1V_C_N {len(cV)}\n")
    w("#define SAS_J1V_C {" + ", ".join("%.9ef" % v for v in cV) + "}\n")
    w("/* sin r = r + r^3 S(r^2), cos r = 1 + r^2 C(r^2) */\n")
    for name, arr in (("SAS_SIN_C", list(cS)), ("SAS_COS_C", list(cC)), ("SAS_J1S_C", list(cs)),
                      ("SAS_J1M_C", list(cm)), ("SAS_J1H_C", list(ch))):
        w(f"#define {name}_N {len(arr)}\n")
        w(f"#define {name} {{" + ", ".join("%.9ef" % v for v in arr) + "}\n")


if __name__ == "__main__":
    main()
