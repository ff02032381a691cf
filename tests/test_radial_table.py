"""The cylinder radial table (host side, CPU): values against scipy, the
derivative column against scipy's J2, the reported interpolation error
against a direct check of the cubic Hermite interpolant.

G(x) = sum_i w_i t_i^4 a(x t_i)^2, a(y) = 2 J1(y)/y, t_i = r_i / rbar; it
replaces the polydisperse radial sum of the cylinder average (Eq. 8 with
the Schulz or Gaussian radius law) when radial_table = 1.
"""
import numpy as np
import pytest

import oracle
import paper_2501_06054_gb300 as sas

sp = pytest.importorskip("scipy.special")


def _a(y):
    y = np.maximum(np.asarray(y, dtype=np.float64), 1e-300)
    return np.where(y < 1e-8, 1.0, 2.0 * sp.j1(y) / y)


def _G(x, r, w, rbar):
    t = r / rbar
    return np.array([np.sum(w * t ** 4 * _a(xx * t) ** 2) for xx in np.atleast_1d(x)])


def _dG(x, r, w, rbar):
    t = r / rbar
    out = []
    for xx in np.atleast_1d(x):
        y = np.maximum(xx * t, 1e-300)
        da = np.where(y < 1e-8, -y / 4.0, -2.0 * sp.jv(2, y) / y)
        out.append(np.sum(w * t ** 4 * 2.0 * _a(y) * da * t))
    return np.array(out)


@pytest.mark.parametrize("law,p,n", [("schulz", 0.1, 40), ("gauss", 0.3, 48), ("schulz", 0.0, 1)])
def test_radial_table_values_derivatives_and_error(law, p, n):
    rbar = 20.0
    r, w = (oracle.schulz_nodes if law == "schulz" else oracle.gaussian_nodes)(rbar, p, n)
    xmax, npts = 0.3 * rbar, 1025
    G, D, err = sas.sas_cylinder_radial_table(r, w, rbar, xmax, npts)
    x = np.linspace(0.0, xmax, npts)
    h = x[1]
    assert np.allclose(G, _G(x, r, w, rbar), rtol=0, atol=1e-13 * G[0])
    assert np.allclose(D, h * _dG(x, r, w, rbar), rtol=0, atol=1e-12 * G[0])
    assert G[0] == pytest.approx(np.sum(w * (r / rbar) ** 4), rel=1e-14)
    # the reported error is the cubic Hermite error at the midpoints
    xm = x[:-1] + 0.5 * h
    herm = 0.5 * (G[:-1] + G[1:]) + 0.125 * (D[:-1] - D[1:])
    direct = np.max(np.abs(herm - _G(xm, r, w, rbar)))
    assert err == pytest.approx(direct, rel=1e-3, abs=1e-15)   # a difference of O(1) values
    assert err < 1e-9 * G[0]
    # and at arbitrary points the interpolant stays within a few midpoint errors
    rng = np.random.default_rng(1)
    xs = rng.uniform(0, xmax * 0.999, 400)
    s = xs / h
    i = np.minimum(s.astype(int), npts - 2)
    f = s - i
    f1 = 1 - f
    hv = f1 * f1 * ((2 * f + 1) * G[i] + f * D[i]) + f * f * ((3 - 2 * f) * G[i + 1] - f1 * D[i + 1])
    assert np.max(np.abs(hv - _G(xs, r, w, rbar))) <= 4 * err + 1e-15


def test_radial_table_refuses_bad_arguments():
    with pytest.raises(sas.SasError):
        sas.sas_cylinder_radial_table(np.ones(1), np.ones(1), 0.0, 1.0, 10)
    with pytest.raises(sas.SasError):
        sas.sas_cylinder_radial_table(np.ones(1), np.ones(1), 1.0, 1.0, 1)
