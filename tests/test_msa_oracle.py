"""Pins of the oracle's Hayter-Penfold S(Q) (oracle/msa.py): the mean
spherical approximation of charged hard spheres, solved numerically.

* zero charge: the MSA of hard spheres is the Percus-Yevick closure, so S
  must equal the oracle's closed-form Percus-Yevick S(Q) (itself pinned in
  test_oracle_pins.py);
* low density: S(Q) - 1 = rho h0^(Q) + O(rho^2), with h0 = -1 in the core
  and -beta u outside, whose transform is closed:
  h0^(q) = -4 pi (sin q - q cos q) / q^3
           - (4 pi gamma_c / q) (k sin q + q cos q) / (k^2 + q^2)
  (reduced units); a wrong sign, range or normalisation of the potential
  fails it;
* the parameter mapping against textbook values: the Bjerrum length of
  water at 25 C (about 7.1 angstrom) and the Debye length of 0.1 M 1:1 salt
  (about 9.6 angstrom), the Debye length scaling as salt^-1/2;
* the Hansen-Hayter rescaling: strong coupling at low density gives s > 1
  with g(s sigma+) = 0; weak coupling leaves s = 1 with g(sigma+) > 0;
* S(Q) -> 1 at large Q;
* the oracle's C-side table (cubic Hermite in Q sigma steps of 0.02)
  against the direct transform at arbitrary Q;
* the library's own host solver (sas_hayter_msa_table: Newton's method
  with an analytic Jacobian, other grids) against the oracle (scipy's
  Newton-Krylov) on S and dS/dQ.
"""
import math

import numpy as np
import pytest

import oracle
import sas_workloads as W
from oracle import msa

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def test_zero_charge_is_percus_yevick():
    L = oracle.lib()
    for R, phi in ((30.0, 0.3), (50.0, 0.1), (20.0, 0.4)):
        sol = msa.Solution(R, phi, 0.0, 298.15, 0.1, 78.4)
        assert sol.s == 1.0
        Q = np.linspace(0.001, 0.6, 400)
        py = np.array([L.oracle_sq_py(float(q), R, phi) for q in Q])
        assert np.max(np.abs(sol.s_of_q(Q) / py - 1.0)) < 1e-7, (R, phi)


def _h0(q, gamma_c, k):
    return (-4.0 * math.pi * (np.sin(q) - q * np.cos(q)) / q ** 3
            - 4.0 * math.pi * gamma_c / q * (k * np.sin(q) + q * np.cos(q)) / (k * k + q * q))


def test_low_density_limit():
    R, salt = 30.0, 0.05
    q = np.linspace(0.2, 25.0, 120)            # reduced: Q sigma
    a = []
    for eta in (1e-4, 2e-4):
        p = msa.parameters(R, eta, 6.0, 298.15, salt, 78.4)
        sol = msa.Solution(R, eta, 6.0, 298.15, salt, 78.4)
        assert sol.s == 1.0
        rho = 6.0 * eta / math.pi
        a.append((sol.s_of_q(q / p["sigma"]) - 1.0) / rho)
    p = msa.parameters(R, 1e-4, 6.0, 298.15, salt, 78.4)
    assert 0.2 < p["gamma_c"] < 2.0
    lim = 2.0 * a[0] - a[1]                    # the O(rho) term removed
    ref = _h0(q, p["gamma_c"], p["k"])
    assert np.max(np.abs(lim - ref)) < 2e-4 * np.max(np.abs(ref))


def test_textbook_lengths():
    assert msa.bjerrum_length(298.15, 78.4) == pytest.approx(7.1, rel=0.01)
    debye = 1.0 / msa.parameters(30.0, 1e-12, 0.0, 298.15, 0.1, 78.4)["kappa"]
    assert debye == pytest.approx(9.6, rel=0.01)
    d4 = 1.0 / msa.parameters(30.0, 1e-12, 0.0, 298.15, 0.4, 78.4)["kappa"]
    assert debye / d4 == pytest.approx(2.0, rel=1e-9)


def test_rescaling():
    strong = msa.Solution(25.0, 0.02, 30.0, 298.15, 0.001, 78.4)
    assert strong.s > 1.5
    assert abs(strong.contact()) < 1e-8
    weak = msa.Solution(40.0, 0.2, 5.0, 298.15, 0.1, 78.4)
    assert weak.s == 1.0 and weak.contact() > 0.0


def test_large_q_limit():
    sol = msa.Solution(20.0, 0.1, 20.0, 298.15, 0.01, 78.4)
    sig = sol.sigma * sol.s
    assert abs(sol.s_of_q(np.array([200.0 / sig]))[0] - 1.0) < 5e-3


def test_c_table_against_the_direct_transform():
    m = W.Model(kind=W.SPHERE, precision=W.FP64, radius=20.0, sld=2e-6, volume_fraction=0.1,
                sq_kind=W.SQ_HAYTER_MSA, sq_radius=22.0, sq_fraction=0.1, sq_charge=20.0, sq_salt=0.01)
    m0 = W.Model(**{**m.as_dict(), "sq_kind": W.SQ_NONE})
    P, P0 = oracle.Prepared(m), oracle.Prepared(m0)
    rng = np.random.default_rng(3)
    Q = rng.uniform(1e-4, 0.9, 300)
    qv = np.stack([Q, np.zeros_like(Q), np.zeros_like(Q)], axis=1)
    S = oracle.dsigma(P, qv) / oracle.dsigma(P0, qv)
    assert np.max(np.abs(S / P.msa.s_of_q(Q) - 1.0)) < 1e-8


@pytest.mark.parametrize("args", [(30.0, 0.3, 0.0, 298.15, 0.1, 78.4), (20.0, 0.1, 20.0, 298.15, 0.01, 78.4),
                                  (25.0, 0.02, 30.0, 298.15, 0.001, 78.4), (40.0, 0.2, 15.0, 310.0, 0.05, 70.0)])
def test_library_host_solver_against_the_oracle(args):
    import paper_2501_06054_gb300 as sas
    T = sas.sas_hayter_msa_table(*args, q_max=0.5)
    o = msa.Solution(*args)
    assert T["s_rescale"] == pytest.approx(o.s, rel=1e-8)
    Q = np.arange(len(T["S"])) * T["dq"]
    m = Q <= 0.5
    assert np.max(np.abs(T["S"][m] / o.s_of_q(Q[m]) - 1.0)) < 1e-7
    D = o.ds_dq(Q[m])
    assert np.max(np.abs(T["dS_dQ"][m] - D)) < 1e-7 * np.max(np.abs(D))
    p = msa.parameters(*args)
    assert T["gamma_c"] == pytest.approx(p["gamma_c"], rel=1e-12)
    assert T["kappa"] == pytest.approx(p["kappa"], rel=1e-12)


def test_library_table_interpolation():
    """The trace interpolates the library's table by cubic Hermite in steps
    of Q sigma' = pi / 64: within 5e-7 of the direct transform (2.2e-7 on
    the densest case here, eta = 0.35), which bounds the FP64 model."""
    import paper_2501_06054_gb300 as sas
    for args in ((22.0, 0.35, 10.0, 298.15, 0.01, 78.4), (25.0, 0.02, 30.0, 298.15, 0.001, 78.4)):
        T = sas.sas_hayter_msa_table(*args, q_max=0.6)
        o = msa.Solution(*args)
        Q = np.random.default_rng(1).uniform(1e-4, 0.5, 2000)
        h = T["dq"]
        s = Q / h
        i = s.astype(int)
        f = s - i
        S0, S1 = T["S"][i], T["S"][i + 1]
        D0, D1 = T["dS_dQ"][i] * h, T["dS_dQ"][i + 1] * h
        val = (1 + 2 * f) * (1 - f) ** 2 * S0 + f * (1 - f) ** 2 * D0 + f * f * (3 - 2 * f) * S1 + f * f * (f - 1) * D1
        assert np.max(np.abs(val / o.s_of_q(Q) - 1.0)) < 5e-7, args
