"""Hayter-Penfold structure factor of charged spheres (test infrastructure
only: the tests, the smoke check and the CPU baseline use it; the library
never does).

The structure factor of Table II's "Hayter MSA" entry: hard spheres of
diameter sigma carrying Z elementary charges in a 1:1 electrolyte, with the
screened Coulomb (DLVO) pair potential outside the hard core,

    beta u(r) = gamma_c sigma exp(-kappa (r - sigma)) / r,   r > sigma,
    gamma_c   = Z^2 l_B / ((1 + kappa sigma / 2)^2 sigma),

l_B = e^2 / (4 pi eps0 eps_r k_B T) the Bjerrum length and
kappa^2 = 4 pi l_B (2 n_salt + |Z| n_p) (salt ions and the particles'
counter-ions, all monovalent; n_p = 6 eta / (pi sigma^3)). The mean
spherical approximation (MSA) closes the Ornstein-Zernike (OZ) equation
with g(r) = 0 inside the core and c(r) = -beta u(r) outside. Where the MSA
contact value g(sigma+) comes out negative (dilute, strongly charged
systems) the Hansen-Hayter rescaling is applied: the hard-core diameter is
raised to s sigma (volume fraction eta s^3, the same potential, so
kappa sigma s and gamma_c exp(-kappa sigma (s - 1)) / s at the new
contact) until g(s sigma+) = 0. S(Q) = 1 / (1 - rho c^(Q)).

This module solves that definition directly: c and the indirect
correlation gamma = h - c on a uniform grid in x = r / sigma, the OZ
relation in Fourier space through the discrete sine transform, and the
closure by Newton-Krylov iteration on gamma (scipy's root finder), the
coupling raised in steps from the hard-sphere solution. S(Q) is the
trapezoid sine transform of c at the exact Q on two grids (dx and dx / 2),
combined by Richardson extrapolation (the discretisation error is of
second order: the jump of c at the core is placed on a grid point with the
mean of its two sides). The printed paper gives no formula for this model;
the readings above are stated beside the model in the design notes.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.fft import dst
from scipy.optimize import newton_krylov

E_CHARGE = 1.602176634e-19      # C
EPS0 = 8.8541878128e-12         # F/m
K_B = 1.380649e-23              # J/K
N_A = 6.02214076e23             # 1/mol


def bjerrum_length(temperature, dielectric):
    """l_B in angstrom."""
    return E_CHARGE ** 2 / (4.0 * math.pi * EPS0 * dielectric * K_B * temperature) * 1e10


def parameters(radius_eff, fraction, charge, temperature, salt, dielectric):
    """Reduced parameters of the hard-core screened Coulomb fluid:
    sigma (angstrom), eta, gamma_c (beta u at contact), k = kappa sigma,
    kappa (1/angstrom), l_B (angstrom)."""
    sigma = 2.0 * radius_eff
    lb = bjerrum_length(temperature, dielectric)
    n_salt = salt * N_A * 1000.0 * 1e-30                     # ions of one sign per angstrom^3
    n_p = 6.0 * fraction / (math.pi * sigma ** 3)
    kappa = math.sqrt(4.0 * math.pi * lb * (2.0 * n_salt + abs(charge) * n_p))
    k = kappa * sigma
    gamma_c = charge ** 2 * lb / ((1.0 + 0.5 * k) ** 2 * sigma)
    return dict(sigma=sigma, eta=fraction, gamma_c=gamma_c, k=k, kappa=kappa, l_b=lb)


class Grid:
    """Uniform grids x_i = i dx (i < n) and q_j = j pi / (n dx)."""

    def __init__(self, dx, length):
        self.dx = dx
        self.n = int(round(length / dx))
        self.x = np.arange(self.n) * dx
        self.dq = math.pi / (self.n * dx)
        self.q = np.arange(self.n) * self.dq
        self.i_core = int(round(1.0 / dx))

    def fwd(self, f):
        """(4 pi / q) int x f(x) sin(q x) dx at q_j (trapezoid; j = 0 left 0)."""
        out = np.zeros(self.n)
        out[1:] = 4.0 * math.pi * self.dx / self.q[1:] * dst((self.x * f)[1:], type=1) / 2.0
        return out

    def inv(self, F):
        """(1 / (2 pi^2 x)) int q F(q) sin(q x) dq at x_i (i = 0 left 0)."""
        out = np.zeros(self.n)
        out[1:] = self.dq / (2.0 * math.pi ** 2 * self.x[1:]) * dst((self.q * F)[1:], type=1) / 2.0
        return out


def _closure(g, eta, gamma_c, k):
    """c(x) of the MSA from gamma = h - c: -1 - gamma in the core, the
    potential's -beta u outside, the mean of both at x = 1."""
    x = g.x
    tail = np.zeros(g.n)
    tail[1:] = -gamma_c * np.exp(-k * (x[1:] - 1.0)) / x[1:]
    inner = -1.0
    def c_of(G):
        c = tail.copy()
        c[:g.i_core] = inner - G[:g.i_core]
        c[g.i_core] = 0.5 * ((inner - G[g.i_core]) + tail[g.i_core])
        return c
    return c_of


def solve(eta, gamma_c, k, dx, length, G0=None, steps=4):
    """The MSA on one grid: returns (grid, c, gamma). The coupling rises in
    `steps` equal steps from the hard-sphere problem (Newton-Krylov from the
    previous solution each time)."""
    g = Grid(dx, length)
    rho = 6.0 * eta / math.pi
    G = np.zeros(g.n) if G0 is None else G0.copy()
    fracs = [1.0] if G0 is not None else [(s + 1) / steps for s in range(steps)]
    for f in ([0.0] if G0 is None else []) + fracs:
        c_of = _closure(g, eta, gamma_c * f, k)

        def resid(G, c_of=c_of):
            C = g.fwd(c_of(G))
            return G - g.inv(rho * C * C / (1.0 - rho * C))
        G = newton_krylov(resid, G, f_tol=1e-12, maxiter=300)
    return g, _closure(g, eta, gamma_c, k)(G), G


def contact_value(g, c, G):
    """g(1+) = 1 + gamma(1) + c(1+), c(1+) = -beta u(1+)."""
    i = g.i_core
    c_out = 2.0 * c[i] - (-1.0 - G[i])      # the outer side of the mean at x = 1
    return 1.0 + G[i] + c_out


def c_hat(q, g, c):
    """The trapezoid sine transform of c at arbitrary q > 0 (x = 0 adds 0)."""
    q = np.atleast_1d(np.asarray(q, dtype=np.float64))
    out = np.empty_like(q)
    w = g.x * c * g.dx
    for a in range(0, len(q), 256):
        qq = q[a:a + 256, None]
        out[a:a + 256] = 4.0 * math.pi / qq[:, 0] * np.sum(w[None, :] * np.sin(qq * g.x[None, :]), axis=1)
    return out


def c_hat_dq(q, g, c):
    """d c^/dq at arbitrary q > 0."""
    q = np.atleast_1d(np.asarray(q, dtype=np.float64))
    out = np.empty_like(q)
    w = g.x * c * g.dx
    for a in range(0, len(q), 256):
        qq = q[a:a + 256, None]
        s, co = np.sin(qq * g.x[None, :]), np.cos(qq * g.x[None, :])
        out[a:a + 256] = 4.0 * math.pi * np.sum(w[None, :] * (g.x[None, :] * co / qq - s / qq ** 2), axis=1)
    return out


def _length(k):
    return float(max(16.0, 2.0 ** math.ceil(math.log2(1.0 + 32.0 / max(k, 1e-3)))))


class Solution:
    """The (rescaled) MSA of one parameter set, on the grids dx and dx / 2.
    Attributes: sigma (angstrom, the original diameter), s (rescaling, 1 if
    none), eta, rho (number density of the rescaled diameter), grids."""

    def __init__(self, radius_eff, fraction, charge, temperature, salt, dielectric, dx=1.0 / 256):
        p = parameters(radius_eff, fraction, charge, temperature, salt, dielectric)
        self.p = p
        self.sigma = p["sigma"]
        L = _length(p["k"])
        self.s = 1.0
        sols = None
        try:
            sols = self._pair(p["eta"], p["gamma_c"], p["k"], dx, L)
            g1 = self._contact(sols)
        except Exception:
            g1 = -1.0
        if g1 < 0.0:
            self.s, sols = self._rescale(p, dx, L)
        self.eta = p["eta"] * self.s ** 3
        self.rho = 6.0 * self.eta / math.pi
        self.sols = sols

    def _pair(self, eta, gamma_c, k, dx, L, warm=None):
        a = solve(eta, gamma_c, k, dx, L, None if warm is None else warm[0][2])
        b = solve(eta, gamma_c, k, dx / 2, L, None if warm is None else warm[1][2])
        return a, b

    @staticmethod
    def _contact(sols):
        g1 = [contact_value(*s) for s in sols]
        return (4.0 * g1[1] - g1[0]) / 3.0

    def _rescale(self, p, dx, L):
        def at(s, warm=None):
            return self._pair(p["eta"] * s ** 3, p["gamma_c"] * math.exp(-p["k"] * (s - 1.0)) / s,
                              p["k"] * s, dx, L, warm)
        lo, hi = 1.0, 1.0
        sols_hi = None
        while True:
            hi = 1.0 + 2.0 * (hi - 1.0) if hi > 1.0 else 1.05
            if p["eta"] * hi ** 3 > 0.45:
                raise ValueError("no Hansen-Hayter rescaling below eta = 0.45")
            try:
                sols_hi = at(hi)
                if self._contact(sols_hi) > 0.0:
                    break
                lo = hi
            except Exception:
                lo = hi
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            try:
                sols = at(mid, sols_hi)
                ok = self._contact(sols) > 0.0
            except Exception:
                ok = False
            if ok:
                hi, sols_hi = mid, sols
            else:
                lo = mid
            if hi - lo < 1e-12 * hi:
                break
        return hi, sols_hi

    def contact(self):
        return self._contact(self.sols)

    def s_of_q(self, Q):
        """S(Q), Q in 1/angstrom (array), Richardson-extrapolated."""
        qs = np.asarray(Q, dtype=np.float64) * self.sigma * self.s
        vals = []
        for g, c, _ in self.sols:
            C = np.where(qs > 0, c_hat(np.maximum(qs, 1e-300), g, c), 4.0 * math.pi * np.sum(g.x ** 2 * c * g.dx))
            vals.append(1.0 / (1.0 - self.rho * C))
        return (4.0 * vals[1] - vals[0]) / 3.0

    def ds_dq(self, Q):
        """dS/dQ (angstrom), Richardson-extrapolated."""
        sc = self.sigma * self.s
        qs = np.maximum(np.asarray(Q, dtype=np.float64) * sc, 1e-9)
        vals = []
        for g, c, _ in self.sols:
            C = c_hat(qs, g, c)
            vals.append(self.rho * c_hat_dq(qs, g, c) * sc / (1.0 - self.rho * C) ** 2)
        return (4.0 * vals[1] - vals[0]) / 3.0

    def table(self, q_max, n):
        """(dq, S[n], dS/dQ[n]) on Q_j = j dq, j < n, dq = q_max / (n - 1)."""
        dq = q_max / (n - 1)
        Q = np.arange(n) * dq
        S = self.s_of_q(Q)
        D = self.ds_dq(Q)
        D[0] = 0.0
        return dq, S, D
