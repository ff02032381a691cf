// Hayter-Penfold structure factor (Table II, "Hayter MSA"): the mean
// spherical approximation of the hard-core screened Coulomb fluid, solved
// on the host when the model is set, and the S(Q) table the trace
// interpolates.
//
// Method (reduced units: x = r / sigma, q = Q sigma, rho = 6 eta / pi):
// - unknowns: the indirect correlation gamma = h - c at the grid points
//   x_l = l dx inside the core and on it (l = 1..M, M = 1/dx); the closure
//   gives c = -1 - gamma inside, c = -beta u = -gamma_c exp(-k (x - 1)) / x
//   outside, the mean of both at x = 1 (second-order trapezoid sums across
//   the jump);
// - the Ornstein-Zernike relation in Fourier space, gamma^ = rho c^2 /
//   (1 - rho c^), with the radial transforms as discrete sine sums
//   c^(q_j) = (4 pi dx / q_j) sum_i x_i c_i sin(pi i j / n), q_j = j pi / L,
//   and back, (dq / (2 pi^2 x_i)) sum_j q_j gamma^_j sin(pi i j / n);
// - Newton's method on R_l = gamma_l - T(gamma)_l with the exact Jacobian of
//   the discrete map: dT_i/dgamma_l = (dq dx x_l a_l / (pi x_i))
//   (K_{i-l} - K_{i+l}), a_l = dc_l/dgamma_l (-1, or -1/2 on the core),
//   K_m = sum_j D_j cos(pi m j / n), D_j = rho c^_j (2 - rho c^_j) /
//   (1 - rho c^_j)^2; the coupling is raised in four steps from the hard
//   spheres, each step started from the previous solution;
// - two grids (dx = 1/128, 1/256) and Richardson's extrapolation of S and
//   of the contact value g(1+) = 1 + gamma(1) - gamma_c;
// - where g(1+) < 0, the Hansen-Hayter rescaling: the diameter s sigma with
//   g(s sigma+) = 0 (bracketed, then the Illinois variant of regula falsi),
//   volume fraction eta s^3, k s and the potential's value at the new
//   contact, gamma_c exp(-k (s - 1)) / s.
// Transforms by a radix-2 FFT of this file (no library).
#include "sas_msa.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>

namespace sas {
namespace msa {
namespace {

using cplx = std::complex<double>;
constexpr double kPi = 3.14159265358979323846;

// In-place radix-2 FFT (forward, e^{-2 pi i k n / N}); N a power of two.
void fft(std::vector<cplx>& a)
{
    const size_t n = a.size();
    for (size_t i = 1, j = 0; i < n; ++i) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    std::vector<cplx> w(n / 2);
    for (size_t k = 0; k < n / 2; ++k) {
        const double ang = -2.0 * kPi * (double)k / (double)n;
        w[k] = cplx(std::cos(ang), std::sin(ang));
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        const size_t step = n / len;
        for (size_t i = 0; i < n; i += len)
            for (size_t k = 0; k < len / 2; ++k) {
                const cplx u = a[i + k], v = a[i + k + len / 2] * w[k * step];
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
    }
}

// out[j] = sum_{i=1}^{n-1} y[i] sin(pi i j / m), j < m (m >= n, a power of two)
void sine_sums(const std::vector<double>& y, size_t m, std::vector<double>& out)
{
    std::vector<cplx> z(2 * m, cplx(0.0, 0.0));
    for (size_t i = 1; i < y.size(); ++i) {
        z[i] = y[i];
        z[2 * m - i] = -y[i];
    }
    fft(z);
    out.resize(m);
    for (size_t j = 0; j < m; ++j) out[j] = -0.5 * z[j].imag();
}

// out[j] = sum_{i=1}^{n-1} y[i] cos(pi i j / m), j < m
void cosine_sums(const std::vector<double>& y, size_t m, std::vector<double>& out)
{
    std::vector<cplx> z(2 * m, cplx(0.0, 0.0));
    for (size_t i = 1; i < y.size(); ++i) {
        z[i] = y[i];
        z[2 * m - i] = y[i];
    }
    fft(z);
    out.resize(m);
    for (size_t j = 0; j < m; ++j) out[j] = 0.5 * z[j].real();
}

// Dense solve A x = b (row-major n x n), partial pivoting; A, b overwritten.
bool lu_solve(std::vector<double>& A, std::vector<double>& b, int n)
{
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[(size_t)r * n + c]) > std::fabs(A[(size_t)p * n + c])) p = r;
        if (!(std::fabs(A[(size_t)p * n + c]) > 0.0)) return false;
        if (p != c) {
            for (int k = 0; k < n; ++k) std::swap(A[(size_t)p * n + k], A[(size_t)c * n + k]);
            std::swap(b[p], b[c]);
        }
        const double inv = 1.0 / A[(size_t)c * n + c];
        for (int r = c + 1; r < n; ++r) {
            const double f = A[(size_t)r * n + c] * inv;
            if (f == 0.0) continue;
            double* rr = &A[(size_t)r * n];
            const double* rc = &A[(size_t)c * n];
            for (int k = c; k < n; ++k) rr[k] -= f * rc[k];
            b[r] -= f * b[c];
        }
    }
    for (int c = n - 1; c >= 0; --c) {
        double s = b[c];
        for (int k = c + 1; k < n; ++k) s -= A[(size_t)c * n + k] * b[k];
        b[c] = s / A[(size_t)c * n + c];
    }
    return true;
}

// One grid: x_i = i dx, i < n = L / dx; q_j = j pi / L.
struct Grid {
    double dx = 0.0, L = 0.0, dq = 0.0;
    int n = 0, M = 0;
    Grid(double dx_, double L_) : dx(dx_), L(L_)
    {
        n = (int)std::lround(L / dx);
        M = (int)std::lround(1.0 / dx);
        dq = kPi / L;
    }
    double x(int i) const { return i * dx; }
    double q(int j) const { return j * dq; }
};

struct State {
    Grid g;
    double rho, gamma_c, k;
    std::vector<double> G;      // gamma at every grid point
    std::vector<double> tail;   // -beta u(x_i)
    State(const Grid& g_, double eta, double gc, double k_) : g(g_), rho(6.0 * eta / kPi), gamma_c(gc), k(k_)
    {
        G.assign(g.n, 0.0);
        set_potential(gc, k_);
    }
    void set_potential(double gc, double k_)
    {
        gamma_c = gc;
        k = k_;
        tail.assign(g.n, 0.0);
        for (int i = 1; i < g.n; ++i) tail[i] = -gc * std::exp(-k * (g.x(i) - 1.0)) / g.x(i);
    }
    void closure(const std::vector<double>& Gv, std::vector<double>& c) const
    {
        c.assign(g.n, 0.0);
        for (int i = 1; i < g.M; ++i) c[i] = -1.0 - Gv[i];
        c[g.M] = 0.5 * ((-1.0 - Gv[g.M]) + tail[g.M]);
        for (int i = g.M + 1; i < g.n; ++i) c[i] = tail[i];
    }
    // c^_j (j >= 1) of a closure's c
    void c_hat(const std::vector<double>& c, std::vector<double>& C) const
    {
        std::vector<double> y(g.n);
        for (int i = 0; i < g.n; ++i) y[i] = g.x(i) * c[i];
        std::vector<double> s;
        sine_sums(y, (size_t)g.n, s);
        C.assign(g.n, 0.0);
        for (int j = 1; j < g.n; ++j) C[j] = 4.0 * kPi * g.dx / g.q(j) * s[j];
    }
    // T(gamma) at every grid point; false where 1 - rho c^ <= 0 (no S)
    bool picard(const std::vector<double>& Gv, std::vector<double>& T, std::vector<double>& C) const
    {
        std::vector<double> c;
        closure(Gv, c);
        c_hat(c, C);
        std::vector<double> w(g.n, 0.0);
        for (int j = 1; j < g.n; ++j) {
            const double d = 1.0 - rho * C[j];
            if (!(d > 0.0)) return false;
            w[j] = g.q(j) * rho * C[j] * C[j] / d;
        }
        std::vector<double> s;
        sine_sums(w, (size_t)g.n, s);
        T.assign(g.n, 0.0);
        for (int i = 1; i < g.n; ++i) T[i] = g.dq / (2.0 * kPi * kPi * g.x(i)) * s[i];
        return true;
    }
    double residual(const std::vector<double>& Gv, std::vector<double>& R, std::vector<double>& C) const
    {
        std::vector<double> T;
        if (!picard(Gv, T, C)) return INFINITY;
        R.assign(g.M + 1, 0.0);
        double mx = 0.0;
        for (int l = 1; l <= g.M; ++l) {
            R[l] = Gv[l] - T[l];
            mx = std::max(mx, std::fabs(R[l]));
        }
        return mx;
    }
    // Newton's method from the current G; true on convergence.
    bool newton()
    {
        const int M = g.M;
        std::vector<double> R, C;
        double norm = residual(G, R, C);
        if (!std::isfinite(norm)) return false;
        for (int it = 0; it < 60; ++it) {
            if (norm < 1e-12) return true;
            std::vector<double> D(g.n, 0.0);
            for (int j = 1; j < g.n; ++j) {
                const double rc = rho * C[j], d = 1.0 - rc;
                D[j] = rc * (2.0 - rc) / (d * d);
            }
            std::vector<double> K;
            cosine_sums(D, (size_t)g.n, K);
            std::vector<double> A((size_t)M * M), b(M);
            const double f0 = g.dq * g.dx / kPi;
            for (int i = 1; i <= M; ++i) {
                for (int l = 1; l <= M; ++l) {
                    const double a = l < M ? -1.0 : -0.5;
                    const double dT = f0 * g.x(l) * a / g.x(i) * (K[std::abs(i - l)] - K[i + l]);
                    A[(size_t)(i - 1) * M + (l - 1)] = (i == l ? 1.0 : 0.0) - dT;
                }
                b[i - 1] = -R[i];
            }
            if (!lu_solve(A, b, M)) return false;
            double t = 1.0;
            bool ok = false;
            for (int h = 0; h < 30 && !ok; ++h, t *= 0.5) {
                std::vector<double> Gt = G;
                for (int l = 1; l <= M; ++l) Gt[l] += t * b[l - 1];
                std::vector<double> Rt, Ct;
                const double nt = residual(Gt, Rt, Ct);
                if (nt < (1.0 - 1e-4 * t) * norm || nt < 1e-12) {
                    G.swap(Gt);
                    R.swap(Rt);
                    C.swap(Ct);
                    norm = nt;
                    ok = true;
                }
            }
            if (!ok) return norm < 1e-10;
        }
        return norm < 1e-10;
    }
    double contact() const { return 1.0 + G[g.M] + tail[g.M]; }
};

// The pair of grids of one parameter set (same length L).
struct Pair {
    State a, b;   // dx = 1/128, 1/256
    Pair(double L, double eta, double gc, double k)
        : a(Grid(1.0 / 128, L), eta, gc, k), b(Grid(1.0 / 256, L), eta, gc, k) {}
    double contact() const { return (4.0 * b.contact() - a.contact()) / 3.0; }
};

// Solve one grid at (eta, gc, k): from its current gamma when warm, else
// from the hard spheres with the coupling raised in four steps.
bool solve_state(State& st, double eta, double gc, double k, bool warm)
{
    st.rho = 6.0 * eta / kPi;
    if (warm) {
        st.set_potential(gc, k);
        if (st.newton()) return true;
    }
    std::fill(st.G.begin(), st.G.end(), 0.0);
    for (int step = 0; step <= 4; ++step) {
        st.set_potential(gc * step / 4.0, k);
        if (!st.newton()) return false;
    }
    return true;
}

bool solve_pair(Pair& p, double eta, double gc, double k, bool warm)
{
    return solve_state(p.a, eta, gc, k, warm) && solve_state(p.b, eta, gc, k, warm);
}

// The screening tail must decay below 1e-14 of its contact value inside the box.
double box_length(double k, double gamma_c)
{
    if (gamma_c == 0.0) return 16.0;
    const double need = 1.0 + 32.0 / std::max(k, 1e-300);
    double L = 16.0;
    while (L < need) L *= 2.0;
    return L;
}

// S and dS/dq (reduced) at q_j = j pi / (P L), j < n_tab, of one grid's solution
void spectrum(const State& st, int P, int n_tab, std::vector<double>& S, std::vector<double>& D)
{
    const Grid& g = st.g;
    std::vector<double> c;
    st.closure(st.G, c);
    const size_t m = (size_t)P * g.n;
    std::vector<double> y1(g.n), y2(g.n);
    double c0 = 0.0;
    for (int i = 0; i < g.n; ++i) {
        y1[i] = g.x(i) * c[i];
        y2[i] = g.x(i) * g.x(i) * c[i];
        if (i > 0) c0 += y2[i];
    }
    std::vector<double> sn, cs;
    sine_sums(y1, m, sn);
    cosine_sums(y2, m, cs);
    S.assign(n_tab, 0.0);
    D.assign(n_tab, 0.0);
    const double dq = kPi / (P * g.L);
    for (int j = 0; j < n_tab; ++j) {
        double C, dC;
        if (j == 0) {
            C = 4.0 * kPi * g.dx * c0;
            dC = 0.0;
        } else {
            const double q = j * dq;
            C = 4.0 * kPi * g.dx * sn[j] / q;
            dC = (4.0 * kPi * g.dx * cs[j] - C) / q;
        }
        const double d = 1.0 - st.rho * C;
        S[j] = 1.0 / d;
        D[j] = st.rho * dC / (d * d);
    }
}

}  // namespace

Reduced reduce(double radius_eff, double fraction, double charge, double temperature, double salt,
               double dielectric)
{
    constexpr double e = 1.602176634e-19, eps0 = 8.8541878128e-12, kb = 1.380649e-23, na = 6.02214076e23;
    Reduced r;
    r.sigma = 2.0 * radius_eff;
    r.eta = fraction;
    r.l_b = e * e / (4.0 * kPi * eps0 * dielectric * kb * temperature) * 1e10;
    const double n_salt = salt * na * 1000.0 * 1e-30;                     // per angstrom^3, each sign
    const double n_p = 6.0 * fraction / (kPi * r.sigma * r.sigma * r.sigma);
    r.kappa = std::sqrt(4.0 * kPi * r.l_b * (2.0 * n_salt + std::fabs(charge) * n_p));
    r.k = r.kappa * r.sigma;
    r.gamma_c = charge * charge * r.l_b / ((1.0 + 0.5 * r.k) * (1.0 + 0.5 * r.k) * r.sigma);
    return r;
}

bool build_table(const Reduced& r, double q_max, Table& out, std::string& err)
{
    if (!(r.sigma > 0.0) || !(r.eta > 0.0) || !(r.eta < 0.45)) {
        err = "Hayter MSA needs sq_radius > 0 and 0 < sq_fraction < 0.45";
        return false;
    }
    if (r.gamma_c > 0.0 && !(r.k >= 32.0 / 511.0)) {
        err = "Hayter MSA: screening length beyond 500 hard-core diameters";
        return false;
    }
    const double L = box_length(r.k, r.gamma_c);
    Pair p(L, r.eta, r.gamma_c, r.k);
    double s = 1.0;
    bool ok = solve_pair(p, r.eta, r.gamma_c, r.k, false);
    double g1 = ok ? p.contact() : -1.0;
    if (g1 < 0.0) {
        // Hansen-Hayter: g(s sigma+) = 0
        auto f = [&](double sv, bool warm, double& gv) {
            const bool k_ok = solve_pair(p, r.eta * sv * sv * sv, r.gamma_c * std::exp(-r.k * (sv - 1.0)) / sv,
                                         r.k * sv, warm);
            gv = k_ok ? p.contact() : -1.0;
            return k_ok;
        };
        double lo = 1.0, hi = 1.0, g_lo = g1, g_hi = 0.0;
        for (;;) {
            hi = hi > 1.0 ? 1.0 + 2.0 * (hi - 1.0) : 1.05;
            if (r.eta * hi * hi * hi > 0.45) {
                err = "Hayter MSA: no Hansen-Hayter rescaling below a volume fraction of 0.45";
                return false;
            }
            f(hi, false, g_hi);
            if (g_hi > 0.0) break;
            lo = hi;
            g_lo = g_hi;
        }
        // Illinois regula falsi on g(s) (a failed solve counts as g < 0)
        int side = 0;
        for (int it = 0; it < 100 && hi - lo > 1e-12 * hi; ++it) {
            double mid = (lo * g_hi - hi * g_lo) / (g_hi - g_lo);
            if (!(mid > lo && mid < hi)) mid = 0.5 * (lo + hi);
            double gm;
            f(mid, true, gm);
            if (std::fabs(gm) < 1e-12 && gm >= 0.0) {
                hi = mid;
                g_hi = gm;
                break;
            }
            if (gm > 0.0) {
                hi = mid;
                g_hi = gm;
                if (side == 1) g_lo *= 0.5;
                side = 1;
            } else {
                lo = mid;
                g_lo = gm;
                if (side == -1) g_hi *= 0.5;
                side = -1;
            }
        }
        s = hi;
        double gfin;
        if (!f(s, true, gfin)) {
            err = "Hayter MSA: the rescaled problem did not converge";
            return false;
        }
        g1 = gfin;
    }
    // the table: q_red spacing pi / (P L) = pi / 64 when L <= 64
    const int P = std::max(1, (int)std::lround(64.0 / L));
    const double dq_red = kPi / (P * L);
    const double sig = r.sigma * s;
    const int n_lim = P * p.a.g.n;                         // the coarse grid's range
    const int n_tab = (int)std::ceil(q_max * sig / dq_red) + 3;
    if (n_tab > (int)(0.75 * n_lim)) {
        err = "Hayter MSA: the largest |Q| times the diameter is beyond the solver's grid";
        return false;
    }
    std::vector<double> Sa, Da, Sb, Db;
    spectrum(p.a, P, n_tab, Sa, Da);
    spectrum(p.b, P, n_tab, Sb, Db);
    out.dq = dq_red / sig;
    out.sd.assign((size_t)2 * n_tab, 0.0);
    for (int j = 0; j < n_tab; ++j) {
        out.sd[2 * j] = (4.0 * Sb[j] - Sa[j]) / 3.0;
        out.sd[2 * j + 1] = (4.0 * Db[j] - Da[j]) / 3.0 * sig;   // dS/dQ
    }
    out.s_rescale = s;
    out.contact = g1;
    for (int j = 0; j < n_tab; ++j)
        if (!(out.sd[2 * j] > 0.0) || !std::isfinite(out.sd[2 * j + 1])) {
            err = "Hayter MSA: non-positive S(Q) in the solution";
            return false;
        }
    return true;
}

}  // namespace msa
}  // namespace sas
