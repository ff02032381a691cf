// Host runtime and C ABI of libsas: experiment objects, FP64 quadrature and
// constant tables, launch configuration, error mapping.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "sas_kernels.cuh"
#include "sas_host.h"
#include "sas_msa.h"
#include "sas_sur_host.h"

namespace {

thread_local std::string g_last_error;

sas_status fail(sas_status s, const std::string& msg)
{
    g_last_error = msg;
    return s;
}

sas_status cuda_fail(cudaError_t e, const char* what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(e == cudaErrorMemoryAllocation ? SAS_ERR_OOM : SAS_ERR_CUDA, m);
}

#define SAS_CUDA(call, what)                        \
    do {                                            \
        cudaError_t _e = (call);                    \
        if (_e != cudaSuccess) return cuda_fail(_e, what); \
    } while (0)

bool finite_all(std::initializer_list<double> v)
{
    for (double x : v)
        if (!std::isfinite(x)) return false;
    return true;
}

}  // namespace

namespace sas {

sas_status set_error(sas_status s, const std::string& msg) { return fail(s, msg); }
sas_status set_cuda_error(cudaError_t e, const char* what) { return cuda_fail(e, what); }

// Cost model of one history in FLOP (FMA = 2): the nominal per-term counts
// of the kernels' formulas (sphere amplitude 33, core-shell node 62,
// cylinder radial term 26, orientation node 60, geometry 150,
// Percus-Yevick 40).
double host_flops_per_history(const sas_model_desc& m, int np, int no)
{
    if (m.sampling == SAS_PER_EVENT) { np = 1; no = 1; }
    if (m.kind == SAS_CYLINDER && m.radial_table && m.sampling == SAS_QUADRATURE)
        return no * 60.0 + 150.0 + (m.sq_kind == SAS_SQ_HARD_SPHERE_PY ? 40.0 : 0.0);
    if (axes3_kind(m.kind)) {
        const int frames = m.sampling == SAS_PER_EVENT ? 1 : std::max(no / 3, 1);
        const double term = m.kind == SAS_TRIAXIAL_ELLIPSOID ? 36.0 : m.kind == SAS_PARALLELEPIPED ? 66.0
                          : m.kind == SAS_ELLIPTICAL_CYLINDER ? 50.0 : 132.0;
        return frames * (20.0 + np * term) + 150.0 + (m.sq_kind == SAS_SQ_HARD_SPHERE_PY ? 40.0 : 0.0);
    }
    if (m.kind == SAS_CAPPED_CYLINDER || m.kind == SAS_BARBELL) {
        // per radius node: the cylinder term (sinc, 2 J1(x)/x; 60) and per cap
        // slice cos + 2 J1(x)/x (30)
        const int nr = (m.poly > 0.0 && m.n_poly > 1 && m.sampling == SAS_QUADRATURE) ? (int)m.n_poly : 1;
        return no * (40.0 + nr * (60.0 + 30.0 * (double)m.n_cap)) + 150.0 +
               (m.sq_kind == SAS_SQ_HARD_SPHERE_PY ? 40.0 : 0.0);
    }
    if (m.kind == SAS_SHAPE_INDEPENDENT) return 150.0 + 30.0;
    if (shelled_cylinder(m.kind))
        return no * (60.0 + 26.0 + np * 2.0 * 26.0) + 150.0 + (m.sq_kind == SAS_SQ_HARD_SPHERE_PY ? 40.0 : 0.0);
    if (m.kind == SAS_CORE_SHELL_ELLIPSOID)
        return no * (60.0 + np * 2.0 * 38.0) + 150.0 + (m.sq_kind == SAS_SQ_HARD_SPHERE_PY ? 40.0 : 0.0);
    double per;
    if (m.kind == SAS_SPHERE) per = np * 36.0;
    else if (m.kind == SAS_CORE_SHELL) per = np * 62.0 + 20.0;
    else if (m.kind == SAS_CYLINDER) per = no * (60.0 + np * 26.0);
    else per = no * (60.0 + np * 38.0);
    return per + 150.0 + (m.sq_kind == SAS_SQ_HARD_SPHERE_PY ? 40.0 : 0.0);
}

// ----------------------------------------------------------- quadrature
// Gauss-Legendre nodes by Newton's method on P_n with the three-term
// recurrence (initial guesses cos(pi (i - 1/4) / (n + 1/2))); weights
// 2 / ((1 - x^2) P_n'(x)^2).
void gauss_legendre(int n, double* x, double* w)
{
    if (n == 1) {
        x[0] = 0.0;
        w[0] = 2.0;
        return;
    }
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        // recompute the derivative at the converged node
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        const double wi = 2.0 / ((1.0 - z * z) * dp * dp);
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = wi;
        w[n - 1 - i] = wi;
    }
}

// Eigenvalues of the symmetric tridiagonal matrix (diagonal d[n],
// off-diagonal e[n-1]) and the first component of each unit eigenvector, by
// the implicit QL iteration with Wilkinson-type shifts (Golub and Van Loan,
// Sec. 8.3): each sweep chases a bulge with Givens rotations from the bottom
// of the active block up to its top; only row 0 of the accumulated rotations
// is kept. O(n^2) work.
static void tridiag_eigen(int n, const double* d_in, const double* e_in, double* lam, double* v0)
{
    std::vector<double> d(d_in, d_in + n), e((size_t)n, 0.0), z((size_t)n, 0.0);
    for (int i = 0; i + 1 < n; ++i) e[i] = e_in[i];
    z[0] = 1.0;
    for (int l = 0; l < n; ++l) {
        for (int iter = 0; iter < 60; ++iter) {
            int m = l;
            for (; m + 1 < n; ++m) {   // a negligible coupling splits the block at m
                const double dd = std::fabs(d[m]) + std::fabs(d[m + 1]);
                if (std::fabs(e[m]) <= 1e-17 * dd) break;
            }
            if (m == l) break;
            // shift: the eigenvalue of the leading 2x2 block closer to d[l]
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = std::hypot(g, 1.0);
            g = d[m] - d[l] + e[l] / (g + (g >= 0.0 ? r : -r));
            double sn = 1.0, cs = 1.0, p = 0.0;
            bool deflated = false;
            for (int i = m - 1; i >= l; --i) {
                const double f = sn * e[i], b = cs * e[i];
                r = std::hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) {        // the bulge vanished: the block splits here
                    d[i + 1] -= p;
                    e[m] = 0.0;
                    deflated = true;
                    break;
                }
                sn = f / r;
                cs = g / r;
                g = d[i + 1] - p;
                r = (d[i] - g) * sn + 2.0 * cs * b;
                p = sn * r;
                d[i + 1] = g + p;
                g = cs * r - b;
                const double zi = z[i], zi1 = z[i + 1];   // rotate columns i, i + 1 of row 0
                z[i + 1] = sn * zi + cs * zi1;
                z[i] = cs * zi - sn * zi1;
            }
            if (deflated) continue;
            d[l] -= p;
            e[l] = g;
            e[m] = 0.0;
        }
    }
    for (int i = 0; i < n; ++i) {
        lam[i] = d[i];
        v0[i] = z[i];
    }
}

// Generalised Gauss-Laguerre rule for x^alpha e^-x (Golub-Welsch), weights
// normalised to sum 1, nodes ascending.
void gauss_laguerre_gen(int n, double alpha, double* x, double* w)
{
    std::vector<double> d(n), e(n > 1 ? n - 1 : 1), lam(n), v0(n);
    for (int k = 0; k < n; ++k) d[k] = 2.0 * k + alpha + 1.0;
    for (int k = 1; k < n; ++k) e[k - 1] = std::sqrt(k * (k + alpha));
    tridiag_eigen(n, d.data(), e.data(), lam.data(), v0.data());
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return lam[a] < lam[b]; });
    double sw = 0.0;
    for (int i = 0; i < n; ++i) sw += v0[i] * v0[i];
    for (int i = 0; i < n; ++i) {
        x[i] = lam[idx[i]];
        w[i] = v0[idx[i]] * v0[idx[i]] / sw;
    }
}

// Schulz distribution of mean `mean`, relative width p: r_i = mean x_i/(z+1)
// with the generalised Gauss-Laguerre rule of alpha = z = 1/p^2 - 1.
void schulz_nodes(double mean, double p, int n, double* r, double* w)
{
    if (p <= 0.0 || n <= 1) {
        r[0] = mean;
        w[0] = 1.0;
        return;
    }
    const double z = 1.0 / (p * p) - 1.0;
    gauss_laguerre_gen(n, z, r, w);
    for (int i = 0; i < n; ++i) r[i] = mean * r[i] / (z + 1.0);
}

// Gaussian N(mean, (p mean)^2) restricted to positive values (the
// polydispersity law of Sec. II.B): Gauss-Legendre nodes on
// [max(0, mean (1 - 8p)), mean (1 + 8p)] weighted by the density and
// normalised; the mass beyond 8 sigma is below 1e-15.
void gaussian_nodes(double mean, double p, int n, double* r, double* w)
{
    if (p <= 0.0 || n <= 1) {
        r[0] = mean;
        w[0] = 1.0;
        for (int i = 1; i < n; ++i) r[i] = mean, w[i] = 0.0;
        return;
    }
    const double a = std::max(0.0, mean * (1.0 - 8.0 * p)), b = mean * (1.0 + 8.0 * p), sd = p * mean;
    std::vector<double> x(n), wx(n);
    gauss_legendre(n, x.data(), wx.data());
    double tot = 0.0;
    for (int i = 0; i < n; ++i) {
        r[i] = 0.5 * (b - a) * (x[i] + 1.0) + a;
        const double d = (r[i] - mean) / sd;
        w[i] = 0.5 * (b - a) * wx[i] * std::exp(-0.5 * d * d);
        tot += w[i];
    }
    for (int i = 0; i < n; ++i) w[i] /= tot;
}

// Axis nodes for theta ~ U[0, pi], phi ~ U[0, 2 pi] (Sec. II.B; uniform in
// the angles, not on the sphere): Gauss-Legendre in both angles.
int uniform_angle_nodes(int nt, int np, double* c, double* wout)
{
    std::vector<double> xt(nt), wt(nt), xp(np), wp(np);
    gauss_legendre(nt, xt.data(), wt.data());
    gauss_legendre(np, xp.data(), wp.data());
    double tot = 0.0;
    int k = 0;
    for (int i = 0; i < nt; ++i) {
        const double th = 0.5 * M_PI * (xt[i] + 1.0), st = std::sin(th), ct = std::cos(th);
        for (int j = 0; j < np; ++j) {
            const double ph = M_PI * (xp[j] + 1.0);
            c[3 * k] = st * std::cos(ph);
            c[3 * k + 1] = st * std::sin(ph);
            c[3 * k + 2] = ct;
            wout[k] = wt[i] * wp[j];
            tot += wout[k];
            ++k;
        }
    }
    for (int i = 0; i < k; ++i) wout[i] /= tot;
    return k;
}

// Frame (rows A, B, C) of the angles: C along (theta, phi); A, B the unit
// vectors e_theta, e_phi of C rotated by psi about C.
void frame_of(double theta, double phi, double psi, double* f)
{
    const double st = std::sin(theta), ct = std::cos(theta), sp = std::sin(phi), cp = std::cos(phi);
    const double sq = std::sin(psi), cq = std::cos(psi);
    const double et[3] = {ct * cp, ct * sp, -st}, ep[3] = {-sp, cp, 0.0};
    for (int k = 0; k < 3; ++k) {
        f[k] = cq * et[k] + sq * ep[k];
        f[3 + k] = -sq * et[k] + cq * ep[k];
    }
    f[6] = st * cp;
    f[7] = st * sp;
    f[8] = ct;
}

// Orientation nodes of a particle without a symmetry axis: frames (9 doubles
// each) and normalised weights. isotropic 0: the C axis on the Gaussian-cap
// nodes, the mean frame carried along by the smallest rotation taking its C
// to the node's (Rodrigues); 1: uniform rotations, Gauss-Legendre in
// cos theta, phi and psi; 2: theta, phi and psi uniform.
int frame_nodes(const sas_model_desc& m, std::vector<double>& fr, std::vector<double>& w)
{
    fr.clear();
    w.clear();
    if (m.isotropic == 0) {
        double f0[9];
        frame_of(m.axis_theta, m.axis_phi, m.axis_psi, f0);
        const int nmax = std::max((int)(m.n_gamma * m.n_psi), 1);
        std::vector<double> c((size_t)3 * nmax), wc(nmax);
        const int n = orientation_nodes(m.axis_theta, m.axis_phi, m.sigma_orient, (int)m.n_gamma, (int)m.n_psi, 0,
                                        c.data(), wc.data());
        for (int o = 0; o < n; ++o) {
            const double* u = f0 + 6;    // mean C
            const double* v = c.data() + 3 * o;
            double k[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
            const double sn = std::sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
            const double cs = u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
            double R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
            if (sn > 1e-15) {
                for (double& x : k) x /= sn;
                const double K[9] = {0, -k[2], k[1], k[2], 0, -k[0], -k[1], k[0], 0};
                double K2[9];
                for (int r = 0; r < 3; ++r)
                    for (int q = 0; q < 3; ++q) {
                        K2[3 * r + q] = 0.0;
                        for (int t = 0; t < 3; ++t) K2[3 * r + q] += K[3 * r + t] * K[3 * t + q];
                    }
                for (int e = 0; e < 9; ++e) R[e] += sn * K[e] + (1.0 - cs) * K2[e];
            }
            for (int row = 0; row < 3; ++row)
                for (int r = 0; r < 3; ++r) {
                    double x = 0.0;
                    for (int q = 0; q < 3; ++q) x += R[3 * r + q] * f0[3 * row + q];
                    fr.push_back(x);
                }
            w.push_back(wc[o]);
        }
        return n;
    }
    const int nt = (int)m.n_gamma, np = (int)m.n_psi, nr = (int)m.n_rot;
    std::vector<double> xt(nt), wt(nt), xp(np), wp(np), xr(nr), wr(nr);
    gauss_legendre(nt, xt.data(), wt.data());
    gauss_legendre(np, xp.data(), wp.data());
    gauss_legendre(nr, xr.data(), wr.data());
    double tot = 0.0;
    for (int i = 0; i < nt; ++i) {
        const double th = m.isotropic == 1 ? std::acos(std::max(-1.0, std::min(1.0, xt[i]))) : 0.5 * M_PI * (xt[i] + 1.0);
        for (int j = 0; j < np; ++j)
            for (int k = 0; k < nr; ++k) {
                double f[9];
                frame_of(th, M_PI * (xp[j] + 1.0), M_PI * (xr[k] + 1.0), f);
                fr.insert(fr.end(), f, f + 9);
                w.push_back(wt[i] * wp[j] * wr[k]);
                tot += w.back();
            }
    }
    for (double& x : w) x /= tot;
    return (int)w.size();
}

// Cylinder radial table (G, h G') on [0, xmax] and its midpoint error.
double cylinder_radial_table(const double* r, const double* w, int np, double rbar, double xmax, int n,
                             double* G, double* D)
{
    const double h = xmax / (double)(n - 1);
    auto eval = [&](double x, double& g, double& dg) {
        g = 0.0;
        dg = 0.0;
        for (int i = 0; i < np; ++i) {
            const double t = r[i] / rbar, y = x * t, t4 = t * t * t * t;
            double a, da;
            if (y < 1e-4) {
                a = 1.0 - y * y / 8.0;
                da = -y / 4.0;
            } else {
                a = 2.0 * ::j1(y) / y;
                da = -2.0 * ::jn(2, y) / y;   // d/dy [2 J1(y) / y]
            }
            g += w[i] * t4 * a * a;
            dg += w[i] * t4 * 2.0 * a * da * t;
        }
    };
    for (int k = 0; k < n; ++k) {
        double g, dg;
        eval(k * h, g, dg);
        G[k] = g;
        D[k] = h * dg;
    }
    double err = 0.0;
    for (int k = 0; k + 1 < n; ++k) {
        double g, dg;
        eval((k + 0.5) * h, g, dg);
        // cubic Hermite at f = 1/2: (G0 + G1)/2 + (D0 - D1)/8
        const double hm = 0.5 * (G[k] + G[k + 1]) + 0.125 * (D[k] - D[k + 1]);
        err = std::max(err, std::fabs(hm - g));
    }
    return err;
}

// Upper bound of |Q| reachable on the instrument: the largest wavelength
// spread k, the steepest incoming ray through both pinholes and the widest
// angle from any sample point to any detector point, with 1 % margin.
double instrument_q_max(const sas_instrument& in)
{
    const double kmax = 2.0 * M_PI / (in.lambda0 * (1.0 - in.dlambda_rel));
    const double t_in = std::atan((in.ap1_radius + in.ap2_radius) / std::fabs(in.ap2_z - in.ap1_z));
    const double half_w = 0.5 * in.nx * in.pixel_x, half_h = 0.5 * in.ny * in.pixel_y;
    const double lat = std::sqrt(half_w * half_w + half_h * half_h) +
                       std::sqrt(in.sample_half_x * in.sample_half_x + in.sample_half_y * in.sample_half_y) +
                       in.ap2_radius;
    const double t_out = std::atan(lat / std::max(in.det_distance - in.sample_thickness, 1e-9));
    const double th = std::min(t_in + t_out, M_PI);
    return 1.01 * 2.0 * kmax * std::sin(0.5 * th);
}

// Orientation nodes: axis = cos(g) n + sin(g) (cos(s) e_theta + sin(s) e_phi),
// g on Gauss-Legendre nodes of [0, gmax] with weight sin(g) (times the
// Gaussian exp(-g^2 / (2 sigma^2)) unless isotropic), s on Gauss-Legendre
// nodes of [0, 2 pi). Returns the node count.
int orientation_nodes(double theta, double phi, double sigma, int ng, int npsi, int isotropic,
                      double* c, double* wout)
{
    const double st = std::sin(theta), ct = std::cos(theta), sp = std::sin(phi), cp = std::cos(phi);
    const double nv[3] = {st * cp, st * sp, ct};
    const double et[3] = {ct * cp, ct * sp, -st};
    const double ep[3] = {-sp, cp, 0.0};
    if (!isotropic && (sigma <= 0.0 || ng * npsi <= 1)) {
        c[0] = nv[0];
        c[1] = nv[1];
        c[2] = nv[2];
        wout[0] = 1.0;
        return 1;
    }
    const double gmax = isotropic ? M_PI : std::min(3.0 * sigma, M_PI);
    std::vector<double> xg(ng), wg(ng), xs(npsi), ws(npsi);
    gauss_legendre(ng, xg.data(), wg.data());
    gauss_legendre(npsi, xs.data(), ws.data());
    double tot = 0.0;
    int k = 0;
    for (int i = 0; i < ng; ++i) {
        const double g = 0.5 * gmax * (xg[i] + 1.0);
        double wgi = 0.5 * gmax * wg[i] * std::sin(g);
        if (!isotropic) wgi *= std::exp(-g * g / (2.0 * sigma * sigma));
        const double sg = std::sin(g), cg = std::cos(g);
        for (int j = 0; j < npsi; ++j) {
            const double s = M_PI * (xs[j] + 1.0);
            const double cs = std::cos(s), ss = std::sin(s);
            for (int a = 0; a < 3; ++a) c[3 * k + a] = cg * nv[a] + sg * (cs * et[a] + ss * ep[a]);
            wout[k] = wgi * M_PI * ws[j];
            tot += wout[k];
            ++k;
        }
    }
    for (int i = 0; i < k; ++i) wout[i] /= tot;
    return k;
}

// Percus-Yevick: coefficients of G(A)/A in powers of A^2, from the Taylor
// coefficients of the three brackets of G (derived in closed form):
//   b1 = sin A - A cos A                      -> A^(2m+3): (-1)^m 2(m+1)/(2m+3)!
//   b2 = 2A sin A + (2 - A^2) cos A - 2       -> A^(2m+4): (-1)^m 2(2m+3)(m+1)/(2m+4)!
//   b3 = -A^4 cos A + 4[(3A^2-6) cos A + (A^3-6A) sin A + 6]
//        -> A^N, N = 2m+6: (-1)^(m+1) [-N(N-1)(N-2)(N-3) - 12N(N-1)
//                                      + 4N(N-1)(N-2) + 24N - 24] / N!
void py_constants(double phi, double* alpha, double* beta, double* gamma, double* series, int nser)
{
    const double d = std::pow(1.0 - phi, 4);
    *alpha = (1.0 + 2.0 * phi) * (1.0 + 2.0 * phi) / d;
    *beta = -6.0 * phi * (1.0 + 0.5 * phi) * (1.0 + 0.5 * phi) / d;
    *gamma = 0.5 * phi * (*alpha);
    for (int m = 0; m < nser; ++m) {
        const double sgn = (m % 2 == 0) ? 1.0 : -1.0;
        const double c1 = sgn * 2.0 * (m + 1) / std::tgamma(2.0 * m + 4.0);
        const double c2 = sgn * 2.0 * (2.0 * m + 3) * (m + 1) / std::tgamma(2.0 * m + 5.0);
        const double N = 2.0 * m + 6.0;
        const double br = -N * (N - 1) * (N - 2) * (N - 3) - 12.0 * N * (N - 1) + 4.0 * N * (N - 1) * (N - 2)
                          + 24.0 * N - 24.0;
        const double c3 = -sgn * br / std::tgamma(N + 1.0);
        series[m] = (*alpha) * c1 + (*beta) * c2 + (*gamma) * c3;
    }
}

// Height of a capped cylinder's or barbell's end cap beyond the end face:
// R - h (the capped cylinder's h = sqrt(R^2 - r^2) formed as r^2 / (R + h),
// free of cancellation for R >> r) or R + h.
double cap_height(const sas_model_desc& m)
{
    const double r = m.radius, R = m.radius_polar;
    const double h = std::sqrt(std::fmax(R * R - r * r, 0.0));
    return m.kind == SAS_CAPPED_CYLINDER ? r * r / (R + h) : R + h;
}

// Volume at the nominal sizes: pi r^2 L + 2 pi R H^2 (1 - H / 3R).
double capped_volume(const sas_model_desc& m)
{
    const double R = m.radius_polar, H = cap_height(m);
    return M_PI * m.radius * m.radius * m.length + 2.0 * M_PI * R * H * H * (1.0 - H / (3.0 * R));
}

// Kinds without a symmetry axis: orientation nodes are frames (A, B, C).
bool axes3_kind(int64_t kind)
{
    return kind == SAS_TRIAXIAL_ELLIPSOID || kind == SAS_PARALLELEPIPED || kind == SAS_ELLIPTICAL_CYLINDER ||
           kind == SAS_HOLLOW_RECTANGULAR_PRISM;
}

// Shelled cylinders: the face layer t_f (0 for the hollow cylinder) and the
// contrasts of the nested cylinders (r, L), (r, L + 2 t_f), (r + t, L),
// (r + t, L + 2 t_f) in the amplitude (Eq. 1 region by region).
bool shelled_cylinder(int64_t kind)
{
    return kind == SAS_CORE_SHELL_CYLINDER || kind == SAS_HOLLOW_CYLINDER || kind == SAS_CORE_SHELL_BICELLE;
}

double face_layer(const sas_model_desc& m) { return m.kind == SAS_HOLLOW_CYLINDER ? 0.0 : m.thickness_face; }

void shelled_contrasts(const sas_model_desc& m, double d[4])
{
    d[0] = d[1] = d[2] = d[3] = 0.0;
    if (m.kind == SAS_CORE_SHELL_CYLINDER) {        // core, then the shell around core and faces
        d[0] = m.sld - m.sld_shell;
        d[3] = m.sld_shell - m.sld_solvent;
    } else if (m.kind == SAS_HOLLOW_CYLINDER) {     // the tube minus its solvent core
        d[0] = -(m.sld - m.sld_solvent);
        d[2] = m.sld - m.sld_solvent;
    } else {                                        // bicelle: core, core + faces, core + faces + rim
        d[0] = m.sld - m.sld_face;
        d[1] = m.sld_face - m.sld_shell;
        d[3] = m.sld_shell - m.sld_solvent;
    }
}

// Tables of one model in FP64 (see sas_types.h for the layouts).
sas_status build_model_tables(const sas_model_desc& m, ModelTables& t, double q_max)
{
    const int np = (int)m.n_poly;
    std::vector<double> r(np), w(np);
    const double rmean = m.kind == SAS_SHAPE_INDEPENDENT ? 1.0 : m.radius;   // no particle: one dummy node
    if (m.poly_dist == SAS_POLY_GAUSSIAN) gaussian_nodes(rmean, m.poly, np, r.data(), w.data());
    else schulz_nodes(rmean, m.poly, np, r.data(), w.data());
    const int npoly = (m.kind != SAS_SHAPE_INDEPENDENT && m.poly > 0.0 && np > 1) ? np : 1;
    t.poly.assign((size_t)npoly * SAS_POLY_STRIDE, 0.0);
    double vmean = 0.0;
    const double pi = M_PI;
    for (int i = 0; i < npoly; ++i) {
        double* p = t.poly.data() + (size_t)i * SAS_POLY_STRIDE;
        const double ri = r[i];
        if (m.kind == SAS_SPHERE) {
            const double V = 4.0 / 3.0 * pi * ri * ri * ri;
            const double F0 = (m.sld - m.sld_solvent) * V;
            p[2] = 9.0 * w[i] * F0 * F0;
            p[0] = ri; p[1] = p[2] / (ri * ri * ri * ri * ri * ri); p[3] = ri * ri; p[4] = 1.0 / ri;
            vmean += w[i] * V;
        } else if (m.kind == SAS_CORE_SHELL) {
            const double ro = ri + m.thickness;
            const double Vc = 4.0 / 3.0 * pi * ri * ri * ri, Vo = 4.0 / 3.0 * pi * ro * ro * ro;
            const double sw = std::sqrt(w[i]);
            p[0] = ri * ri; p[1] = ro * ro;
            p[2] = 3.0 * sw * (m.sld - m.sld_shell) * Vc;
            p[3] = 3.0 * sw * (m.sld_shell - m.sld_solvent) * Vo;
            p[4] = p[2] / (ri * ri * ri);
            p[5] = p[3] / (ro * ro * ro);
            p[6] = ri; p[7] = ro;
            vmean += w[i] * Vo;
        } else if (m.kind == SAS_CYLINDER) {
            const double V = pi * ri * ri * m.length;
            const double F0 = (m.sld - m.sld_solvent) * V;
            p[0] = ri * ri; p[1] = w[i] * F0 * F0; p[2] = ri; p[3] = 1.0 / ri; p[4] = 1.0 / std::sqrt(ri);
            vmean += w[i] * V;
        } else if (m.kind == SAS_CAPPED_CYLINDER || m.kind == SAS_BARBELL) {
            const double sc = ri / m.radius;   // one polydisperse factor for r, R and L
            const double V = capped_volume(m) * sc * sc * sc;
            const double d = (m.sld - m.sld_solvent) * sc * sc * sc;
            p[0] = sc;
            p[1] = w[i] * d * d;
            p[2] = sc * sc;
            vmean += w[i] * V;
        } else if (shelled_cylinder(m.kind)) {
            // the nested cylinders (r, L), (r, L_o), (r_o, L), (r_o, L_o)
            const double ro = ri + m.thickness, L = m.length, Lo = L + 2.0 * face_layer(m);
            const double V[4] = {pi * ri * ri * L, pi * ri * ri * Lo, pi * ro * ro * L, pi * ro * ro * Lo};
            double d[4];
            shelled_contrasts(m, d);
            const double sw = std::sqrt(w[i]);
            p[0] = ri * ri; p[1] = ro * ro;
            for (int k = 0; k < 4; ++k) p[2 + k] = sw * d[k] * V[k];
            p[6] = ri; p[7] = ro;
            vmean += w[i] * (m.kind == SAS_HOLLOW_CYLINDER ? pi * (ro * ro - ri * ri) * L : V[3]);
        } else if (m.kind == SAS_CORE_SHELL_ELLIPSOID) {
            const double ro = ri + m.thickness, rp = m.radius_polar, rpo = rp + m.thickness_face;
            const double Vc = 4.0 / 3.0 * pi * ri * ri * rp, Vo = 4.0 / 3.0 * pi * ro * ro * rpo;
            const double sw = std::sqrt(w[i]);
            p[0] = ri * ri; p[1] = ro * ro;
            p[2] = 3.0 * sw * (m.sld - m.sld_shell) * Vc;
            p[3] = 3.0 * sw * (m.sld_shell - m.sld_solvent) * Vo;
            vmean += w[i] * Vo;
        } else if (m.kind == SAS_ELLIPTICAL_CYLINDER) {
            const double sc = ri / m.radius;
            const double V = pi * m.radius * m.radius_b * m.length * sc * sc * sc;
            const double F0 = (m.sld - m.sld_solvent) * V;
            p[0] = sc;
            p[1] = w[i] * F0 * F0;
            vmean += w[i] * V;
        } else if (m.kind == SAS_HOLLOW_RECTANGULAR_PRISM) {
            // amplitude / (drho 8 s^3) = a b c sinc sinc sinc - a_i b_i c_i sinc_i sinc_i sinc_i
            const double sc = ri / m.radius, s3 = sc * sc * sc, t = m.thickness;
            const double F0 = (m.sld - m.sld_solvent) * 8.0 * s3;
            p[0] = sc;
            p[1] = w[i] * F0 * F0;
            vmean += w[i] * 8.0 * s3 *
                     (m.radius * m.radius_b * m.radius_polar - (m.radius - t) * (m.radius_b - t) * (m.radius_polar - t));
        } else if (m.kind == SAS_TRIAXIAL_ELLIPSOID || m.kind == SAS_PARALLELEPIPED) {
            const double sc = ri / m.radius;   // one polydisperse factor for the three sizes
            const double V = (m.kind == SAS_TRIAXIAL_ELLIPSOID ? 4.0 / 3.0 * pi : 8.0) * m.radius * m.radius_b *
                             m.radius_polar * sc * sc * sc;
            const double F0 = (m.sld - m.sld_solvent) * V;
            p[0] = sc;
            p[1] = (m.kind == SAS_TRIAXIAL_ELLIPSOID ? 9.0 : 1.0) * w[i] * F0 * F0;
            vmean += w[i] * V;
        } else {
            const double V = 4.0 / 3.0 * pi * m.radius_polar * ri * ri;
            const double F0 = (m.sld - m.sld_solvent) * V;
            p[0] = ri * ri; p[1] = 9.0 * w[i] * F0 * F0;
            vmean += w[i] * V;
        }
    }
    t.n_poly = npoly;
    t.r_max = 0.0;
    for (int i = 0; i < npoly; ++i) t.r_max = std::fmax(t.r_max, r[i]);
    t.scale = m.volume_fraction / vmean;
    t.vmean = vmean;
    if (m.kind == SAS_SHAPE_INDEPENDENT) {   // f_scale f(|Q|): no particle and no nodes
        std::fill(t.poly.begin(), t.poly.end(), 0.0);
        t.scale = m.f_scale;
        t.vmean = 1.0;
    }
    if (axes3_kind(m.kind)) {
        std::vector<double> fr, wf;
        const int nf = frame_nodes(m, fr, wf);
        t.orient.assign((size_t)3 * nf * SAS_ORIENT_STRIDE, 0.0);
        for (int o = 0; o < nf; ++o)
            for (int row = 0; row < 3; ++row) {
                double* d = t.orient.data() + ((size_t)3 * o + row) * SAS_ORIENT_STRIDE;
                d[0] = fr[9 * o + 3 * row];
                d[1] = fr[9 * o + 3 * row + 1];
                d[2] = fr[9 * o + 3 * row + 2];
                d[3] = row == 0 ? wf[o] : 0.0;
            }
        t.n_orient = 3 * nf;
    } else if (m.kind == SAS_CYLINDER || m.kind == SAS_ELLIPSOID || m.kind == SAS_CAPPED_CYLINDER ||
               m.kind == SAS_BARBELL || shelled_cylinder(m.kind) || m.kind == SAS_CORE_SHELL_ELLIPSOID) {
        const int nmax = (int)(m.n_gamma * m.n_psi);
        std::vector<double> c((size_t)3 * std::max(nmax, 1)), wo(std::max(nmax, 1));
        const int no = m.isotropic == 2
                           ? uniform_angle_nodes((int)m.n_gamma, (int)m.n_psi, c.data(), wo.data())
                           : orientation_nodes(m.axis_theta, m.axis_phi, m.sigma_orient, (int)m.n_gamma,
                                               (int)m.n_psi, (int)m.isotropic, c.data(), wo.data());
        t.orient.assign((size_t)no * SAS_ORIENT_STRIDE, 0.0);
        for (int i = 0; i < no; ++i) {
            t.orient[(size_t)i * 4 + 0] = c[3 * i];
            t.orient[(size_t)i * 4 + 1] = c[3 * i + 1];
            t.orient[(size_t)i * 4 + 2] = c[3 * i + 2];
            t.orient[(size_t)i * 4 + 3] = wo[i];
        }
        t.n_orient = no;
    } else {
        t.orient.assign(SAS_ORIENT_STRIDE, 0.0);
        t.n_orient = 0;
    }
    t.n_rad = t.n_poly;
    t.n_tab = 0;
    t.n_cap = 0;
    if (m.kind == SAS_CAPPED_CYLINDER || m.kind == SAS_BARBELL) {
        // the cap slices at depth R u_j below the tip, u_j Gauss-Legendre on
        // [0, H / R]: z_j = L/2 + H - R u_j, rho_j^2 = R^2 u_j (2 - u_j),
        // c_j = 2 pi R^3 w_j u_j (2 - u_j); two slices per row behind the nodes
        const int nc = (int)m.n_cap;
        const double r0 = m.radius, R = m.radius_polar, H = cap_height(m);
        std::vector<double> gx(nc), gw(nc);
        gauss_legendre(nc, gx.data(), gw.data());
        const int rows = (nc + 1) / 2;
        t.poly.resize((size_t)(t.n_poly + rows) * SAS_POLY_STRIDE, 0.0);
        double* cap = t.poly.data() + (size_t)t.n_poly * SAS_POLY_STRIDE;
        double rho2max = r0 * r0;
        for (int j = 0; j < nc; ++j) {
            const double u = 0.5 * (H / R) * (1.0 + gx[j]), wj = 0.5 * (H / R) * gw[j];
            const double v = u * (2.0 - u);
            cap[4 * j] = 0.5 * m.length + H - R * u;
            cap[4 * j + 1] = R * R * v;
            cap[4 * j + 2] = 2.0 * pi * R * R * R * wj * v;
            rho2max = std::fmax(rho2max, R * R * v);
        }
        t.n_poly += rows;
        t.n_cap = nc;
        t.cap_body = pi * r0 * r0 * m.length;
        t.cap_r2 = r0 * r0;
        t.cap_rho2max = rho2max;
    }
    if (m.kind == SAS_CYLINDER && m.radial_table && m.sampling == SAS_QUADRATURE && q_max > 0.0) {
        // the polydisperse radial sum depends on x = q_AB rbar alone: tabulate
        // G(x) with h G'(x), doubling the grid until the cubic Hermite error at
        // the midpoints is at most 1e-7 G(0) (FP64 models: 1e-13); stored
        // behind the nodes
        const double rbar = m.radius, xmax = q_max * rbar;
        std::vector<double> rr(npoly), ww(npoly);
        for (int i = 0; i < npoly; ++i) {
            rr[i] = t.poly[(size_t)i * SAS_POLY_STRIDE + 2];   // r
            ww[i] = npoly == 1 ? 1.0 : w[i];
        }
        const double F0 = (m.sld - m.sld_solvent) * pi * rbar * rbar * m.length;
        std::vector<double> G, D;
        double err = 0.0, g0 = 0.0;
        const double target = m.precision == SAS_FP64 ? 1e-13 : 1e-7;   // relative to G(0)
        int n = 1024;
        for (; n <= SAS_MAX_RADIAL_TABLE; n *= 2) {
            G.assign(n, 0.0);
            D.assign(n, 0.0);
            err = cylinder_radial_table(rr.data(), ww.data(), npoly, rbar, xmax, n, G.data(), D.data());
            g0 = G[0];
            if (err <= target * g0) break;
        }
        if (n <= SAS_MAX_RADIAL_TABLE) {
            const int rows = (2 * n + SAS_POLY_STRIDE - 1) / SAS_POLY_STRIDE;
            t.poly.resize((size_t)(npoly + rows) * SAS_POLY_STRIDE, 0.0);
            double* tab = t.poly.data() + (size_t)npoly * SAS_POLY_STRIDE;
            for (int k = 0; k < n; ++k) {
                tab[2 * k] = G[k];
                tab[2 * k + 1] = D[k];
            }
            t.n_poly = npoly + rows;
            t.n_tab = n;
            t.tab_inv_h = (double)(n - 1) / xmax;
            t.tab_xmax = xmax;
            t.tab_c0 = F0 * F0;
            t.tab_rbar = rbar;
            t.tab_err = err / g0;
        }
    }
    if (m.sampling == SAS_PER_EVENT) {
        // per-event histories draw their own radius and axis: the nodes only
        // gave <V> above, and one node keeps the kernels' staging minimal
        // (the cap slices of the capped kinds move up behind it)
        const int cap_rows = t.n_poly - t.n_rad;
        if (t.n_cap > 0 && t.n_rad > 1)
            std::copy(t.poly.begin() + (size_t)t.n_rad * SAS_POLY_STRIDE, t.poly.end(),
                      t.poly.begin() + SAS_POLY_STRIDE);
        t.poly.resize((size_t)(1 + (t.n_cap > 0 ? cap_rows : 0)) * SAS_POLY_STRIDE);
        t.n_poly = 1 + (t.n_cap > 0 ? cap_rows : 0);
        t.n_rad = 1;
        if (t.n_orient > 0) {
            const int rows = axes3_kind(m.kind) ? 3 : 1;
            t.orient.resize((size_t)rows * SAS_ORIENT_STRIDE);
            t.n_orient = rows;
        }
    }
    t.half_length = 0.5 * m.length;
    t.rp2 = m.radius_polar * m.radius_polar;
    t.sq_kind = (int)m.sq_kind;
    t.sq_2r = 2.0 * m.sq_radius;
    t.sq_24phi = 24.0 * m.sq_fraction;
    t.sq_switch = 3.0;
    t.sq_series.assign(SAS_SQ_NSER, 0.0);
    if (m.sq_kind == SAS_SQ_HARD_SPHERE_PY)
        py_constants(m.sq_fraction, &t.sq_alpha, &t.sq_beta, &t.sq_gamma, t.sq_series.data(), SAS_SQ_NSER);
    else
        t.sq_alpha = t.sq_beta = t.sq_gamma = 0.0;
    if (m.sq_kind == SAS_SQ_HAYTER_MSA) {
        const msa::Reduced r = msa::reduce(m.sq_radius, m.sq_fraction, m.sq_charge, m.sq_temperature, m.sq_salt,
                                           m.sq_dielectric);
        msa::Table tab;
        std::string err;
        // past 1/angstrom where the grid allows, else past the instrument's largest |Q|
        if (!msa::build_table(r, std::max(1.0, 1.05 * q_max), tab, err) &&
            !msa::build_table(r, 1.05 * q_max, tab, err))
            return fail(SAS_ERR_ARG, err.c_str());
        t.sq_dq = tab.dq;
        t.sq_rescale = tab.s_rescale;
        t.sq_contact = tab.contact;
        t.sq_tab = tab.sd;
        for (size_t j = 1; j < t.sq_tab.size(); j += 2) t.sq_tab[j] *= tab.dq;   // h dS/dQ
    }
    return SAS_OK;
}

template <typename T>
ModelConst<T> model_const(const sas_model_desc& m, const ModelTables& t)
{
    ModelConst<T> c;
    std::memset(&c, 0, sizeof(c));
    c.kind = (int)m.kind;
    c.sq_kind = t.sq_kind;
    c.n_poly = t.n_poly;
    c.n_orient = t.n_orient;
    c.scale = (T)t.scale;
    c.half_length = (T)t.half_length;
    c.shell = (T)m.thickness;
    c.rp2 = (T)t.rp2;
    c.fuzz2 = (T)(m.kind == SAS_SPHERE ? m.fuzziness * m.fuzziness * 1.4426950408889634 : 0.0);   // log2(e)
    c.sq_2r = (T)t.sq_2r;
    c.sq_24phi = (T)t.sq_24phi;
    c.sq_alpha = (T)t.sq_alpha;
    c.sq_beta = (T)t.sq_beta;
    c.sq_gamma = (T)t.sq_gamma;
    c.sq_switch = (T)t.sq_switch;
    for (int k = 0; k < SAS_SQ_NSER; ++k) c.sq_series[k] = (T)t.sq_series[k];
    c.sq_tab = nullptr;   // set once the table is on the device
    c.sq_n = (int)(t.sq_tab.size() / 2);
    c.sq_inv_dq = (T)(t.sq_dq > 0.0 ? 1.0 / t.sq_dq : 0.0);
    c.event = m.sampling == SAS_PER_EVENT ? 1 : 0;
    c.orient_mode = (m.kind == SAS_CYLINDER || m.kind == SAS_ELLIPSOID || m.kind == SAS_CAPPED_CYLINDER ||
                     m.kind == SAS_BARBELL || shelled_cylinder(m.kind) || m.kind == SAS_CORE_SHELL_ELLIPSOID)
                        ? (int)m.isotropic : 0;
    c.ev_r = (T)m.radius;
    c.ev_p = (T)(m.poly_dist == SAS_POLY_GAUSSIAN ? m.poly : 0.0);
    const double lo = c.ev_p > (T)0 ? 0.5 * std::erfc(1.0 / (m.poly * std::sqrt(2.0))) : 0.0;
    c.ev_lo = (T)lo;
    c.ev_1mlo = (T)(1.0 - lo);
    // contrasts of the per-event amplitudes (the shelled cylinders use ev_k)
    const bool shelled = m.kind == SAS_CORE_SHELL || m.kind == SAS_CORE_SHELL_ELLIPSOID;
    c.ev_c1 = (T)(shelled ? m.sld - m.sld_shell : m.sld - m.sld_solvent);
    c.ev_c2 = (T)(shelled ? m.sld_shell - m.sld_solvent : 0.0);
    c.ev_len = (T)m.length;
    c.ev_rp = (T)m.radius_polar;
    c.ev_axis[0] = (T)(std::sin(m.axis_theta) * std::cos(m.axis_phi));
    c.ev_axis[1] = (T)(std::sin(m.axis_theta) * std::sin(m.axis_phi));
    c.ev_axis[2] = (T)std::cos(m.axis_theta);
    c.ax_a = (T)m.radius;
    c.ax_b = (T)m.radius_b;
    c.ax_c = (T)(m.kind == SAS_ELLIPTICAL_CYLINDER ? 0.5 * m.length : m.radius_polar);
    if (m.kind == SAS_HOLLOW_RECTANGULAR_PRISM) {
        const double t = m.thickness;
        c.ax_ai = (T)(m.radius - t);
        c.ax_bi = (T)(m.radius_b - t);
        c.ax_ci = (T)(m.radius_polar - t);
        c.ax_v = (T)(m.radius * m.radius_b * m.radius_polar);
        c.ax_vi = (T)((m.radius - t) * (m.radius_b - t) * (m.radius_polar - t));
    }
    {
        double f[9];
        frame_of(m.axis_theta, m.axis_phi, m.axis_psi, f);
        for (int k = 0; k < 6; ++k) c.ev_frame[k] = (T)f[k];
    }
    if (axes3_kind(m.kind))
        c.orient_mode = (int)m.isotropic;
    c.n_rad = t.n_rad;
    c.n_tab = t.n_tab;
    c.n_cap = t.n_cap;
    c.half_length_o = (T)(0.5 * m.length + (shelled_cylinder(m.kind) ? face_layer(m) : 0.0));
    if (shelled_cylinder(m.kind)) {
        double d[4];
        shelled_contrasts(m, d);
        for (int k = 0; k < 4; ++k) c.ev_k[k] = (T)d[k];
    }
    c.function = (int)m.function;
    if (m.kind == SAS_SHAPE_INDEPENDENT) {
        const double p0 = m.f_p0, p1 = m.f_p1;
        switch (m.function) {
        case SAS_FN_GUINIER: c.f_a = (T)(p0 * p0 / 3.0); break;
        case SAS_FN_GAUSS_COIL:
        case SAS_FN_LORENTZ:
        case SAS_FN_DAB: c.f_a = (T)(p0 * p0); break;
        case SAS_FN_POWER_LAW: c.f_a = (T)p0; break;
        case SAS_FN_GAUSS_PEAK: c.f_a = (T)p0; c.f_b = (T)(0.5 / (p1 * p1)); break;
        case SAS_FN_PEAK_LORENTZ: c.f_a = (T)p0; c.f_b = (T)(1.0 / p1); break;
        case SAS_FN_TWO_POWER_LAW:
            c.f_a = (T)p0;
            c.f_b = (T)p1;
            c.f_c = (T)m.f_p2;
            c.f_d = (T)std::pow(p0, m.f_p2 - p1);
            break;
        case SAS_FN_GUINIER_POROD: {
            const double sd = p1, mp = m.f_p2;
            const double q1 = std::sqrt((mp - sd) * (3.0 - sd) / 2.0) / p0;
            c.f_a = (T)(p0 * p0 / (3.0 - sd));
            c.f_b = (T)sd;
            c.f_c = (T)mp;
            c.f_d = (T)q1;
            c.f_e = (T)(std::pow(q1, mp - sd) * std::exp(-(mp - sd) / 2.0));
            break;
        }
        case SAS_FN_GAUSS_LORENTZ_GEL:
            c.f_a = (T)(0.5 * p0 * p0);
            c.f_b = (T)(p1 * p1);
            c.f_c = (T)m.f_p2;
            break;
        case SAS_FN_POLY_GAUSS_COIL: c.f_a = (T)(p0 * p0 / (1.0 + 2.0 * p1)); c.f_b = (T)p1; break;
        case SAS_FN_STAR_POLYMER: c.f_a = (T)(p0 * p0 * p1 / (3.0 * p1 - 2.0)); c.f_b = (T)p1; break;
        case SAS_FN_MASS_FRACTAL: c.f_a = (T)p0; c.f_b = (T)(p1 - 1.0); c.f_c = (T)m.f_p2; break;
        case SAS_FN_FRACTAL:   // f_d = Gamma(D + 1) (xi / R0)^D
            c.f_a = (T)p0;
            c.f_b = (T)(p1 - 1.0);
            c.f_c = (T)m.f_p2;
            c.f_d = (T)(std::tgamma(p1 + 1.0) * std::pow(m.f_p2 / p0, p1));
            break;
        case SAS_FN_SPINODAL: c.f_a = (T)(1.0 / p0); c.f_b = (T)p1; c.f_c = (T)(0.5 * p1); c.f_d = (T)(1.0 + 0.5 * p1); break;
        case SAS_FN_LINEAR_PEARLS:   // R, centre distance d, N, 1 / N^2
            c.f_a = (T)p0;
            c.f_b = (T)(2.0 * p0 + p1);
            c.f_c = (T)m.f_p2;
            c.f_d = (T)(1.0 / (m.f_p2 * m.f_p2));
            break;
        case SAS_FN_POLYMER_EXCL_VOLUME: {   // U = Q^2 f_a; m, Gamma(m / 2), Gamma(m)
            const double nu = 1.0 / p1;
            c.f_a = (T)(p0 * p0 * (2.0 * nu + 1.0) * (2.0 * nu + 2.0) / 6.0);
            c.f_b = (T)p1;
            c.f_c = (T)std::tgamma(0.5 * p1);
            c.f_d = (T)std::tgamma(p1);
            break;
        }
        default: c.f_a = (T)m.f_p0; c.f_b = (T)m.f_p1; c.f_c = (T)m.f_p2; break;
        }
    }
    c.rp_o = (T)(m.radius_polar + (m.kind == SAS_CORE_SHELL_ELLIPSOID ? m.thickness_face : 0.0));
    c.rp2o = c.rp_o * c.rp_o;
    c.cap_body = (T)t.cap_body;
    c.cap_r2 = (T)t.cap_r2;
    c.cap_rho2max = (T)t.cap_rho2max;
    c.tab_inv_h = (T)t.tab_inv_h;
    c.tab_xmax = (T)t.tab_xmax;
    c.tab_c0 = (T)t.tab_c0;
    c.tab_rbar = (T)t.tab_rbar;
    c.att.n = t.att_n;
    if (t.att_n > 1) {
        c.att.t_mul = (T)(2.0 / (t.att_lmax - t.att_lmin));
        c.att.t_add = (T)(-(t.att_lmin + t.att_lmax) / (t.att_lmax - t.att_lmin));
    }
    for (int j = 0; j < t.att_n; ++j) c.att.c[j] = (T)t.att_c[j];
    return c;
}

template <typename T>
InstConst<T> inst_const(const sas_instrument& in)
{
    InstConst<T> c;
    c.lambda0 = (T)in.lambda0;
    c.dlambda = (T)in.dlambda_rel;
    c.ap1_r = (T)in.ap1_radius;
    c.ap1_z = (T)in.ap1_z;
    c.ap2_r = (T)in.ap2_radius;
    c.ap2_z = (T)in.ap2_z;
    c.hx = (T)in.sample_half_x;
    c.hy = (T)in.sample_half_y;
    c.thick = (T)in.sample_thickness;
    c.mu = (T)in.mu;
    c.det_z = (T)in.det_distance;
    c.px = (T)in.pixel_x;
    c.py = (T)in.pixel_y;
    c.half_wx = (T)(0.5 * (double)in.nx * in.pixel_x);
    c.half_wy = (T)(0.5 * (double)in.ny * in.pixel_y);
    c.area = (T)((double)in.nx * in.pixel_x * (double)in.ny * in.pixel_y);
    c.two_pi = (T)(2.0 * M_PI);
    c.nx = (int)in.nx;
    c.ny = (int)in.ny;
    return c;
}

template ModelConst<float> model_const<float>(const sas_model_desc&, const ModelTables&);
template ModelConst<double> model_const<double>(const sas_model_desc&, const ModelTables&);
template InstConst<float> inst_const<float>(const sas_instrument&);
template InstConst<double> inst_const<double>(const sas_instrument&);

sas_status validate_instrument(const sas_instrument* in)
{
    if (!in) return fail(SAS_ERR_ARG, "instrument is NULL");
    if (!finite_all({in->lambda0, in->dlambda_rel, in->ap1_radius, in->ap1_z, in->ap2_radius,
                     in->ap2_z, in->sample_half_x, in->sample_half_y, in->sample_thickness, in->mu,
                     in->det_distance, in->pixel_x, in->pixel_y}))
        return fail(SAS_ERR_ARG, "instrument has a non-finite value");
    if (in->lambda0 <= 0.0) return fail(SAS_ERR_ARG, "lambda0 must be > 0");
    if (in->dlambda_rel < 0.0 || in->dlambda_rel >= 1.0) return fail(SAS_ERR_ARG, "dlambda_rel must be in [0, 1)");
    if (in->ap1_radius < 0.0 || in->ap2_radius < 0.0) return fail(SAS_ERR_ARG, "aperture radii must be >= 0");
    if (!(in->ap1_z < in->ap2_z)) return fail(SAS_ERR_ARG, "ap1_z must be upstream of ap2_z");
    if (in->ap2_z > 0.0) return fail(SAS_ERR_ARG, "ap2_z must be <= 0 (sample front face)");
    if (in->sample_half_x <= 0.0 || in->sample_half_y <= 0.0 || in->sample_thickness <= 0.0)
        return fail(SAS_ERR_ARG, "sample dimensions must be > 0");
    if (in->mu < 0.0) return fail(SAS_ERR_ARG, "mu must be >= 0");
    if (!(in->det_distance > in->sample_thickness)) return fail(SAS_ERR_ARG, "detector must be behind the sample");
    if (in->pixel_x <= 0.0 || in->pixel_y <= 0.0) return fail(SAS_ERR_ARG, "pixel sizes must be > 0");
    if (in->nx < 1 || in->ny < 1 || in->nx > 4096 || in->ny > 4096)
        return fail(SAS_ERR_ARG, "nx, ny must be in [1, 4096]");
    return SAS_OK;
}

sas_status validate_model(const sas_model_desc* m)
{
    if (!m) return fail(SAS_ERR_ARG, "model is NULL");
    if (m->kind < 0 || m->kind > 14) return fail(SAS_ERR_ARG, "unknown model kind");
    if (!(m->fuzziness >= 0.0) || !std::isfinite(m->fuzziness) || (m->kind != SAS_SPHERE && m->fuzziness != 0.0))
        return fail(SAS_ERR_ARG, "fuzziness must be finite, >= 0, and 0 for every kind but the sphere");
    if (m->kind == SAS_SHAPE_INDEPENDENT) {
        if (m->function < SAS_FN_GUINIER || m->function > SAS_FN_LINEAR_PEARLS)
            return fail(SAS_ERR_ARG, "unknown shape-independent function");
        if (!finite_all({m->f_scale, m->f_p0, m->f_p1, m->f_p2}) || m->f_scale < 0.0)
            return fail(SAS_ERR_ARG, "f_scale must be finite and >= 0, f_p0..f_p2 finite");
        const int64_t fn = m->function;
        if ((fn <= SAS_FN_DAB && !(m->f_p0 > 0.0)) || (fn == SAS_FN_GAUSS_PEAK && !(m->f_p1 > 0.0)))
            return fail(SAS_ERR_ARG, "Rg, xi and sigma must be > 0");
        if (fn == SAS_FN_TEUBNER_STREY &&
            !(m->f_p0 > 0.0 && m->f_p2 >= 0.0 && (m->f_p1 >= 0.0 || m->f_p1 * m->f_p1 < 4.0 * m->f_p0 * m->f_p2)))
            return fail(SAS_ERR_ARG, "Teubner-Strey needs a2 > 0, c2 >= 0 and a2 + c1 Q^2 + c2 Q^4 > 0");
        if (fn == SAS_FN_PEAK_LORENTZ && !(m->f_p1 > 0.0))
            return fail(SAS_ERR_ARG, "peak Lorentz needs a width B > 0");
        if (fn == SAS_FN_TWO_POWER_LAW && !(m->f_p0 > 0.0))
            return fail(SAS_ERR_ARG, "two power laws need a crossover Qc > 0");
        if (fn == SAS_FN_GUINIER_POROD && !(m->f_p0 > 0.0 && m->f_p1 >= 0.0 && m->f_p1 < 3.0 && m->f_p2 > m->f_p1))
            return fail(SAS_ERR_ARG, "Guinier-Porod needs Rg > 0, 0 <= s < 3 and m > s");
        if (fn == SAS_FN_GAUSS_LORENTZ_GEL && !(m->f_p0 > 0.0 && m->f_p1 > 0.0 && m->f_p2 >= 0.0))
            return fail(SAS_ERR_ARG, "Gauss-Lorentz gel needs Xi > 0, xi > 0 and r >= 0");
        if (fn == SAS_FN_POLY_GAUSS_COIL && !(m->f_p0 > 0.0 && m->f_p1 >= 0.0))
            return fail(SAS_ERR_ARG, "polydisperse coil needs Rg > 0 and U = Mw/Mn - 1 >= 0");
        if (fn == SAS_FN_STAR_POLYMER && !(m->f_p0 > 0.0 && m->f_p1 >= 1.0))
            return fail(SAS_ERR_ARG, "star polymer needs Rg > 0 and at least one arm");
        if ((fn == SAS_FN_MASS_FRACTAL || fn == SAS_FN_FRACTAL) &&
            !((fn == SAS_FN_FRACTAL ? m->f_p0 > 0.0 : m->f_p0 >= 0.0) && m->f_p1 > 1.0 && m->f_p1 < 6.0 &&
              m->f_p2 > 0.0))
            return fail(SAS_ERR_ARG, "fractals need a sphere radius (> 0 for Teixeira's, >= 0 for the mass "
                                     "fractal), 1 < D < 6 and a cutoff xi > 0");
        if (fn == SAS_FN_FRACTAL && !std::isfinite(std::tgamma(m->f_p1 + 1.0) * std::pow(m->f_p2 / m->f_p0, m->f_p1)))
            return fail(SAS_ERR_ARG, "fractal: Gamma(D + 1) (xi / R0)^D overflows");
        if (fn == SAS_FN_SPINODAL && !(m->f_p0 > 0.0 && m->f_p1 > 0.0))
            return fail(SAS_ERR_ARG, "spinodal needs Qmax > 0 and an exponent g > 0");
        if (fn == SAS_FN_LINEAR_PEARLS &&
            !(m->f_p0 > 0.0 && m->f_p1 >= 0.0 && m->f_p2 >= 1.0 && m->f_p2 <= 1000.0 && m->f_p2 == std::floor(m->f_p2)))
            return fail(SAS_ERR_ARG, "linear pearls need R > 0, a separation s >= 0 and an integer N in [1, 1000]");
        if (fn == SAS_FN_POLYMER_EXCL_VOLUME && !(m->f_p0 > 0.0 && m->f_p1 > 1.0 && m->f_p1 < 6.0))
            return fail(SAS_ERR_ARG, "excluded-volume chain needs Rg > 0 and a Porod exponent 1 < m < 6");
        if (m->sq_kind != SAS_SQ_NONE || m->sampling != SAS_QUADRATURE || m->self_attenuation != 0)
            return fail(SAS_ERR_ARG, "shape-independent laws take no S(Q), per-event sampling or self-attenuation");
    }
    if (m->kind == SAS_ELLIPTICAL_CYLINDER && (!(m->radius_b > 0.0) || !(m->length > 0.0) ||
                                               !std::isfinite(m->radius_b) || !std::isfinite(m->axis_psi)))
        return fail(SAS_ERR_ARG, "elliptical cylinder needs radius, radius_b, length > 0 and a finite axis_psi");
    if (m->kind == SAS_HOLLOW_RECTANGULAR_PRISM &&
        !(m->thickness > 0.0 && m->thickness < std::fmin(m->radius, std::fmin(m->radius_b, m->radius_polar))))
        return fail(SAS_ERR_ARG, "hollow rectangular prism needs 0 < thickness < every half-edge");
    if (shelled_cylinder(m->kind) || m->kind == SAS_CORE_SHELL_ELLIPSOID) {
        if (!std::isfinite(m->thickness_face) || !std::isfinite(m->sld_face) || m->thickness < 0.0 ||
            m->thickness_face < 0.0)
            return fail(SAS_ERR_ARG, "shell thicknesses must be finite and >= 0");
        if (m->kind != SAS_CORE_SHELL_ELLIPSOID && !(m->length > 0.0)) return fail(SAS_ERR_ARG, "length must be > 0");
        if (m->kind == SAS_HOLLOW_CYLINDER && !(m->thickness > 0.0))
            return fail(SAS_ERR_ARG, "hollow cylinder needs a wall thickness > 0");
        if (m->kind == SAS_CORE_SHELL_ELLIPSOID && !(m->radius_polar > 0.0))
            return fail(SAS_ERR_ARG, "radius_polar must be > 0");
    }
    if (m->kind == SAS_CAPPED_CYLINDER || m->kind == SAS_BARBELL) {
        if (!std::isfinite(m->length) || !std::isfinite(m->radius_polar) || m->length < 0.0 ||
            !(m->radius_polar >= m->radius))
            return fail(SAS_ERR_ARG, "capped cylinder and barbell need length >= 0 and radius_polar >= radius");
        if (m->n_cap < 1 || m->n_cap > SAS_MAX_CAP_NODES) return fail(SAS_ERR_ARG, "n_cap must be in [1, 64]");
    }
    const bool axes3 = axes3_kind(m->kind);
    const bool boxlike = axes3 && m->kind != SAS_ELLIPTICAL_CYLINDER;
    if (boxlike && (!(m->radius_b > 0.0) || !(m->radius_polar > 0.0) || !std::isfinite(m->radius_b) ||
                    !std::isfinite(m->axis_psi)))
        return fail(SAS_ERR_ARG, "3-axis models need radius, radius_b, radius_polar > 0 and a finite axis_psi");
    if (axes3 && (m->n_rot < 1 || m->n_rot > SAS_MAX_ORIENT_SIDE)) return fail(SAS_ERR_ARG, "n_rot must be in [1, 128]");
    if (axes3 && m->isotropic != 0 && m->n_gamma * m->n_psi * m->n_rot > (1 << 17))
        return fail(SAS_ERR_ARG, "n_gamma * n_psi * n_rot must be <= 131072");
    if (m->sq_kind != SAS_SQ_NONE && m->sq_kind != SAS_SQ_HARD_SPHERE_PY && m->sq_kind != SAS_SQ_HAYTER_MSA)
        return fail(SAS_ERR_ARG, "unknown S(Q) kind");
    if (m->sq_kind == SAS_SQ_HAYTER_MSA &&
        (!(m->sq_radius > 0.0) || !(m->sq_fraction > 0.0 && m->sq_fraction < 0.45) || !(m->sq_charge >= 0.0) ||
         !(m->sq_temperature > 0.0) || !(m->sq_salt >= 0.0) || !(m->sq_dielectric > 0.0) ||
         !std::isfinite(m->sq_charge) || !std::isfinite(m->sq_salt) || !std::isfinite(m->sq_temperature) ||
         !std::isfinite(m->sq_dielectric)))
        return fail(SAS_ERR_ARG, "Hayter MSA needs sq_radius > 0, 0 < sq_fraction < 0.45, sq_charge >= 0, "
                                 "sq_temperature > 0, sq_salt >= 0 and sq_dielectric > 0");
    if (m->precision != SAS_FP32 && m->precision != SAS_FP64) return fail(SAS_ERR_ARG, "unknown precision");
    if (m->n_poly < 1 || m->n_poly > SAS_MAX_POLY) return fail(SAS_ERR_ARG, "n_poly must be in [1, 64]");
    if (m->n_gamma < 1 || m->n_gamma > SAS_MAX_ORIENT_SIDE || m->n_psi < 1 || m->n_psi > SAS_MAX_ORIENT_SIDE)
        return fail(SAS_ERR_ARG, "n_gamma, n_psi must be in [1, 128]");
    if (!finite_all({m->radius, m->thickness, m->length, m->radius_polar, m->sld, m->sld_shell,
                     m->sld_solvent, m->volume_fraction, m->poly, m->sigma_orient, m->axis_theta,
                     m->axis_phi, m->sq_radius, m->sq_fraction}))
        return fail(SAS_ERR_ARG, "model has a non-finite value");
    if (m->radius <= 0.0 && m->kind != SAS_SHAPE_INDEPENDENT) return fail(SAS_ERR_ARG, "radius must be > 0");
    if (m->kind == SAS_CORE_SHELL && m->thickness < 0.0) return fail(SAS_ERR_ARG, "thickness must be >= 0");
    if (m->kind == SAS_CYLINDER && m->length <= 0.0) return fail(SAS_ERR_ARG, "length must be > 0");
    if (m->kind == SAS_ELLIPSOID && m->radius_polar <= 0.0) return fail(SAS_ERR_ARG, "radius_polar must be > 0");
    if (m->volume_fraction < 0.0) return fail(SAS_ERR_ARG, "volume_fraction must be >= 0");
    if (m->poly < 0.0 || m->poly >= 1.0) return fail(SAS_ERR_ARG, "poly must be in [0, 1)");
    if (m->sigma_orient < 0.0) return fail(SAS_ERR_ARG, "sigma_orient must be >= 0");
    if (m->isotropic < 0 || m->isotropic > 2) return fail(SAS_ERR_ARG, "isotropic must be 0, 1 or 2");
    if (m->sampling != SAS_QUADRATURE && m->sampling != SAS_PER_EVENT) return fail(SAS_ERR_ARG, "unknown sampling");
    if (m->poly_dist != SAS_POLY_SCHULZ && m->poly_dist != SAS_POLY_GAUSSIAN)
        return fail(SAS_ERR_ARG, "unknown poly_dist");
    if (m->radial_table != 0 && m->radial_table != 1) return fail(SAS_ERR_ARG, "radial_table must be 0 or 1");
    if (m->self_attenuation != 0 && m->self_attenuation != 1)
        return fail(SAS_ERR_ARG, "self_attenuation must be 0 or 1");
    if (m->self_attenuation && m->sampling != SAS_QUADRATURE)
        return fail(SAS_ERR_ARG, "self_attenuation needs the model's deterministic dSigma/dOmega: sampling "
                                 "SAS_QUADRATURE");
    if (m->sampling == SAS_PER_EVENT) {
        if (m->poly > 0.0 && m->poly_dist != SAS_POLY_GAUSSIAN)
            return fail(SAS_ERR_ARG, "per-event sampling draws Gaussian radii (Sec. II.B): set poly_dist to "
                                     "SAS_POLY_GAUSSIAN or poly to 0");
        if ((m->kind >= SAS_CYLINDER) && m->isotropic == 0 && m->sigma_orient > 0.0)
            return fail(SAS_ERR_ARG, "per-event axes are uniform on the sphere (isotropic 1), in the angles "
                                     "(isotropic 2) or fixed (sigma_orient 0); the Gaussian cap is a quadrature option");
    }
    if (m->sq_kind == SAS_SQ_HARD_SPHERE_PY) {
        if (m->sq_radius <= 0.0) return fail(SAS_ERR_ARG, "sq_radius must be > 0");
        if (m->sq_fraction < 0.0 || m->sq_fraction >= 0.74) return fail(SAS_ERR_ARG, "sq_fraction must be in [0, 0.74)");
    }
    return SAS_OK;
}

}  // namespace sas

using namespace sas;

struct sas_experiment {
    sas_instrument inst;
    int device = 0, sm_count = 0, smem_optin = 0;
    cudaStream_t stream = nullptr;
    uint32_t exp_id = 0;
    double* d_sum_w = nullptr;
    double* d_sum_w2 = nullptr;
    unsigned long long* d_count = nullptr;
    double* d_trans = nullptr;
    bool has_model = false;
    sas_model_desc model;
    ModelTables tables;
    void* d_poly = nullptr;
    void* d_orient = nullptr;
    void* d_sqtab = nullptr;   // Hayter-Penfold S(Q) table (model precision)
    ModelConst<float> mcf;
    ModelConst<double> mcd;
    InstConst<float> icf;
    InstConst<double> icd;
    LaunchCfg cfg;
    int stage_orient = 0;
    // learned surrogate (models of its kind in its training box)
    const sas_surrogate* sur = nullptr;
    WorkItem* d_items = nullptr;
    uint32_t* d_prefix = nullptr;      // 256-history pairs before each item
    size_t items_cap = 0;
    uint64_t* d_seed = nullptr;
    sur::SurExp* d_sexp = nullptr;
    BatchExp* d_bexp = nullptr;
    unsigned long long* d_fallbacks = nullptr;
};

namespace {

template <typename T>
cudaError_t dispatch_trace(sas_experiment* e, const TraceParams<T>& P, int* grid)
{
    switch (e->model.kind) {
    case SAS_SPHERE: return Launcher<T, SAS_SPHERE>::trace(P, e->cfg, e->sm_count, e->stream, grid);
    case SAS_CORE_SHELL: return Launcher<T, SAS_CORE_SHELL>::trace(P, e->cfg, e->sm_count, e->stream, grid);
    case SAS_CYLINDER: return Launcher<T, SAS_CYLINDER>::trace(P, e->cfg, e->sm_count, e->stream, grid);
    case SAS_TRIAXIAL_ELLIPSOID: return Launcher<T, SAS_TRIAXIAL_ELLIPSOID>::trace(P, e->cfg, e->sm_count, e->stream, grid);
    case SAS_PARALLELEPIPED: return Launcher<T, SAS_PARALLELEPIPED>::trace(P, e->cfg, e->sm_count, e->stream, grid);
    case SAS_CAPPED_CYLINDER: return Launcher<T, SAS_CAPPED_CYLINDER>::trace(P, e->cfg, e->sm_count, e->stream, grid);
    case SAS_BARBELL: return Launcher<T, SAS_BARBELL>::trace(P, e->cfg, e->sm_count, e->stream, grid);
    case SAS_CORE_SHELL_CYLINDER: return Launcher<T, SAS_CORE_SHELL_CYLINDER>::trace(P, e->cfg, e->sm_count, e->stream, grid);
    case SAS_HOLLOW_CYLINDER: return Launcher<T, SAS_HOLLOW_CYLINDER>::trace(P, e->cfg, e->sm_count, e->stream, grid);
    case SAS_CORE_SHELL_ELLIPSOID: return Launcher<T, SAS_CORE_SHELL_ELLIPSOID>::trace(P, e->cfg, e->sm_count, e->stream, grid);
    case SAS_CORE_SHELL_BICELLE: return Launcher<T, SAS_CORE_SHELL_BICELLE>::trace(P, e->cfg, e->sm_count, e->stream, grid);
    case SAS_ELLIPTICAL_CYLINDER: return Launcher<T, SAS_ELLIPTICAL_CYLINDER>::trace(P, e->cfg, e->sm_count, e->stream, grid);
    case SAS_HOLLOW_RECTANGULAR_PRISM: return Launcher<T, SAS_HOLLOW_RECTANGULAR_PRISM>::trace(P, e->cfg, e->sm_count, e->stream, grid);
    case SAS_SHAPE_INDEPENDENT: return Launcher<T, SAS_SHAPE_INDEPENDENT>::trace(P, e->cfg, e->sm_count, e->stream, grid);
    default: return Launcher<T, SAS_ELLIPSOID>::trace(P, e->cfg, e->sm_count, e->stream, grid);
    }
}

template <typename T>
cudaError_t dispatch_records(sas_experiment* e, const TraceParams<T>& P)
{
    switch (e->model.kind) {
    case SAS_SPHERE: return Launcher<T, SAS_SPHERE>::records(P, e->stream);
    case SAS_CORE_SHELL: return Launcher<T, SAS_CORE_SHELL>::records(P, e->stream);
    case SAS_CYLINDER: return Launcher<T, SAS_CYLINDER>::records(P, e->stream);
    case SAS_TRIAXIAL_ELLIPSOID: return Launcher<T, SAS_TRIAXIAL_ELLIPSOID>::records(P, e->stream);
    case SAS_PARALLELEPIPED: return Launcher<T, SAS_PARALLELEPIPED>::records(P, e->stream);
    case SAS_CAPPED_CYLINDER: return Launcher<T, SAS_CAPPED_CYLINDER>::records(P, e->stream);
    case SAS_BARBELL: return Launcher<T, SAS_BARBELL>::records(P, e->stream);
    case SAS_CORE_SHELL_CYLINDER: return Launcher<T, SAS_CORE_SHELL_CYLINDER>::records(P, e->stream);
    case SAS_HOLLOW_CYLINDER: return Launcher<T, SAS_HOLLOW_CYLINDER>::records(P, e->stream);
    case SAS_CORE_SHELL_ELLIPSOID: return Launcher<T, SAS_CORE_SHELL_ELLIPSOID>::records(P, e->stream);
    case SAS_CORE_SHELL_BICELLE: return Launcher<T, SAS_CORE_SHELL_BICELLE>::records(P, e->stream);
    case SAS_ELLIPTICAL_CYLINDER: return Launcher<T, SAS_ELLIPTICAL_CYLINDER>::records(P, e->stream);
    case SAS_HOLLOW_RECTANGULAR_PRISM: return Launcher<T, SAS_HOLLOW_RECTANGULAR_PRISM>::records(P, e->stream);
    case SAS_SHAPE_INDEPENDENT: return Launcher<T, SAS_SHAPE_INDEPENDENT>::records(P, e->stream);
    default: return Launcher<T, SAS_ELLIPSOID>::records(P, e->stream);
    }
}

template <typename T>
cudaError_t dispatch_eval(sas_experiment* e, const ModelConst<T>& mc, const T* q, T* out, size_t n)
{
    const T* poly = (const T*)e->d_poly;
    const T* orient = (const T*)e->d_orient;
    switch (e->model.kind) {
    case SAS_SPHERE: return Launcher<T, SAS_SPHERE>::eval(mc, poly, orient, q, out, n, e->stream);
    case SAS_CORE_SHELL: return Launcher<T, SAS_CORE_SHELL>::eval(mc, poly, orient, q, out, n, e->stream);
    case SAS_CYLINDER: return Launcher<T, SAS_CYLINDER>::eval(mc, poly, orient, q, out, n, e->stream);
    case SAS_TRIAXIAL_ELLIPSOID: return Launcher<T, SAS_TRIAXIAL_ELLIPSOID>::eval(mc, poly, orient, q, out, n, e->stream);
    case SAS_PARALLELEPIPED: return Launcher<T, SAS_PARALLELEPIPED>::eval(mc, poly, orient, q, out, n, e->stream);
    case SAS_CAPPED_CYLINDER: return Launcher<T, SAS_CAPPED_CYLINDER>::eval(mc, poly, orient, q, out, n, e->stream);
    case SAS_BARBELL: return Launcher<T, SAS_BARBELL>::eval(mc, poly, orient, q, out, n, e->stream);
    case SAS_CORE_SHELL_CYLINDER: return Launcher<T, SAS_CORE_SHELL_CYLINDER>::eval(mc, poly, orient, q, out, n, e->stream);
    case SAS_HOLLOW_CYLINDER: return Launcher<T, SAS_HOLLOW_CYLINDER>::eval(mc, poly, orient, q, out, n, e->stream);
    case SAS_CORE_SHELL_ELLIPSOID: return Launcher<T, SAS_CORE_SHELL_ELLIPSOID>::eval(mc, poly, orient, q, out, n, e->stream);
    case SAS_CORE_SHELL_BICELLE: return Launcher<T, SAS_CORE_SHELL_BICELLE>::eval(mc, poly, orient, q, out, n, e->stream);
    case SAS_ELLIPTICAL_CYLINDER: return Launcher<T, SAS_ELLIPTICAL_CYLINDER>::eval(mc, poly, orient, q, out, n, e->stream);
    case SAS_HOLLOW_RECTANGULAR_PRISM: return Launcher<T, SAS_HOLLOW_RECTANGULAR_PRISM>::eval(mc, poly, orient, q, out, n, e->stream);
    case SAS_SHAPE_INDEPENDENT: return Launcher<T, SAS_SHAPE_INDEPENDENT>::eval(mc, poly, orient, q, out, n, e->stream);
    default: return Launcher<T, SAS_ELLIPSOID>::eval(mc, poly, orient, q, out, n, e->stream);
    }
}

bool can_order_q(const sas_experiment* e, const LaunchCfg& c);
float order_q_scale(const sas_experiment* e);

template <typename T>
TraceParams<T> make_params(sas_experiment* e, uint64_t first, uint64_t n, uint64_t seed)
{
    TraceParams<T> P;
    std::memset(&P, 0, sizeof(P));
    if constexpr (sizeof(T) == sizeof(float)) {
        P.in = e->icf;
        P.mc = e->mcf;
    } else {
        P.in = e->icd;
        P.mc = e->mcd;
    }
    P.poly = (const T*)e->d_poly;
    P.orient = (const T*)e->d_orient;
    P.seed = seed;
    P.first = first;
    P.n = n;
    P.exp_id = e->exp_id;
    P.stage_orient = e->stage_orient;
    P.sum_w = e->d_sum_w;
    P.sum_w2 = e->d_sum_w2;
    P.count = e->d_count;
    P.trans = e->d_trans;
    P.q2_bin = (e->cfg.order_q && can_order_q(e, e->cfg)) ? order_q_scale(e) : 0.f;
    return P;
}

// The |Q|-ordered trace pass applies to the FP32 sphere and core-shell sphere
// with quadrature averages over at least four radius nodes in ascending order
// whose tables, histogram and ordering buffers fit in one CTA's shared memory.
bool can_order_q(const sas_experiment* e, const LaunchCfg& c)
{
    const sas_model_desc& m = e->model;
    if (m.precision != SAS_FP32 || (m.kind != SAS_SPHERE && m.kind != SAS_CORE_SHELL)) return false;
    if (m.sampling != SAS_QUADRATURE) return false;
    const int np = e->tables.n_poly;
    if (np < 4) return false;
    for (int i = 1; i < np; ++i)
        if (e->tables.poly[(size_t)i * SAS_POLY_STRIDE] < e->tables.poly[(size_t)(i - 1) * SAS_POLY_STRIDE])
            return false;   // column 0 is r (sphere) or r_c^2 (core-shell): ascending with the radius
    size_t need = table_bytes<float>(np, e->tables.n_orient, 0) + sort_bytes(c.block);
    if (c.tally == TALLY_SMEM) need += hist_bytes((int)(e->inst.nx * e->inst.ny));
    return need <= (size_t)e->smem_optin;
}

// Bins per unit |Q|^2 of the ordering: SORT_BINS bins up to the largest |Q|
// the geometry allows (shortest wavelength, detector corner seen from the
// edge of the sample); larger values share the last bin.
float order_q_scale(const sas_experiment* e)
{
    const sas_instrument& in = e->inst;
    const double kmax = 2.0 * M_PI / (in.lambda0 * (1.0 - in.dlambda_rel));
    const double hx = 0.5 * in.nx * in.pixel_x + in.sample_half_x + in.ap2_radius;
    const double hy = 0.5 * in.ny * in.pixel_y + in.sample_half_y + in.ap2_radius;
    const double theta = std::atan2(std::sqrt(hx * hx + hy * hy), in.det_distance);
    const double qmax = 2.0 * kmax * std::sin(0.5 * theta);
    return (float)(SORT_BINS / (qmax * qmax));
}

// Default launch configuration: the shared-memory histogram when it fits
// next to the tables and the model has no orientation average (cheap
// histories, tally-bound); otherwise the orientation table goes to shared
// memory and tallies use FP64 global atomics (histories cost 1e5+ FLOP).
void choose_config(sas_experiment* e)
{
    const size_t optin = (size_t)e->smem_optin;
    const int npix = (int)(e->inst.nx * e->inst.ny);
    const bool fp32 = e->model.precision == SAS_FP32;
    const int np = e->tables.n_poly, no = e->tables.n_orient;
    LaunchCfg c;
    c.block = 512;
    c.agg = 0;
    c.ctas_per_sm = 0;
    c.tally = TALLY_GLOBAL;
    c.order_q = 0;
    e->stage_orient = 0;
    if (fp32) {
        if (no > 1) {
            e->stage_orient = table_bytes<float>(np, no, 1) <= optin ? 1 : 0;
        } else if (table_bytes<float>(np, no, 0) + hist_bytes(npix) <= optin) {
            c.tally = TALLY_SMEM;
            c.block = 1024;
        }
    } else {
        e->stage_orient = (no > 1 && table_bytes<double>(np, no, 1) <= optin) ? 1 : 0;
        c.block = 256;
    }
    c.order_q = can_order_q(e, c) ? 1 : 0;
    e->cfg = c;
}

// Process-wide cache of tuned launch configurations, keyed by what decides
// the kernel's cost profile: model kind, precision, node counts, detector
// size and structure factor.
struct TuneKey {
    int64_t kind, precision, sq;
    int np, no, npix;
    bool operator==(const TuneKey& o) const
    {
        return kind == o.kind && precision == o.precision && sq == o.sq && np == o.np && no == o.no &&
               npix == o.npix;
    }
};
struct TuneEntry {
    TuneKey key;
    LaunchCfg cfg;
    int stage_orient;
};
std::vector<TuneEntry> g_tuned;
std::mutex g_tuned_mu;

TuneKey tune_key(const sas_experiment* e)
{
    TuneKey k;
    k.kind = e->model.kind;
    k.precision = e->model.precision;
    k.sq = e->model.sq_kind;
    k.np = e->tables.n_poly;
    k.no = e->tables.n_orient;
    k.npix = (int)(e->inst.nx * e->inst.ny);
    return k;
}

bool lookup_tuned(sas_experiment* e)
{
    std::lock_guard<std::mutex> lk(g_tuned_mu);
    const TuneKey k = tune_key(e);
    for (const TuneEntry& t : g_tuned)
        if (t.key == k) {
            e->cfg = t.cfg;
            e->stage_orient = t.stage_orient;
            return true;
        }
    return false;
}

void store_tuned(const sas_experiment* e)
{
    std::lock_guard<std::mutex> lk(g_tuned_mu);
    const TuneKey k = tune_key(e);
    for (TuneEntry& t : g_tuned)
        if (t.key == k) {
            t.cfg = e->cfg;
            t.stage_orient = e->stage_orient;
            return;
        }
    g_tuned.push_back(TuneEntry{k, e->cfg, e->stage_orient});
}

sas_status upload_surrogate_exp(sas_experiment* e)
{
    if (!e->sur || !e->has_model) return SAS_OK;
    if (!e->d_sexp) {
        SAS_CUDA(cudaMalloc(&e->d_sexp, sizeof(sur::SurExp)), "alloc");
        SAS_CUDA(cudaMalloc(&e->d_bexp, sizeof(BatchExp)), "alloc");
        SAS_CUDA(cudaMalloc(&e->d_seed, sizeof(uint64_t)), "alloc");
        SAS_CUDA(cudaMalloc(&e->d_fallbacks, sizeof(unsigned long long)), "alloc");
        SAS_CUDA(cudaMemset(e->d_fallbacks, 0, sizeof(unsigned long long)), "memset");
    }
    const sur::SurExp se = surrogate_exp(e->model, surrogate_covers(e->sur, e->model));
    BatchExp be;
    std::memset(&be, 0, sizeof(be));
    be.mc = e->mcf;
    SAS_CUDA(cudaMemcpy(e->d_sexp, &se, sizeof(se), cudaMemcpyHostToDevice), "upload");
    SAS_CUDA(cudaMemcpy(e->d_bexp, &be, sizeof(be), cudaMemcpyHostToDevice), "upload");
    return SAS_OK;
}

// Trace through the tensor-core surrogate: items of 2^16
// histories, cut into 256-history pairs that a grid of one CTA per SM takes
// round-robin.
sas_status trace_surrogate(sas_experiment* e, uint64_t first, uint64_t n, uint64_t seed)
{
    const uint64_t chunk = 1ull << 16;
    std::vector<WorkItem> items;
    for (uint64_t f = 0; f < n; f += chunk) {
        WorkItem w;
        w.first = first + f;
        w.exp = 0;
        w.n = (uint32_t)std::min<uint64_t>(chunk, n - f);
        items.push_back(w);
    }
    std::vector<uint32_t> prefix;
    const uint64_t n_pairs = surrogate_pair_prefix(items, prefix);
    if (n_pairs > 0xFFFFFFFFull) return fail(SAS_ERR_ARG, "too many histories for one surrogate trace");
    if (items.size() > e->items_cap) {
        SAS_CUDA(cudaStreamSynchronize(e->stream), "sync");
        cudaFree(e->d_items);
        cudaFree(e->d_prefix);
        e->d_items = nullptr;
        e->d_prefix = nullptr;
        e->items_cap = 0;
        SAS_CUDA(cudaMalloc(&e->d_items, items.size() * sizeof(WorkItem)), "alloc items");
        SAS_CUDA(cudaMalloc(&e->d_prefix, items.size() * sizeof(uint32_t)), "alloc items");
        e->items_cap = items.size();
    }
    SAS_CUDA(cudaMemcpyAsync(e->d_items, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice,
                             e->stream), "upload items");
    SAS_CUDA(cudaMemcpyAsync(e->d_prefix, prefix.data(), prefix.size() * sizeof(uint32_t), cudaMemcpyHostToDevice,
                             e->stream), "upload items");
    SAS_CUDA(cudaMemcpyAsync(e->d_seed, &seed, sizeof(seed), cudaMemcpyHostToDevice, e->stream), "upload seed");
    sur::STParams P;
    std::memset(&P, 0, sizeof(P));
    P.in = e->icf;
    P.box = surrogate_dbox(e->sur);
    P.epi = surrogate_epi(e->sur);
    P.seed = e->d_seed;
    P.philox_base = e->exp_id;
    P.items = e->d_items;
    P.pair_prefix = e->d_prefix;
    P.n_items = (uint32_t)items.size();
    P.n_pairs = (uint32_t)n_pairs;
    P.sexp = e->d_sexp;
    P.bexp = e->d_bexp;
    P.poly = (const float*)e->d_poly;
    P.orient = (const float*)e->d_orient;
    P.sum_w = e->d_sum_w;
    P.sum_w2 = e->d_sum_w2;
    P.count = e->d_count;
    P.trans = e->d_trans;
    P.npix = (int)(e->inst.nx * e->inst.ny);
    P.fallbacks = e->d_fallbacks;
    P.err = surrogate_err(e->sur);
    SAS_CUDA(launch_sur_trace(e->sur, P, e->sm_count, e->stream), "surrogate trace launch");
    return SAS_OK;
}

}  // namespace

namespace sas {
unsigned long long* experiment_fallback_counter(const sas_experiment* e) { return e ? e->d_fallbacks : nullptr; }
cudaStream_t experiment_stream(const sas_experiment* e) { return e->stream; }
}  // namespace sas

extern "C" {

const char* sas_last_error(void) { return g_last_error.c_str(); }

sas_status sas_attach_surrogate(sas_experiment* e, const sas_surrogate* s)
{
    if (!e) return fail(SAS_ERR_ARG, "experiment is NULL");
    SAS_CUDA(cudaStreamSynchronize(e->stream), "sync");
    e->sur = s;
    return upload_surrogate_exp(e);
}

sas_status sas_get_launch_config(const sas_experiment* e, sas_launch_config* c)
{
    if (!e || !c) return fail(SAS_ERR_ARG, "NULL argument");
    c->block = e->cfg.block;
    c->tally = e->cfg.tally;
    c->agg = e->cfg.agg;
    c->ctas_per_sm = e->cfg.ctas_per_sm;
    c->stage_orient = e->stage_orient;
    c->order_q = e->cfg.order_q;
    return SAS_OK;
}

sas_status sas_set_launch_config(sas_experiment* e, const sas_launch_config* c)
{
    if (!e || !c) return fail(SAS_ERR_ARG, "NULL argument");
    if (!e->has_model) return fail(SAS_ERR_STATE, "sas_set_model has not been called");
    if (c->block < 32 || c->block > 1024 || c->block % 32) return fail(SAS_ERR_ARG, "bad block size");
    if (c->tally != TALLY_GLOBAL && c->tally != TALLY_SMEM) return fail(SAS_ERR_ARG, "bad tally mode");
    if (c->ctas_per_sm < 0) return fail(SAS_ERR_ARG, "bad ctas_per_sm");
    const bool fp32 = e->model.precision == SAS_FP32;
    const int np = e->tables.n_poly, no = e->tables.n_orient;
    const size_t optin = (size_t)e->smem_optin;
    const int stage = (c->stage_orient && no > 1) ? 1 : 0;
    size_t need = fp32 ? table_bytes<float>(np, no, stage) : table_bytes<double>(np, no, stage);
    if (c->tally == TALLY_SMEM) {
        if (!fp32) return fail(SAS_ERR_ARG, "the shared-memory histogram is FP32 only");
        need += hist_bytes((int)(e->inst.nx * e->inst.ny));
    }
    if (need > optin) return fail(SAS_ERR_ARG, "configuration needs more shared memory than a CTA has");
    e->cfg.block = c->block;
    e->cfg.tally = c->tally;
    e->cfg.agg = c->agg ? 1 : 0;
    e->cfg.ctas_per_sm = c->ctas_per_sm;
    e->cfg.order_q = c->order_q ? 1 : 0;
    e->stage_orient = stage;
    return SAS_OK;
}

// Time the candidate launch configurations on n_sample histories (after one
// warm-up each) and keep the fastest; the result is cached for every later
// experiment with the same key.
sas_status sas_autotune(sas_experiment* e, uint64_t n_sample, uint64_t seed, sas_launch_config* best_out,
                        double* best_ms)
{
    if (!e) return fail(SAS_ERR_ARG, "experiment is NULL");
    if (!e->has_model) return fail(SAS_ERR_STATE, "sas_set_model has not been called");
    if (n_sample == 0) return fail(SAS_ERR_ARG, "n_sample must be > 0");
    const int blocks[] = {256, 512, 1024};
    cudaEvent_t e0, e1;
    SAS_CUDA(cudaEventCreate(&e0), "event");
    SAS_CUDA(cudaEventCreate(&e1), "event");
    sas_launch_config best;
    sas_get_launch_config(e, &best);
    float best_t = 1e30f;
    const bool aniso = e->tables.n_orient > 1;
    const bool orderable = can_order_q(e, LaunchCfg{32, TALLY_GLOBAL, 0, 0, 1});
    for (int tally : {TALLY_SMEM, TALLY_GLOBAL})
        for (int agg : {0, 1})
            for (int stage : {1, 0})
                for (int oq : {1, 0}) {
                if (!aniso && stage) continue;
                if (!orderable && oq) continue;
                for (int blk : blocks) {
                    sas_launch_config c;
                    c.block = blk;
                    c.tally = tally;
                    c.agg = agg;
                    c.ctas_per_sm = 0;
                    c.stage_orient = stage;
                    c.order_q = oq;
                    if (sas_set_launch_config(e, &c) != SAS_OK) continue;
                    if (sas_trace_range(e, 0, n_sample, seed) != SAS_OK) continue;
                    cudaEventRecord(e0, e->stream);
                    sas_status st = sas_trace_range(e, 0, n_sample, seed);
                    cudaEventRecord(e1, e->stream);
                    if (cudaEventSynchronize(e1) != cudaSuccess || st != SAS_OK) continue;
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (ms < best_t) {
                        best_t = ms;
                        best = c;
                    }
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    sas_status st = sas_reset_detector(e);
    if (st != SAS_OK) return st;
    if (best_t >= 1e30f) return fail(SAS_ERR_CUDA, "no launch configuration ran");
    st = sas_set_launch_config(e, &best);
    if (st != SAS_OK) return st;
    store_tuned(e);
    if (best_out) *best_out = best;
    if (best_ms) *best_ms = best_t;
    return SAS_OK;
}

sas_status sas_device_info(int* sm_count, int* smem_per_block_optin, int* cc_major, int* cc_minor)
{
    int dev = 0;
    SAS_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    cudaDeviceProp p;
    SAS_CUDA(cudaGetDeviceProperties(&p, dev), "cudaGetDeviceProperties");
    if (sm_count) *sm_count = p.multiProcessorCount;
    if (smem_per_block_optin) *smem_per_block_optin = (int)p.sharedMemPerBlockOptin;
    if (cc_major) *cc_major = p.major;
    if (cc_minor) *cc_minor = p.minor;
    return SAS_OK;
}

sas_status sas_create_experiment(const sas_instrument* inst, void* stream, sas_experiment** out)
{
    if (!out) return fail(SAS_ERR_ARG, "out is NULL");
    *out = nullptr;
    sas_status st = validate_instrument(inst);
    if (st != SAS_OK) return st;
    sas_experiment* e = new (std::nothrow) sas_experiment();
    if (!e) return fail(SAS_ERR_OOM, "host allocation failed");
    e->inst = *inst;
    e->stream = (cudaStream_t)stream;
    cudaError_t ce = cudaGetDevice(&e->device);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&e->sm_count, cudaDevAttrMultiProcessorCount, e->device);
    if (ce == cudaSuccess)
        ce = cudaDeviceGetAttribute(&e->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, e->device);
    const size_t npix = (size_t)inst->nx * (size_t)inst->ny;
    if (ce == cudaSuccess) ce = cudaMalloc(&e->d_sum_w, npix * sizeof(double));
    if (ce == cudaSuccess) ce = cudaMalloc(&e->d_sum_w2, npix * sizeof(double));
    if (ce == cudaSuccess) ce = cudaMalloc(&e->d_count, npix * sizeof(unsigned long long));
    if (ce == cudaSuccess) ce = cudaMalloc(&e->d_trans, sizeof(double));
    if (ce != cudaSuccess) {
        sas_destroy_experiment(e);
        return cuda_fail(ce, "sas_create_experiment");
    }
    e->icf = inst_const<float>(*inst);
    e->icd = inst_const<double>(*inst);
    st = sas_reset_detector(e);
    if (st != SAS_OK) {
        sas_destroy_experiment(e);
        return st;
    }
    *out = e;
    return SAS_OK;
}

sas_status sas_set_model(sas_experiment* e, const sas_model_desc* m)
{
    if (!e) return fail(SAS_ERR_ARG, "experiment is NULL");
    sas_status st = validate_model(m);
    if (st != SAS_OK) return st;
    ModelTables t;
    st = build_model_tables(*m, t, instrument_q_max(e->inst));
    if (st != SAS_OK) return st;
    const bool fp32 = m->precision == SAS_FP32;
    const size_t es = fp32 ? sizeof(float) : sizeof(double);
    std::vector<float> pf, of;
    const void* hp;
    const void* ho;
    if (fp32) {
        pf.assign(t.poly.begin(), t.poly.end());
        of.assign(t.orient.begin(), t.orient.end());
        hp = pf.data();
        ho = of.data();
    } else {
        hp = t.poly.data();
        ho = t.orient.data();
    }
    // the previous tables may still be read by queued kernels
    SAS_CUDA(cudaStreamSynchronize(e->stream), "cudaStreamSynchronize");
    cudaFree(e->d_poly);
    cudaFree(e->d_orient);
    cudaFree(e->d_sqtab);
    e->d_poly = e->d_orient = e->d_sqtab = nullptr;
    e->has_model = false;
    std::vector<float> sqf(t.sq_tab.begin(), t.sq_tab.end());
    if (!t.sq_tab.empty()) {
        SAS_CUDA(cudaMalloc(&e->d_sqtab, t.sq_tab.size() * es), "cudaMalloc(S table)");
        SAS_CUDA(cudaMemcpyAsync(e->d_sqtab, fp32 ? (const void*)sqf.data() : (const void*)t.sq_tab.data(),
                                 t.sq_tab.size() * es, cudaMemcpyHostToDevice, e->stream), "upload S table");
    }
    SAS_CUDA(cudaMalloc(&e->d_poly, t.poly.size() * es), "cudaMalloc(poly)");
    SAS_CUDA(cudaMalloc(&e->d_orient, t.orient.size() * es), "cudaMalloc(orient)");
    SAS_CUDA(cudaMemcpyAsync(e->d_poly, hp, t.poly.size() * es, cudaMemcpyHostToDevice, e->stream), "upload poly");
    SAS_CUDA(cudaMemcpyAsync(e->d_orient, ho, t.orient.size() * es, cudaMemcpyHostToDevice, e->stream), "upload orient");
    // the host vectors go out of scope: finish the copies first
    SAS_CUDA(cudaStreamSynchronize(e->stream), "cudaStreamSynchronize");
    e->model = *m;
    e->tables = std::move(t);
    if (m->self_attenuation) {
        AttRule r;
        att_rule(e->inst, *m, e->tables, r);
        double mu[SAS_ATT_MAX];
        SAS_CUDA(att_nodes(*m, e->tables, e->d_poly, e->d_orient, r, e->stream, mu), "self-attenuation table");
        for (int j = 0; j < r.n_lambda; ++j)
            if (!std::isfinite(mu[j]) || mu[j] < 0.0)
                return fail(SAS_ERR_NUMERIC, "self-attenuation: non-finite or negative total cross section");
        att_fit(r, mu, e->tables);
    }
    e->mcf = model_const<float>(*m, e->tables);
    e->mcd = model_const<double>(*m, e->tables);
    e->mcf.sq_tab = fp32 ? (const float*)e->d_sqtab : nullptr;
    e->mcd.sq_tab = fp32 ? nullptr : (const double*)e->d_sqtab;
    e->has_model = true;
    if (!lookup_tuned(e)) choose_config(e);
    return upload_surrogate_exp(e);
}

sas_status sas_hayter_msa_table(double radius_eff, double fraction, double charge, double temperature, double salt,
                                double dielectric, double q_max, int n_max, double* dq, double* s_dsdq, int* n_out,
                                double* s_rescale, double* contact, double* gamma_c, double* kappa)
{
    if (!(radius_eff > 0.0) || !(fraction > 0.0 && fraction < 0.45) || !(charge >= 0.0) || !(temperature > 0.0) ||
        !(salt >= 0.0) || !(dielectric > 0.0) || !(q_max > 0.0) || n_max < 0 || (n_max > 0 && !s_dsdq))
        return fail(SAS_ERR_ARG, "Hayter MSA table: parameters out of range");
    const msa::Reduced r = msa::reduce(radius_eff, fraction, charge, temperature, salt, dielectric);
    if (gamma_c) *gamma_c = r.gamma_c;
    if (kappa) *kappa = r.kappa;
    msa::Table tab;
    std::string err;
    if (!msa::build_table(r, q_max, tab, err)) return fail(SAS_ERR_ARG, err);
    const int n = (int)(tab.sd.size() / 2);
    if (n_out) *n_out = n;
    if (dq) *dq = tab.dq;
    if (s_rescale) *s_rescale = tab.s_rescale;
    if (contact) *contact = tab.contact;
    if (n > n_max) return fail(SAS_ERR_ARG, "Hayter MSA table: n_max too small");
    std::copy(tab.sd.begin(), tab.sd.end(), s_dsdq);
    return SAS_OK;
}

sas_status sas_set_experiment_id(sas_experiment* e, uint32_t id)
{
    if (!e) return fail(SAS_ERR_ARG, "experiment is NULL");
    e->exp_id = id;
    return SAS_OK;
}

sas_status sas_set_stream(sas_experiment* e, void* stream)
{
    if (!e) return fail(SAS_ERR_ARG, "experiment is NULL");
    e->stream = (cudaStream_t)stream;
    return SAS_OK;
}

sas_status sas_reset_detector(sas_experiment* e)
{
    if (!e) return fail(SAS_ERR_ARG, "experiment is NULL");
    const size_t npix = (size_t)e->inst.nx * (size_t)e->inst.ny;
    SAS_CUDA(cudaMemsetAsync(e->d_sum_w, 0, npix * sizeof(double), e->stream), "memset");
    SAS_CUDA(cudaMemsetAsync(e->d_sum_w2, 0, npix * sizeof(double), e->stream), "memset");
    SAS_CUDA(cudaMemsetAsync(e->d_count, 0, npix * sizeof(unsigned long long), e->stream), "memset");
    SAS_CUDA(cudaMemsetAsync(e->d_trans, 0, sizeof(double), e->stream), "memset");
    return SAS_OK;
}

sas_status sas_trace_range(sas_experiment* e, uint64_t first, uint64_t n, uint64_t seed)
{
    if (!e) return fail(SAS_ERR_ARG, "experiment is NULL");
    if (!e->has_model) return fail(SAS_ERR_STATE, "sas_set_model has not been called");
    if (first + n < first) return fail(SAS_ERR_ARG, "neutron index range overflows 64 bits");
    if (n == 0) return SAS_OK;
    if (e->sur && e->model.precision == SAS_FP32 && surrogate_covers(e->sur, e->model))
        return trace_surrogate(e, first, n, seed);
    cudaError_t ce;
    int grid = 0;
    if (e->model.precision == SAS_FP32)
        ce = dispatch_trace<float>(e, make_params<float>(e, first, n, seed), &grid);
    else
        ce = dispatch_trace<double>(e, make_params<double>(e, first, n, seed), &grid);
    if (ce != cudaSuccess) return cuda_fail(ce, "trace launch");
    return SAS_OK;
}

sas_status sas_trace(sas_experiment* e, uint64_t n, uint64_t seed)
{
    sas_status st = sas_reset_detector(e);
    if (st != SAS_OK) return st;
    return sas_trace_range(e, 0, n, seed);
}

sas_status sas_read_detector(const sas_experiment* e, double* sum_w, double* sum_w2, uint64_t* count,
                             size_t n_pixels, double* transmitted)
{
    if (!e) return fail(SAS_ERR_ARG, "experiment is NULL");
    const size_t npix = (size_t)e->inst.nx * (size_t)e->inst.ny;
    if ((sum_w || sum_w2 || count) && n_pixels != npix)
        return fail(SAS_ERR_ARG, "n_pixels does not match nx*ny");
    if (sum_w) SAS_CUDA(cudaMemcpyAsync(sum_w, e->d_sum_w, npix * 8, cudaMemcpyDeviceToHost, e->stream), "read sum_w");
    if (sum_w2) SAS_CUDA(cudaMemcpyAsync(sum_w2, e->d_sum_w2, npix * 8, cudaMemcpyDeviceToHost, e->stream), "read sum_w2");
    if (count) SAS_CUDA(cudaMemcpyAsync(count, e->d_count, npix * 8, cudaMemcpyDeviceToHost, e->stream), "read count");
    if (transmitted) SAS_CUDA(cudaMemcpyAsync(transmitted, e->d_trans, 8, cudaMemcpyDeviceToHost, e->stream), "read trans");
    SAS_CUDA(cudaStreamSynchronize(e->stream), "cudaStreamSynchronize");
    if (e->sur) return surrogate_take_error(e->sur, e->stream);
    return SAS_OK;
}

sas_status sas_detector_device(const sas_experiment* e, const double** sum_w, const double** sum_w2,
                               const uint64_t** count, const double** transmitted)
{
    if (!e) return fail(SAS_ERR_ARG, "experiment is NULL");
    if (sum_w) *sum_w = e->d_sum_w;
    if (sum_w2) *sum_w2 = e->d_sum_w2;
    if (count) *count = (const uint64_t*)e->d_count;
    if (transmitted) *transmitted = e->d_trans;
    return SAS_OK;
}

sas_status sas_eval_model(sas_experiment* e, const void* q_xyz, size_t n, void* out)
{
    if (!e) return fail(SAS_ERR_ARG, "experiment is NULL");
    if (!e->has_model) return fail(SAS_ERR_STATE, "sas_set_model has not been called");
    if (n == 0) return SAS_OK;
    if (!q_xyz || !out) return fail(SAS_ERR_ARG, "NULL buffer");
    if (e->model.sampling == SAS_PER_EVENT)
        return fail(SAS_ERR_STATE, "a per-event model has no deterministic dSigma/dOmega; evaluate the same model "
                                   "with sampling SAS_QUADRATURE");
    cudaError_t ce;
    if (e->model.precision == SAS_FP32)
        ce = dispatch_eval<float>(e, e->mcf, (const float*)q_xyz, (float*)out, n);
    else
        ce = dispatch_eval<double>(e, e->mcd, (const double*)q_xyz, (double*)out, n);
    if (ce != cudaSuccess) return cuda_fail(ce, "eval launch");
    return SAS_OK;
}

sas_status sas_attenuation_table(const sas_experiment* e, int* n, double* lambda, double* mu_s, double* coef,
                                 double* lmin_lmax)
{
    if (!e) return fail(SAS_ERR_ARG, "experiment is NULL");
    if (!e->has_model) return fail(SAS_ERR_STATE, "sas_set_model has not been called");
    const ModelTables& t = e->tables;
    if (n) *n = t.att_n;
    for (int j = 0; j < SAS_ATT_MAX; ++j) {
        const bool on = j < t.att_n;
        if (lambda) lambda[j] = on ? t.att_lam[j] : 0.0;
        if (mu_s) mu_s[j] = on ? t.att_mu[j] : 0.0;
        if (coef) coef[j] = on ? t.att_c[j] : 0.0;
    }
    if (lmin_lmax) {
        lmin_lmax[0] = t.att_lmin;
        lmin_lmax[1] = t.att_lmax;
    }
    return SAS_OK;
}

sas_status sas_total_cross_section(sas_experiment* e, double lambda, double* sigma, double* panels,
                                  int max_panels, int* n_panels)
{
    if (!e) return fail(SAS_ERR_ARG, "experiment is NULL");
    if (!e->has_model) return fail(SAS_ERR_STATE, "sas_set_model has not been called");
    if (e->model.sampling != SAS_QUADRATURE)
        return fail(SAS_ERR_STATE, "a per-event model has no deterministic dSigma/dOmega");
    if (!(lambda > 0.0) || !std::isfinite(lambda)) return fail(SAS_ERR_ARG, "lambda must be > 0");
    if (max_panels < 0 || (max_panels > 0 && !panels)) return fail(SAS_ERR_ARG, "bad panel buffer");
    AttRule r;
    att_rule(e->inst, e->model, e->tables, r);
    const int np = (int)r.panels.size();
    if (n_panels) *n_panels = np;
    std::vector<double> part((size_t)np);
    double mu = 0.0;
    SAS_CUDA(att_run(e->model, e->tables, e->d_poly, e->d_orient, r, &lambda, 1, e->stream, &mu, part.data()),
             "total cross section");
    if (sigma) *sigma = mu * 1e-10;
    for (int i = 0; i < std::min(np, max_panels); ++i) panels[i] = part[(size_t)i];
    return SAS_OK;
}

sas_status sas_trace_records(sas_experiment* e, uint64_t first, uint64_t n, uint64_t seed,
                             int32_t* pixel, double* weight)
{
    if (!e) return fail(SAS_ERR_ARG, "experiment is NULL");
    if (!e->has_model) return fail(SAS_ERR_STATE, "sas_set_model has not been called");
    if (n == 0) return SAS_OK;
    if (!pixel || !weight) return fail(SAS_ERR_ARG, "NULL buffer");
    if (first + n < first) return fail(SAS_ERR_ARG, "neutron index range overflows 64 bits");
    cudaError_t ce;
    if (e->model.precision == SAS_FP32) {
        TraceParams<float> P = make_params<float>(e, first, n, seed);
        P.pixel_out = pixel;
        P.weight_out = weight;
        ce = dispatch_records<float>(e, P);
    } else {
        TraceParams<double> P = make_params<double>(e, first, n, seed);
        P.pixel_out = pixel;
        P.weight_out = weight;
        ce = dispatch_records<double>(e, P);
    }
    if (ce != cudaSuccess) return cuda_fail(ce, "records launch");
    return SAS_OK;
}

sas_status sas_sync(sas_experiment* e)
{
    if (!e) return fail(SAS_ERR_ARG, "experiment is NULL");
    SAS_CUDA(cudaStreamSynchronize(e->stream), "cudaStreamSynchronize");
    return SAS_OK;
}

sas_status sas_destroy_experiment(sas_experiment* e)
{
    if (!e) return SAS_OK;
    if (e->stream || true) cudaStreamSynchronize(e->stream);
    cudaFree(e->d_sum_w);
    cudaFree(e->d_sum_w2);
    cudaFree(e->d_count);
    cudaFree(e->d_trans);
    cudaFree(e->d_poly);
    cudaFree(e->d_orient);
    cudaFree(e->d_sqtab);
    cudaFree(e->d_items);
    cudaFree(e->d_prefix);
    cudaFree(e->d_seed);
    cudaFree(e->d_sexp);
    cudaFree(e->d_bexp);
    cudaFree(e->d_fallbacks);
    delete e;
    return SAS_OK;
}

// ---- host-side utilities (no GPU needed): the library's own quadrature

sas_status sas_gauss_legendre(int n, double* x, double* w)
{
    if (n < 1 || n > 1024 || !x || !w) return fail(SAS_ERR_ARG, "bad arguments");
    gauss_legendre(n, x, w);
    return SAS_OK;
}

sas_status sas_schulz_nodes(double mean, double p, int n, double* r, double* w)
{
    if (n < 1 || n > SAS_MAX_POLY || !r || !w || !(mean > 0.0) || !(p >= 0.0 && p < 1.0))
        return fail(SAS_ERR_ARG, "bad arguments");
    schulz_nodes(mean, p, n, r, w);
    return SAS_OK;
}

sas_status sas_cylinder_radial_table(const double* r, const double* w, int n_nodes, double rbar, double xmax,
                                     int n_points, double* G, double* D, double* max_err)
{
    if (!r || !w || !G || !D || n_nodes < 1 || n_points < 2 || !(rbar > 0.0) || !(xmax > 0.0))
        return fail(SAS_ERR_ARG, "bad arguments");
    const double e = cylinder_radial_table(r, w, n_nodes, rbar, xmax, n_points, G, D);
    if (max_err) *max_err = e;
    return SAS_OK;
}

sas_status sas_orientation_nodes(double theta, double phi, double sigma, int n_gamma, int n_psi,
                                 int isotropic, double* c_xyz, double* w, int* n_out)
{
    if (n_gamma < 1 || n_psi < 1 || n_gamma > SAS_MAX_ORIENT_SIDE || n_psi > SAS_MAX_ORIENT_SIDE ||
        !c_xyz || !w || !n_out)
        return fail(SAS_ERR_ARG, "bad arguments");
    *n_out = orientation_nodes(theta, phi, sigma, n_gamma, n_psi, isotropic, c_xyz, w);
    return SAS_OK;
}

sas_status sas_py_series(double phi, double* alpha_beta_gamma, double* series, int nser)
{
    if (!alpha_beta_gamma || !series || nser < 1 || nser > 64) return fail(SAS_ERR_ARG, "bad arguments");
    py_constants(phi, alpha_beta_gamma, alpha_beta_gamma + 1, alpha_beta_gamma + 2, series, nser);
    return SAS_OK;
}

}  // extern "C"
