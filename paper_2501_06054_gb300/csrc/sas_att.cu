// Attenuation of the beam by the particles' own scattering.
//
// A neutron crossing the sample is removed from the beam at the rate of the
// total scattering cross section per unit volume,
//
//   Sigma_s(lambda) = integral over all directions k_f of dSigma/dOmega(Q),
//   Q = k (k_f - k_i), k = 2 pi / lambda, k_i along the beam axis (+z),
//
// so the trace attenuates with mu(lambda) = mu + Sigma_s(lambda) along the
// path to the scattering point and on the way out (single scattering: a
// neutron that would scatter twice is lost, not redistributed).
//
// With k_f parametrised by |Q| and its azimuth phi about z,
//   Q = (Q s cos phi, Q s sin phi, -Q^2 / (2k)), s = sqrt(1 - Q^2 / (4k^2)),
//   dOmega = Q dQ dphi / k^2, 0 <= Q <= 2k.
// The rule is fixed once per model and instrument at the band's shortest
// wavelength (k_max) and scaled with k, so Sigma_s is smooth in lambda:
//   |Q| panels [a, b] covering [0, 2 k_max], b - a = max(pi / D, a / 8) with
//   D the particle's largest extent (half a period of the amplitude's
//   oscillation near the origin, geometric growth further out), the last
//   one ending at 2 k_max; 8 Gauss-Legendre nodes per panel;
//   phi: midpoint rule, n_phi = 8 clamp(ceil(Q_mid D / 2), 2, 64) with
//   Q_mid the panel's midpoint at k_max; a single point for the sphere and
//   the core-shell sphere (their dSigma/dOmega depends on |Q| only).
// mu_s(lambda) = 1e10 Sigma_s (1/angstrom -> 1/m) is evaluated on the GPU at
// the 8 Chebyshev points of the source band [lambda0 (1 - d), lambda0 (1 + d)]
// (one point at lambda0 without a spread) and interpolated per history.
#include <cmath>
#include <cstring>
#include <vector>

#include "sas_host.h"
#include "sas_kernels.cuh"

namespace sas {

// One CTA per (panel x, wavelength y): the panel's evaluations summed in a
// fixed order (strided per thread, then a fixed tree) into partial[y][x].
__global__ void __launch_bounds__(256) att_reduce_kernel(const double* __restrict__ values,
                                                         const int* __restrict__ off, int n_pan, int E,
                                                         double* __restrict__ partial)
{
    __shared__ double red[256];
    const size_t base = (size_t)blockIdx.y * E;
    const int a = off[blockIdx.x], b = off[blockIdx.x + 1];
    double acc = 0.0;
    for (int i = a + (int)threadIdx.x; i < b; i += blockDim.x) acc += values[base + i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[(size_t)blockIdx.y * n_pan + blockIdx.x] = red[0];
}

// Sums each wavelength's panel shares in panel order (deterministic).
__global__ void att_sum_kernel(const double* __restrict__ partial, int n_pan, int n_lambda,
                               double* __restrict__ mu)
{
    const int j = threadIdx.x;
    if (j >= n_lambda) return;
    double s = 0.0;
    for (int p = 0; p < n_pan; ++p) s += partial[(size_t)j * n_pan + p];
    mu[j] = 1e10 * s;
}

double model_extent(const sas_model_desc& m, const ModelTables& t)
{
    const double r = t.r_max;
    switch (m.kind) {
    case SAS_SPHERE: return 2.0 * r;
    case SAS_CORE_SHELL: return 2.0 * (r + m.thickness);
    case SAS_CYLINDER: return std::sqrt(m.length * m.length + 4.0 * r * r);
    case SAS_ELLIPSOID: return 2.0 * std::fmax(r, m.radius_polar);
    case SAS_TRIAXIAL_ELLIPSOID:
        return 2.0 * (r / m.radius) * std::fmax(m.radius, std::fmax(m.radius_b, m.radius_polar));
    case SAS_CORE_SHELL_CYLINDER:
    case SAS_CORE_SHELL_BICELLE:
    case SAS_HOLLOW_CYLINDER: {   // the outer cylinder's diagonal
        const double lo = m.length + 2.0 * face_layer(m);
        const double ro = r + m.thickness;
        return std::sqrt(lo * lo + 4.0 * ro * ro);
    }
    case SAS_CORE_SHELL_ELLIPSOID: return 2.0 * std::fmax(r + m.thickness, m.radius_polar + m.thickness_face);
    case SAS_ELLIPTICAL_CYLINDER: {
        const double a = std::fmax(m.radius, m.radius_b);
        return 2.0 * (r / m.radius) * std::sqrt(a * a + 0.25 * m.length * m.length);
    }
    case SAS_CAPPED_CYLINDER:
    case SAS_BARBELL:   // tip to tip, L + 2H, or the caps' diameter
        return (r / m.radius) * std::fmax(m.length + 2.0 * cap_height(m), 2.0 * m.radius_polar);
    default:
        return 2.0 * (r / m.radius) *
               std::sqrt(m.radius * m.radius + m.radius_b * m.radius_b + m.radius_polar * m.radius_polar);
    }
}

void att_rule(const sas_instrument& in, const sas_model_desc& m, const ModelTables& t, AttRule& r)
{
    const double pi = M_PI;
    r.lmin = in.lambda0 * (1.0 - in.dlambda_rel);
    r.lmax = in.lambda0 * (1.0 + in.dlambda_rel);
    r.n_lambda = in.dlambda_rel > 0.0 ? SAS_ATT_MAX : 1;
    for (int j = 0; j < r.n_lambda; ++j) {
        const double tj = std::cos(pi * (j + 0.5) / r.n_lambda);
        r.lam[j] = r.n_lambda > 1 ? 0.5 * (r.lmin + r.lmax) + 0.5 * (r.lmax - r.lmin) * tj : in.lambda0;
    }
    r.kmax = 2.0 * pi / r.lmin;
    const double D = model_extent(m, t);
    const bool iso = m.kind == SAS_SPHERE || m.kind == SAS_CORE_SHELL;
    double gx[SAS_ATT_GL], gw[SAS_ATT_GL];
    gauss_legendre(SAS_ATT_GL, gx, gw);
    r.panels.clear();
    const double top = 2.0 * r.kmax;
    double a = 0.0;
    while (a < top) {
        double b = a + std::fmax(pi / D, a / 8.0);
        if (b > top) b = top;
        AttPanel p;
        std::memset(&p, 0, sizeof(p));
        const double mid = 0.5 * (a + b), half = 0.5 * (b - a);
        for (int g = 0; g < SAS_ATT_GL; ++g) {
            p.q[g] = mid + half * gx[g];
            p.w[g] = half * gw[g];
        }
        p.n_phi = iso ? 1 : 8 * (int)std::fmin(std::fmax(std::ceil(mid * D / 2.0), 2.0), 64.0);
        r.panels.push_back(p);
        a = b;
    }
}

void att_fit(const AttRule& r, const double* mu, ModelTables& t)
{
    const int n = r.n_lambda;
    t.att_n = n;
    t.att_lmin = r.lmin;
    t.att_lmax = r.lmax;
    for (int j = 0; j < n; ++j) {
        t.att_lam[j] = r.lam[j];
        t.att_mu[j] = mu[j];
    }
    // interpolant at the Chebyshev points: c_i = (2 - [i = 0]) / n sum_j mu_j cos(pi i (j + 1/2) / n)
    for (int i = 0; i < n; ++i) {
        double c = 0.0;
        for (int j = 0; j < n; ++j) c += mu[j] * std::cos(M_PI * i * (j + 0.5) / n);
        t.att_c[i] = (i == 0 ? 1.0 : 2.0) * c / n;
    }
}

namespace {

template <typename T>
cudaError_t att_launch(const sas_model_desc& m, const ModelConst<T>& mc, const T* poly, const T* orient,
                       const AttPanel* pan, const int* off, int n_pan, int E, const double* k, int n_lambda,
                       double kmax, double* values, cudaStream_t s)
{
#define SAS_ATT_CASE(K) Launcher<T, K>::att(mc, poly, orient, pan, off, n_pan, E, k, n_lambda, kmax, values, s)
    switch (m.kind) {
    case SAS_SPHERE: return SAS_ATT_CASE(SAS_SPHERE);
    case SAS_CORE_SHELL: return SAS_ATT_CASE(SAS_CORE_SHELL);
    case SAS_CYLINDER: return SAS_ATT_CASE(SAS_CYLINDER);
    case SAS_TRIAXIAL_ELLIPSOID: return SAS_ATT_CASE(SAS_TRIAXIAL_ELLIPSOID);
    case SAS_PARALLELEPIPED: return SAS_ATT_CASE(SAS_PARALLELEPIPED);
    case SAS_CAPPED_CYLINDER: return SAS_ATT_CASE(SAS_CAPPED_CYLINDER);
    case SAS_BARBELL: return SAS_ATT_CASE(SAS_BARBELL);
    case SAS_CORE_SHELL_CYLINDER: return SAS_ATT_CASE(SAS_CORE_SHELL_CYLINDER);
    case SAS_HOLLOW_CYLINDER: return SAS_ATT_CASE(SAS_HOLLOW_CYLINDER);
    case SAS_CORE_SHELL_ELLIPSOID: return SAS_ATT_CASE(SAS_CORE_SHELL_ELLIPSOID);
    case SAS_CORE_SHELL_BICELLE: return SAS_ATT_CASE(SAS_CORE_SHELL_BICELLE);
    case SAS_ELLIPTICAL_CYLINDER: return SAS_ATT_CASE(SAS_ELLIPTICAL_CYLINDER);
    case SAS_HOLLOW_RECTANGULAR_PRISM: return SAS_ATT_CASE(SAS_HOLLOW_RECTANGULAR_PRISM);
    case SAS_SHAPE_INDEPENDENT: return SAS_ATT_CASE(SAS_SHAPE_INDEPENDENT);
    default: return SAS_ATT_CASE(SAS_ELLIPSOID);
    }
#undef SAS_ATT_CASE
}

}  // namespace

cudaError_t att_run(const sas_model_desc& m, const ModelTables& t, const void* d_poly, const void* d_orient,
                    const AttRule& r, const double* lam, int nl, cudaStream_t s, double* mu_out, double* partial_out)
{
    if (nl < 1 || nl > SAS_ATT_MAX) return cudaErrorInvalidValue;
    const int n_pan = (int)r.panels.size();
    std::vector<int> off((size_t)n_pan + 1, 0);
    for (int p = 0; p < n_pan; ++p) off[p + 1] = off[p] + SAS_ATT_GL * r.panels[p].n_phi;
    const int E = off[n_pan];
    double k[SAS_ATT_MAX];
    for (int j = 0; j < nl; ++j) k[j] = 2.0 * M_PI / lam[j];
    AttPanel* d_pan = nullptr;
    int* d_off = nullptr;
    double *d_k = nullptr, *d_values = nullptr, *d_partial = nullptr, *d_mu = nullptr;
    cudaError_t e = cudaMalloc(&d_pan, sizeof(AttPanel) * (size_t)n_pan);
    if (e == cudaSuccess) e = cudaMalloc(&d_off, sizeof(int) * off.size());
    if (e == cudaSuccess) e = cudaMalloc(&d_k, sizeof(double) * SAS_ATT_MAX);
    if (e == cudaSuccess) e = cudaMalloc(&d_values, sizeof(double) * (size_t)E * nl);
    if (e == cudaSuccess) e = cudaMalloc(&d_partial, sizeof(double) * (size_t)n_pan * nl);
    if (e == cudaSuccess) e = cudaMalloc(&d_mu, sizeof(double) * SAS_ATT_MAX);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_pan, r.panels.data(), sizeof(AttPanel) * (size_t)n_pan, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_k, k, sizeof(double) * nl, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        if (m.precision == SAS_FP32)
            e = att_launch<float>(m, model_const<float>(m, t), (const float*)d_poly, (const float*)d_orient, d_pan,
                                  d_off, n_pan, E, d_k, nl, r.kmax, d_values, s);
        else
            e = att_launch<double>(m, model_const<double>(m, t), (const double*)d_poly, (const double*)d_orient,
                                   d_pan, d_off, n_pan, E, d_k, nl, r.kmax, d_values, s);
    }
    if (e == cudaSuccess) {
        att_reduce_kernel<<<dim3((unsigned)n_pan, (unsigned)nl), 256, 0, s>>>(d_values, d_off, n_pan, E, d_partial);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        att_sum_kernel<<<1, 32, 0, s>>>(d_partial, n_pan, nl, d_mu);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && mu_out) e = cudaMemcpyAsync(mu_out, d_mu, sizeof(double) * nl, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && partial_out)
        e = cudaMemcpyAsync(partial_out, d_partial, sizeof(double) * (size_t)n_pan * nl, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_pan);
    cudaFree(d_off);
    cudaFree(d_k);
    cudaFree(d_values);
    cudaFree(d_partial);
    cudaFree(d_mu);
    return e;
}

cudaError_t att_nodes(const sas_model_desc& m, const ModelTables& t, const void* d_poly, const void* d_orient,
                      const AttRule& r, cudaStream_t s, double* mu_out)
{
    return att_run(m, t, d_poly, d_orient, r, r.lam, r.n_lambda, s, mu_out, nullptr);
}

}  // namespace sas
