// Kernels of the SANS trace (templated; instantiated per model kind in the
// k_<kind>.cu translation units).
//
// trace_kernel: persistent grid (a multiple of the SM count); every warp
// takes batches of 32 consecutive neutron indices (one per lane), follows
// each history, evaluates the averaged model and tallies the weight:
//   TALLY_SMEM   per-CTA FP32 histogram in shared memory: Kahan pair for
//                sum w (64-bit CAS), FP32 sum w^2, 16-bit counts (two per
//                word, carried to global memory every 2^15), flushed once
//                per CTA with FP64 atomics -- the FP64 per-bin reduction;
//   TALLY_GLOBAL FP64 atomics into global memory per history.
// With AGG, lanes of a warp that hit the same pixel are combined first
// (__match_any_sync) so one lane updates the bin.
#pragma once

#include <cuda_runtime.h>
#include "sas_device.cuh"

namespace sas {

enum { TALLY_GLOBAL = 0, TALLY_SMEM = 1 };

template <typename T>
struct TraceParams {
    InstConst<T> in;
    ModelConst<T> mc;
    const T* poly;             // device, n_poly * SAS_POLY_STRIDE
    const T* orient;           // device, n_orient * SAS_ORIENT_STRIDE
    uint64_t seed, first, n;
    uint32_t exp_id;
    int stage_orient;          // copy the orientation table into shared memory
    double* sum_w;
    double* sum_w2;
    unsigned long long* count;
    double* trans;
    int* pixel_out;            // records mode
    double* weight_out;        // records mode
};

// bytes of shared memory: staged tables followed by the histogram
template <typename T>
__host__ __device__ inline size_t table_bytes(int n_poly, int n_orient, int stage_orient)
{
    size_t b = sizeof(T) * SAS_POLY_STRIDE * (size_t)n_poly;
    if (stage_orient) b += sizeof(T) * SAS_ORIENT_STRIDE * (size_t)n_orient;
    return (b + 15) & ~(size_t)15;
}

__host__ __device__ inline size_t hist_bytes(int npix)
{
    return (size_t)npix * 12 + (size_t)((npix + 1) / 2) * 4;
}

// ------------------------------------------------------------- tallies

__device__ __forceinline__ void kahan_add_shared(float2* cell, float v)
{
    unsigned long long* a = reinterpret_cast<unsigned long long*>(cell);
    unsigned long long old = *reinterpret_cast<volatile unsigned long long*>(a);
    // lock-free retry; bounded, falls back to a plain add of the sum
    for (int it = 0; it < (1 << 16); ++it) {
        const float s = __uint_as_float((uint32_t)old);
        const float c = __uint_as_float((uint32_t)(old >> 32));
        const float y = v - c;
        const float t = s + y;
        const float cn = (t - s) - y;
        const unsigned long long nw =
            ((unsigned long long)__float_as_uint(cn) << 32) | (unsigned long long)__float_as_uint(t);
        const unsigned long long prev = atomicCAS(a, old, nw);
        if (prev == old) return;
        old = prev;
    }
    atomicAdd(&cell->x, v);
}

struct SmemHist {
    float2* kw;      // (sum, compensation)
    float* w2;
    uint32_t* cnt;   // two 16-bit counts per word
    int npix;
};

__device__ __forceinline__ void hist_add(const SmemHist& h, unsigned long long* gcount, int p,
                                         float w, float w2, uint32_t inc)
{
    kahan_add_shared(h.kw + p, w);
    atomicAdd(h.w2 + p, w2);
    const int sh = (p & 1) * 16;
    uint32_t* cw = h.cnt + (p >> 1);
    const uint32_t old = atomicAdd(cw, inc << sh);
    const uint32_t half = (old >> sh) & 0xFFFFu;
    if (half < 0x8000u && half + inc >= 0x8000u) {   // carry 2^15 to global memory
        atomicSub(cw, 0x8000u << sh);
        atomicAdd(gcount + p, 0x8000ull);
    }
}

// Combine lanes of the warp that hit the same pixel. On return, the lane is
// the group leader iff `leader`; w/w2/n are the group sums there.
template <typename T>
__device__ __forceinline__ void warp_aggregate(int pix, T& w, T& w2, uint32_t& n, bool& leader)
{
    const int lane = threadIdx.x & 31;
    const int key = (pix >= 0) ? pix : -(lane + 1);
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    leader = (pix >= 0) && ((__ffs(peers) - 1) == lane);
    n = 1;
    w2 = w * w;
    const bool multi = __popc(peers) > 1 && pix >= 0;
    if (__any_sync(0xffffffffu, multi)) {
        const T w_own = w;
        T sw = 0, sw2 = 0;
        uint32_t cn = 0;
        for (int src = 0; src < 32; ++src) {
            const T ws = __shfl_sync(0xffffffffu, w_own, src);
            if ((peers >> src) & 1u) {
                sw += ws;
                sw2 = fma(ws, ws, sw2);
                ++cn;
            }
        }
        w = sw;
        w2 = sw2;
        n = cn;
    }
}

template <typename T, int TALLY, int AGG>
__device__ __forceinline__ void tally(const TraceParams<T>& P, const SmemHist& h, int pix, T w)
{
    T w2 = w * w;
    uint32_t n = 1;
    bool lead = pix >= 0;
    if (AGG) warp_aggregate<T>(pix, w, w2, n, lead);
    if (!lead) return;
    if (TALLY == TALLY_SMEM) {
        hist_add(h, P.count, pix, (float)w, (float)w2, n);
    } else {
        atomicAdd(P.sum_w + pix, (double)w);
        atomicAdd(P.sum_w2 + pix, (double)w2);
        atomicAdd(P.count + pix, (unsigned long long)n);
    }
}

// ------------------------------------------------------------- kernels

template <typename T, int KIND, int TALLY, int AGG, bool ATT>
__global__ void __launch_bounds__(1024) trace_kernel(const TraceParams<T> P)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const T* poly = P.poly;
    const T* orient = P.orient;
    {   // stage the quadrature tables
        T* s_poly = reinterpret_cast<T*>(smem);
        const int np = P.mc.n_poly * SAS_POLY_STRIDE;
        for (int i = threadIdx.x; i < np; i += blockDim.x) s_poly[i] = P.poly[i];
        poly = s_poly;
        if (P.stage_orient) {
            T* s_or = s_poly + np;
            const int no = P.mc.n_orient * SAS_ORIENT_STRIDE;
            for (int i = threadIdx.x; i < no; i += blockDim.x) s_or[i] = P.orient[i];
            orient = s_or;
        }
    }
    SmemHist h;
    h.npix = P.in.nx * P.in.ny;
    if (TALLY == TALLY_SMEM) {
        unsigned char* base = smem + table_bytes<T>(P.mc.n_poly, P.mc.n_orient, P.stage_orient);
        h.kw = reinterpret_cast<float2*>(base);
        h.w2 = reinterpret_cast<float*>(base + (size_t)h.npix * 8);
        h.cnt = reinterpret_cast<uint32_t*>(base + (size_t)h.npix * 12);
        for (int i = threadIdx.x; i < h.npix; i += blockDim.x) {
            h.kw[i] = make_float2(0.f, 0.f);
            h.w2[i] = 0.f;
        }
        for (int i = threadIdx.x; i < (h.npix + 1) / 2; i += blockDim.x) h.cnt[i] = 0u;
    }
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const uint64_t stride = (uint64_t)gridDim.x * wpb * 32;
    Kahan<T> tr;
    for (uint64_t base = ((uint64_t)blockIdx.x * wpb + (threadIdx.x >> 5)) * 32; base < P.n;
         base += stride) {
        const uint64_t j = base + lane;
        int pix = -1;
        T w = 0;
        if (j < P.n) {
            const History<T> hs = history<T, ATT>(P.in, P.mc.att, P.seed, P.exp_id, P.first + j);
            tr.add(hs.wt);
            if (hs.pixel >= 0) {
                w = hs.pref * dsigma_history<T, KIND>(hs.q, P.mc, poly, orient, P.seed, P.exp_id, P.first + j);
                pix = hs.pixel;
            }
        }
        tally<T, TALLY, AGG>(P, h, pix, w);
    }
    // transmitted weight: warp sum in FP64, one atomic per warp
    double t = (double)tr.s - (double)tr.c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) atomicAdd(P.trans, t);

    if (TALLY == TALLY_SMEM) {   // FP64 per-bin reduction of the CTA's histogram
        __syncthreads();
        for (int p = threadIdx.x; p < h.npix; p += blockDim.x) {
            const float2 kw = h.kw[p];
            const float s2 = h.w2[p];
            const uint32_t c = (h.cnt[p >> 1] >> ((p & 1) * 16)) & 0xFFFFu;
            if (c != 0u || kw.x != 0.f || s2 != 0.f) {
                atomicAdd(P.sum_w + p, (double)kw.x - (double)kw.y);
                atomicAdd(P.sum_w2 + p, (double)s2);
                if (c) atomicAdd(P.count + p, (unsigned long long)c);
            }
        }
    }
}

// One thread per neutron; writes (pixel, weight) without tallying.
template <typename T, int KIND>
__global__ void records_kernel(const TraceParams<T> P)
{
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P.n) return;
    const History<T> hs = history<T>(P.in, P.mc.att, P.seed, P.exp_id, P.first + j);
    double w = 0.0;
    if (hs.pixel >= 0)
        w = (double)(hs.pref * dsigma_history<T, KIND>(hs.q, P.mc, P.poly, P.orient, P.seed, P.exp_id, P.first + j));
    P.pixel_out[j] = hs.pixel;
    P.weight_out[j] = w;
}

// One thread per scattering vector: dSigma/dOmega in 1/angstrom.
template <typename T, int KIND>
__global__ void eval_kernel(const ModelConst<T> mc, const T* __restrict__ poly,
                            const T* __restrict__ orient, const T* __restrict__ q, T* out, size_t n)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const T qv[3] = {q[3 * i], q[3 * i + 1], q[3 * i + 2]};
    out[i] = dsigma<T, KIND>(qv, mc, poly, orient);
}

// Total scattering cross section (1/angstrom): one thread per evaluation of
// the rule, flattened over (wavelength y, |Q| panel p, node g, azimuth m);
// panel p holds evaluations [off[p], off[p + 1]) of each wavelength's E.
// On the Ewald sphere of k = k_lambda[y], with the panel's nodes scaled by
// k / k_max,
//   Q = (Q s cos phi, Q s sin phi, -Q^2 / (2k)), s = sqrt(1 - Q^2 / (4 k^2)),
//   phi = 2 pi (m + 1/2) / n_phi,  dOmega = Q dQ dphi / k^2;
// values[i] is the evaluation's weighted share (summed per panel by the
// caller in a fixed order).
template <typename T, int KIND>
__global__ void __launch_bounds__(256) att_eval_kernel(const ModelConst<T> mc, const T* __restrict__ poly,
                                                       const T* __restrict__ orient,
                                                       const AttPanel* __restrict__ pan,
                                                       const int* __restrict__ off, int n_pan, int E,
                                                       const double* __restrict__ k_lambda, int n_lambda,
                                                       double kmax, double* __restrict__ values)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)n_lambda * (size_t)E) return;
    const int y = (int)(i / (size_t)E);
    const int r = (int)(i - (size_t)y * E);
    int lo = 0, hi = n_pan;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= r) lo = mid;
        else hi = mid;
    }
    const AttPanel& P = pan[lo];
    const int nphi = P.n_phi;
    const int rr = r - off[lo];
    const int g = rr / nphi;
    const int m = rr - g * nphi;
    const double k = k_lambda[y];
    const double sc = k / kmax;
    const double Q = sc * P.q[g];
    const double st = sqrt(fmax(1.0 - Q * Q / (4.0 * k * k), 0.0));
    double sp, cp;
    sincospi((double)(2 * m + 1) / (double)nphi, &sp, &cp);
    const T qv[3] = {(T)(Q * st * cp), (T)(Q * st * sp), (T)(-Q * Q / (2.0 * k))};
    const double f = (double)dsigma<T, KIND>(qv, mc, poly, orient);
    values[i] = sc * P.w[g] * Q * f * (2.0 * 3.14159265358979323846 / nphi) / (k * k);
}

// ------------------------------------------------------------- launchers

struct LaunchCfg {
    int block;        // threads per CTA
    int tally;        // TALLY_GLOBAL / TALLY_SMEM
    int agg;          // warp aggregation
    int ctas_per_sm;  // 0: as many as fit
};

template <typename T, int KIND>
struct Launcher {
    static cudaError_t trace(const TraceParams<T>& P, const LaunchCfg& cfg, int sm_count,
                             cudaStream_t s, int* grid_used);
    static cudaError_t records(const TraceParams<T>& P, cudaStream_t s);
    static cudaError_t eval(const ModelConst<T>& mc, const T* poly, const T* orient, const T* q,
                            T* out, size_t n, cudaStream_t s);
    static cudaError_t att(const ModelConst<T>& mc, const T* poly, const T* orient, const AttPanel* pan,
                           const int* off, int n_pan, int E, const double* k_lambda, int n_lambda, double kmax,
                           double* values, cudaStream_t s);
};

template <typename T, int KIND, int TALLY, int AGG>
static cudaError_t launch_trace_variant(const TraceParams<T>& P, const LaunchCfg& cfg,
                                        int sm_count, cudaStream_t s, int* grid_used)
{
    // the self-attenuation table is a separate instantiation: the plain path
    // carries none of its instructions
    auto kern = P.mc.att.n > 0 ? trace_kernel<T, KIND, TALLY, AGG, true> : trace_kernel<T, KIND, TALLY, AGG, false>;
    size_t smem = table_bytes<T>(P.mc.n_poly, P.mc.n_orient, P.stage_orient);
    if (TALLY == TALLY_SMEM) smem += hist_bytes(P.in.nx * P.in.ny);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, cfg.block, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (cfg.ctas_per_sm > 0 && cfg.ctas_per_sm < per_sm) per_sm = cfg.ctas_per_sm;
    const uint64_t warps_needed = (P.n + 31) / 32;
    const uint64_t wpb = (uint64_t)cfg.block / 32;
    uint64_t grid = (uint64_t)sm_count * per_sm;
    const uint64_t useful = (warps_needed + wpb - 1) / wpb;
    if (useful < grid) grid = useful > 0 ? useful : 1;
    if (grid_used) *grid_used = (int)grid;
    kern<<<(unsigned)grid, cfg.block, smem, s>>>(P);
    return cudaGetLastError();
}

template <typename T, int KIND>
cudaError_t Launcher<T, KIND>::trace(const TraceParams<T>& P, const LaunchCfg& cfg, int sm_count,
                                     cudaStream_t s, int* grid_used)
{
    if (P.n == 0) return cudaSuccess;
    if constexpr (sizeof(T) == sizeof(float)) {
        if (cfg.tally == TALLY_SMEM)
            return cfg.agg
                       ? launch_trace_variant<T, KIND, TALLY_SMEM, 1>(P, cfg, sm_count, s, grid_used)
                       : launch_trace_variant<T, KIND, TALLY_SMEM, 0>(P, cfg, sm_count, s, grid_used);
        return cfg.agg
                   ? launch_trace_variant<T, KIND, TALLY_GLOBAL, 1>(P, cfg, sm_count, s, grid_used)
                   : launch_trace_variant<T, KIND, TALLY_GLOBAL, 0>(P, cfg, sm_count, s, grid_used);
    } else {
        if (cfg.tally == TALLY_SMEM) return cudaErrorInvalidValue;   // FP64 tallies go to global memory
        return launch_trace_variant<T, KIND, TALLY_GLOBAL, 0>(P, cfg, sm_count, s, grid_used);
    }
}

template <typename T, int KIND>
cudaError_t Launcher<T, KIND>::records(const TraceParams<T>& P, cudaStream_t s)
{
    if (P.n == 0) return cudaSuccess;
    const int block = 128;
    const uint64_t grid = (P.n + block - 1) / block;
    if (grid > 0x7FFFFFFFull) return cudaErrorInvalidValue;
    records_kernel<T, KIND><<<(unsigned)grid, block, 0, s>>>(P);
    return cudaGetLastError();
}

template <typename T, int KIND>
cudaError_t Launcher<T, KIND>::eval(const ModelConst<T>& mc, const T* poly, const T* orient,
                                    const T* q, T* out, size_t n, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const int block = 128;
    const size_t grid = (n + block - 1) / block;
    if (grid > 0x7FFFFFFFull) return cudaErrorInvalidValue;
    eval_kernel<T, KIND><<<(unsigned)grid, block, 0, s>>>(mc, poly, orient, q, out, n);
    return cudaGetLastError();
}

template <typename T, int KIND>
cudaError_t Launcher<T, KIND>::att(const ModelConst<T>& mc, const T* poly, const T* orient, const AttPanel* pan,
                                   const int* off, int n_pan, int E, const double* k_lambda, int n_lambda,
                                   double kmax, double* values, cudaStream_t s)
{
    const size_t total = (size_t)n_lambda * (size_t)E;
    if (n_pan <= 0 || total == 0) return cudaSuccess;
    const size_t grid = (total + 255) / 256;
    if (grid > 0x7FFFFFFFull) return cudaErrorInvalidValue;
    att_eval_kernel<T, KIND><<<(unsigned)grid, 256, 0, s>>>(mc, poly, orient, pan, off, n_pan, E, k_lambda,
                                                              n_lambda, kmax, values);
    return cudaGetLastError();
}

}  // namespace sas
