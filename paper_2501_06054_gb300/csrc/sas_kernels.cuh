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

#include <cuda_bf16.h>
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
    float q2_bin;              // > 0: order each CTA's histories by |Q|^2, SORT_BINS bins per q2_bin^-1
};

// |Q|^2 bins of the per-CTA ordering (plus one for histories that missed the
// sample) and the shared memory it takes next to the histogram
constexpr int SORT_BINS = 128;
constexpr int SORT_PER = 2;   // histories per thread and pass

// independent sort groups of a CTA: two where each half is whole warps
__host__ __device__ inline int sort_groups(int block)
{
    return block % 64 == 0 ? 2 : 1;
}

__host__ __device__ inline size_t sort_bytes(int block)
{
    return (size_t)block * SORT_PER * 12 + (size_t)sort_groups(block) * 2 * (SORT_BINS + 1) * 4;
}

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
    return (size_t)npix * 12;
}

// ------------------------------------------------------------- tallies

// Per-CTA FP32 histogram in shared memory. Each pixel holds one 64-bit word,
//   bits  0..31  s   the FP32 running sum of w,
//   bits 32..47  c   Kahan's compensation of s, rounded to bfloat16,
//   bits 48..63  n   the count, carried to global memory every 2^15,
// updated together by one compare-and-swap, and an FP32 sum of w^2. The
// compensation is the rounding error of the last addition (at most half an
// ulp of s); keeping it to 8 bits leaves at most 2^-10 ulp of s per
// addition uncorrected, where plain FP32 summation leaves up to half an ulp.
struct SmemHist {
    unsigned long long* kw;
    float* w2;
    int npix;

    __device__ __forceinline__ void bind(unsigned char* base, int n)
    {
        npix = n;
        kw = reinterpret_cast<unsigned long long*>(base);
        w2 = reinterpret_cast<float*>(base + (size_t)n * 8);
    }
    __device__ __forceinline__ void clear() const
    {
        for (int i = threadIdx.x; i < npix; i += blockDim.x) {
            kw[i] = 0ull;
            w2[i] = 0.f;
        }
    }
    // sum w, sum w^2 and count n of one group of histories landing in pixel p
    __device__ __forceinline__ void add(unsigned long long* gcount, int p, float w, float ww, uint32_t n) const
    {
        unsigned long long* a = kw + p;
        unsigned long long old = *reinterpret_cast<volatile unsigned long long*>(a);
        bool done = false, carry = false;
        // lock-free retry; bounded, falls back to plain adds of the sum and the count
        for (int it = 0; it < (1 << 16) && !done; ++it) {
            const float sum = __uint_as_float((uint32_t)old);
            const float c = __uint_as_float((uint32_t)(old >> 16) & 0xFFFF0000u);
            const float y = w - c;
            const float t = sum + y;
            const float cn = (t - sum) - y;
            uint32_t cnt = (uint32_t)(old >> 48) + n;
            carry = cnt >= 0x8000u;
            if (carry) cnt -= 0x8000u;
            const unsigned long long nw = ((unsigned long long)cnt << 48) |
                                          ((unsigned long long)__bfloat16_as_ushort(__float2bfloat16_rn(cn)) << 32) |
                                          (unsigned long long)__float_as_uint(t);
            const unsigned long long prev = atomicCAS(a, old, nw);
            done = prev == old;
            old = prev;
        }
        if (!done) {
            atomicAdd(reinterpret_cast<float*>(a), w);
            atomicAdd(gcount + p, (unsigned long long)n);
        } else if (carry) {
            atomicAdd(gcount + p, 0x8000ull);
        }
        atomicAdd(w2 + p, ww);
    }
    // FP64 per-bin reduction of the CTA's histogram into a detector
    __device__ __forceinline__ void flush(double* sw, double* sw2, unsigned long long* cnt) const
    {
        for (int p = threadIdx.x; p < npix; p += blockDim.x) {
            const unsigned long long v = kw[p];
            const float s2 = w2[p];
            const double sum = (double)__uint_as_float((uint32_t)v) -
                               (double)__uint_as_float((uint32_t)(v >> 16) & 0xFFFF0000u);
            const uint32_t c = (uint32_t)(v >> 48);
            if (c != 0u || sum != 0.0 || s2 != 0.f) {
                atomicAdd(sw + p, sum);
                atomicAdd(sw2 + p, (double)s2);
                if (c) atomicAdd(cnt + p, (unsigned long long)c);
            }
        }
    }
};

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
        h.add(P.count, pix, (float)w, (float)w2, n);
    } else {
        atomicAdd(P.sum_w + pix, (double)w);
        atomicAdd(P.sum_w2 + pix, (double)w2);
        atomicAdd(P.count + pix, (unsigned long long)n);
    }
}

// ------------------------------------------------------------- kernels

// barrier of `count` threads (a multiple of 32) under the named barrier `id`
__device__ __forceinline__ void group_sync(int id, int count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// One pass of a |Q|-ordered trace (SORT) by a group of nb threads (tid its
// thread, bar its named barrier) over SORT_PER x nb consecutive histories.
// Each thread traces SORT_PER of them and counts each
// into its |Q|^2 bin (the shared-memory atomic returns its rank in the bin);
// after an exclusive prefix sum over the bins every history's (|Q|^2, pixel,
// prefactor) goes to its place in bin order, and each warp then evaluates
// and tallies 32 x SORT_PER consecutive places, i.e. histories of nearby
// |Q|, SORT_PER neighbouring places per lane in the same node loops (more
// independent work per warp, one node-table load for all of them). The
// set of histories, their values and
// their tallies are those of the plain loop; only which lane evaluates which
// history changes. The bin counters alternate between two arrays: the ones
// of this pass are cleared after the last read of them and next counted into
// two passes later, behind this pass's and the next pass's barriers.
template <int KIND, int TALLY, int AGG, bool ATT>
__device__ __forceinline__ void trace_sorted_pass(const TraceParams<float>& P, const SmemHist& h, const float* poly,
                                                  float* s_q2, int* s_pix, float* s_pref, int* s_bin,
                                                  uint64_t base, Kahan<float>& tr, int tid, int nb, int bar)
{
    int key[SORT_PER], rank[SORT_PER], pix[SORT_PER];
    float q2[SORT_PER], pref[SORT_PER];
#pragma unroll
    for (int k = 0; k < SORT_PER; ++k) {
        const uint64_t j = base + (uint64_t)k * nb + tid;
        pix[k] = -1;
        pref[k] = 0.f;
        q2[k] = -1.f;
        if (j < P.n) {
            const History<float> hs = history<float, ATT>(P.in, P.mc.att, P.seed, P.exp_id, P.first + j);
            tr.add(hs.wt);
            if (hs.pixel >= 0) {
                pix[k] = hs.pixel;
                pref[k] = hs.pref;
                q2[k] = fmaf(hs.q[0], hs.q[0], fmaf(hs.q[1], hs.q[1], hs.q[2] * hs.q[2]));
            }
        }
        key[k] = pix[k] >= 0 ? min((int)(q2[k] * P.q2_bin), SORT_BINS - 1) : SORT_BINS;
        rank[k] = atomicAdd(s_bin + key[k], 1);
    }
    group_sync(bar, nb);
    if (tid < 32) {   // exclusive prefix sum of the bin counts, in place
        constexpr int per = (SORT_BINS + 1 + 31) / 32;
        const int b0 = tid * per;
        int loc[per], sum = 0;
#pragma unroll
        for (int k = 0; k < per; ++k) {
            loc[k] = (b0 + k <= SORT_BINS) ? s_bin[b0 + k] : 0;
            sum += loc[k];
        }
        int inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, o);
            if (tid >= o) inc += v;
        }
        int run = inc - sum;
#pragma unroll
        for (int k = 0; k < per; ++k) {
            if (b0 + k <= SORT_BINS) s_bin[b0 + k] = run;
            run += loc[k];
        }
    }
    group_sync(bar, nb);
#pragma unroll
    for (int k = 0; k < SORT_PER; ++k) {
        const int pos = s_bin[key[k]] + rank[k];
        s_q2[pos] = q2[k];
        s_pix[pos] = pix[k];
        s_pref[pos] = pref[k];
    }
    group_sync(bar, nb);
    for (int i = tid; i <= SORT_BINS; i += nb) s_bin[i] = 0;
    // a warp evaluates 32 x SORT_PER consecutive places, SORT_PER neighbours per lane
    const int base_place = (tid >> 5) * 32 * SORT_PER + (tid & 31) * SORT_PER;
    float q2v[SORT_PER], val[SORT_PER];
#pragma unroll
    for (int k = 0; k < SORT_PER; ++k) q2v[k] = s_q2[base_place + k];
    dsigma_sorted<KIND, SORT_PER>(q2v, P.mc, poly, val);
#pragma unroll
    for (int k = 0; k < SORT_PER; ++k)
        tally<float, TALLY, AGG>(P, h, s_pix[base_place + k], s_pref[base_place + k] * val[k]);
}

template <typename T, int KIND, int TALLY, int AGG, bool ATT, bool SORT = false>
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
    unsigned char* hbase = smem + table_bytes<T>(P.mc.n_poly, P.mc.n_orient, P.stage_orient);
    h.bind(hbase, P.in.nx * P.in.ny);
    if (TALLY == TALLY_SMEM) h.clear();
    // |Q|-ordered passes: the CTA's warps form sort_groups() independent
    // groups (named barriers 1, 2), each with its own buffers, so that one
    // group's barrier and prefix-sum phases overlap the other's work.
    float* s_q2 = nullptr;
    float* s_pref = nullptr;
    int* s_pix = nullptr;
    int* s_bin = nullptr;
    int grp = 0, gsize = 0, gtid = 0;
    if constexpr (SORT) {
        gsize = (int)blockDim.x / sort_groups((int)blockDim.x);
        grp = (int)threadIdx.x / gsize;
        gtid = (int)threadIdx.x - grp * gsize;
        const int places = SORT_PER * gsize;
        unsigned char* gbase = hbase + (TALLY == TALLY_SMEM ? hist_bytes(h.npix) : 0) +
                               (size_t)grp * ((size_t)places * 12 + (size_t)2 * (SORT_BINS + 1) * 4);
        s_q2 = reinterpret_cast<float*>(gbase);
        s_pref = s_q2 + places;
        s_pix = reinterpret_cast<int*>(s_pref + places);
        s_bin = s_pix + places;
        for (int i = gtid; i < 2 * (SORT_BINS + 1); i += gsize) s_bin[i] = 0;
    }
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const uint64_t stride = (uint64_t)gridDim.x * wpb * 32;
    Kahan<T> tr;
    if constexpr (SORT) {
        static_assert(sizeof(T) == sizeof(float), "the |Q|-ordered pass is FP32");
        const uint64_t places = (uint64_t)SORT_PER * gsize;
        const uint64_t ngroups = (uint64_t)gridDim.x * (blockDim.x / gsize);
        int parity = 0;
        for (uint64_t base = ((uint64_t)blockIdx.x * (blockDim.x / gsize) + grp) * places; base < P.n;
             base += ngroups * places, parity ^= 1)
            trace_sorted_pass<KIND, TALLY, AGG, ATT>(P, h, poly, s_q2, s_pix, s_pref,
                                                     s_bin + parity * (SORT_BINS + 1), base, tr, gtid, gsize,
                                                     1 + grp);
    } else
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
        h.flush(P.sum_w, P.sum_w2, P.count);
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
    int order_q;      // order each CTA's histories by |Q| (sphere, core-shell; FP32)
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
    if constexpr (sizeof(T) == sizeof(float) && (KIND == SAS_SPHERE || KIND == SAS_CORE_SHELL)) {
        if (P.q2_bin > 0.f) {
            kern = P.mc.att.n > 0 ? trace_kernel<T, KIND, TALLY, AGG, true, true>
                                  : trace_kernel<T, KIND, TALLY, AGG, false, true>;
            smem += sort_bytes(cfg.block);
        }
    }
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
