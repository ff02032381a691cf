// Learned surrogate: exact-target generation, BF16 tcgen05 training
// (forward, backward, weight gradients, Adam) captured in a CUDA graph,
// fused inference, and the cylinder trace that uses it.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sas_batch.cuh"
#include "sas_host.h"
#include "sas_surrogate.cuh"
#include "sas_sur_trace.cuh"

namespace sas {
sas_status set_error(sas_status s, const std::string& msg);
sas_status set_cuda_error(cudaError_t e, const char* what);
}  // namespace sas

using namespace sas;
using namespace sas::mlp;

#define SAS_CUDA_S(call, what)                                     \
    do {                                                           \
        cudaError_t _e = (call);                                   \
        if (_e != cudaSuccess) return set_cuda_error(_e, what);    \
    } while (0)

namespace sas {
namespace sur {

// ------------------------------------------------------------- kernels

// Targets are log(max(P, TARGET_FLOOR)): bins fainter than 1e-6 of P(0)
// carry no weight in the detector comparisons, so the fit spends no
// capacity on the depth of the minima below it.
constexpr float TARGET_FLOOR = 1e-6f;

// Training targets: per sample draw the raw parameters uniformly in the box
// (|Q| = q_max sqrt(u): area-uniform like the detector; cos(angle to the
// axis) uniform; sigma_poly from the bucket grid) and evaluate the exact
// quadrature. One warp per sample.
__global__ void data_kernel(Box b, Tables t, uint64_t seed, uint64_t first, uint64_t n, Raw* raw, float* y,
                            int draw)
{
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (uint64_t s = warp; s < n; s += nw) {
        Raw r;
        if (draw) {
            const uint64_t idx = first + s;
            const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
            const uint4 x = philox(make_uint4(4u, DATA_EXP_ID, (uint32_t)idx, (uint32_t)(idx >> 32)), key);
            const uint4 z = philox(make_uint4(5u, DATA_EXP_ID, (uint32_t)idx, (uint32_t)(idx >> 32)), key);
            const float q = b.q_max * sqrtf(u01<float>(x.x));
            const float ca = u01<float>(x.y);
            r.qpar = q * ca;
            r.qperp = q * sqrtf(fmaxf(1.0f - ca * ca, 0.0f));
            r.R = b.r_min + (b.r_max - b.r_min) * u01<float>(x.z);
            r.L = b.l_min + (b.l_max - b.l_min) * u01<float>(x.w);
            r.so = b.so_min + (b.so_max - b.so_min) * u01<float>(z.x);
            const int bk = (int)(((uint64_t)(z.y >> 9) * (uint64_t)b.n_buckets) >> 23);
            r.bucket = (float)bk;
            r.sp = t.bucket_sp[bk];
            r.pad = 0.f;
        } else {
            r = raw[s];
        }
        const double p = exact_pbar_warp(b, t, r);
        if (lane == 0) {
            if (draw) raw[s] = r;
            y[s] = (float)log(fmax(p, (double)TARGET_FLOOR));
        }
    }
}

struct FwdParams {
    Box box;
    const Raw* raw;        // dataset
    uint64_t n_data;       // rows in the dataset (minibatches wrap around)
    const uint32_t* step;  // training step counter (device), nullptr for plain evaluation
    uint32_t batch;        // rows of this launch
    uint64_t first;        // first row (plain evaluation)
    const float* params;   // FP32 master parameters
    float* out;            // [batch] predicted log P
    __nv_bfloat16* xt;     // [64][batch]
    __nv_bfloat16* zt[4];  // [256][batch]
    __nv_bfloat16* ht[4];
    int* err;
    uint64_t stall_ns;     // test hook: > 0 makes CTA 0 wait that long on a barrier nothing completes
};

__device__ __forceinline__ uint64_t batch_row(const FwdParams& P, uint32_t i)
{
    if (P.step) return ((uint64_t)(*P.step) * P.batch + i) % P.n_data;
    return P.first + i;
}

template <bool TRAIN>
__global__ void __launch_bounds__(THREADS, 1) mlp_fwd_kernel(const FwdParams P, const __grid_constant__ Maps maps)
{
    extern __shared__ unsigned char raw_sm[];
    Ctx c;
    ctx_init(c, raw_sm, P.err);
    if (P.stall_ns) {
        // Test of the bounded waits: before any copy or MMA is issued, CTA 0
        // waits on the MMA barrier, which nothing completes, gives up after
        // stall_ns and records the failure; every CTA then frees its tensor
        // memory and returns without work, and the host reports
        // SAS_ERR_TIMEOUT.
        if (blockIdx.x == 0 && threadIdx.x == 0 && !tc::mbar_wait(c.bar_mma, 0, P.stall_ns)) atomicExch(P.err, 9);
        ctx_finish(c);
        return;
    }
    stage_params(c, P.params);
    load_weights(c, &maps.w1, 1);
    __syncthreads();
    const int m = row_of_thread(), h = group_of_thread();
    float* s_row = reinterpret_cast<float*>(c.sm + SM_ROW);
    const uint32_t ntiles = (P.batch + TILE - 1) / TILE;
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint32_t i = tile * TILE + m;
        const bool valid = i < P.batch;
        if (h == 0) {
            float f[64];
            if (valid) {
                const Raw r = P.raw[batch_row(P, i)];
                features(P.box, r.qpar, r.qperp, r.R, r.L, r.so, r.sp, f);
            } else {
#pragma unroll
                for (int k = 0; k < 64; ++k) f[k] = 0.f;
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) st_row8(c.sm + SM_A0, m, 8 * q, f + 8 * q);
            if (TRAIN && valid)
                for (int k = 0; k < 64; ++k) P.xt[(size_t)k * P.batch + i] = __float2bfloat16_rn(f[k]);
        }
        const float dot = forward_tile<TRAIN>(c, maps, P.zt, P.ht, P.batch, i, valid);
        s_row[h * TILE + m] = dot;
        __syncthreads();
        if (h == 0 && valid) {
            float o = P.params[OFF_B5];
#pragma unroll
            for (int g = 0; g < NGROUP; ++g) o += s_row[g * TILE + m];
            P.out[i] = o;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && !tc::mbar_wait(c.bar_tma, c.ph_tma, WAIT_NS)) atomicExch(P.err, 3);
    ctx_finish(c);
}

struct BwdParams {
    const float* params;
    const float* pred;    // [batch]
    const float* y;       // dataset targets
    const uint32_t* step;
    uint64_t n_data;
    uint32_t batch;
    float scale;          // d loss / d pred = scale (pred - y)
    float* dout;          // [batch]
    const __nv_bfloat16* zt[4];
    __nv_bfloat16* dzt[4];
    int* err;
};

// Backward pass of one tile through the hidden layers (SiLU'(z) from the
// stored pre-activations); dZ_l^T is written for the weight gradients.
__global__ void __launch_bounds__(THREADS, 1) mlp_bwd_kernel(const BwdParams P, const __grid_constant__ Maps maps)
{
    extern __shared__ unsigned char raw_sm[];
    Ctx c;
    ctx_init(c, raw_sm, P.err);
    stage_params(c, P.params);
    load_weights(c, &maps.wt[2], 4);
    __syncthreads();
    const int m = row_of_thread(), h = group_of_thread();
    float* s_row = reinterpret_cast<float*>(c.sm + SM_ROW);
    const float* w5 = reinterpret_cast<const float*>(c.sm + SM_W5);
    const size_t ld = P.batch;
    const uint32_t ntiles = (P.batch + TILE - 1) / TILE;
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint32_t i = tile * TILE + m;
        const bool valid = i < P.batch;
        if (h == 0) {
            float d = 0.f;
            if (valid) {
                const uint64_t row = ((uint64_t)(*P.step) * P.batch + i) % P.n_data;
                d = P.scale * (P.pred[i] - P.y[row]);
                P.dout[i] = d;
            }
            s_row[m] = d;
        }
        __syncthreads();
        const float dout = s_row[m];
        // dZ4 = dout w5 SiLU'(z4)
        for (int ch = 0; ch < GCOLS / 32; ++ch) {
            const int col0 = GCOLS * h + 32 * ch;
            float v[32];
            // all loads of the chunk first (they may not pass the stores below)
#pragma unroll
            for (int j = 0; j < 32; ++j)
                v[j] = valid ? __bfloat162float(P.zt[3][(size_t)(col0 + j) * ld + i]) : 0.f;
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = valid ? dout * w5[col0 + j] * dsilu(v[j]) : 0.f;
            if (valid) {
#pragma unroll
                for (int j = 0; j < 32; ++j) P.dzt[3][(size_t)(col0 + j) * ld + i] = __float2bfloat16_rn(v[j]);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) st_row8(c.sm + SM_A, m, col0 + 8 * q, v + 8 * q);
        }
        for (int l = 3; l >= 1; --l) {
            publish_smem();
            issue_layer(c, SM_A, 4);       // dH_{l-1} = dZ_l W_l  (B = W_l^T)
            wait_layer(c);
            if (l > 1) load_weights(c, &maps.wt[l - 2], 4);
            else load_weights(c, &maps.wt[2], 4);   // next tile starts again at W4^T
            for (int ch = 0; ch < GCOLS / 32; ++ch) {
                const int col0 = GCOLS * h + 32 * ch;
                float z[32], v[32];
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    z[j] = valid ? __bfloat162float(P.zt[l - 1][(size_t)(col0 + j) * ld + i]) : 0.f;
                tc::tmem_ld32(tmem_addr(c, col0), v);
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = valid ? v[j] * dsilu(z[j]) : 0.f;
                if (valid) {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        P.dzt[l - 1][(size_t)(col0 + j) * ld + i] = __float2bfloat16_rn(v[j]);
                }
                if (l > 1) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) st_row8(c.sm + SM_A, m, col0 + 8 * q, v + 8 * q);
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
    }
    if (threadIdx.x == 0 && !tc::mbar_wait(c.bar_tma, c.ph_tma, WAIT_NS)) atomicExch(P.err, 4);
    ctx_finish(c);
}

// Weight gradients dW_l[out][in] = sum_b dZ_l^T[out][b] H_{l-1}^T[in][b]:
// both 128-row halves of `out` per CTA into two TMEM accumulators (columns
// 0..255 and 256..511), so that H^T is read once per layer; N = 256 (64 for
// layer 1), K = the batch, split over CTAs; 3-stage TMA pipeline (a stage
// holds the two dZ^T halves and the H^T block); FP32 vector atomics into the
// gradient.
constexpr int WG_STAGES = 3;
constexpr uint32_t WG_A_BYTES = 32768, WG_B_BYTES = 32768;   // A: two 128 x 64 halves
constexpr size_t WG_SMEM = (size_t)WG_STAGES * (WG_A_BYTES + WG_B_BYTES) + 256 + 1024;

struct WgMaps {
    CUtensorMap dz[4];   // dZ_l^T [256][batch], box {64, 128}
    CUtensorMap h[4];    // index 0: X^T [64][batch] box {64, 64}; l>0: H_l^T [256][batch] box {64, 256}
};

struct WgParams {
    float* grad;
    uint32_t kb_total;   // batch / 64
    uint32_t kb_per;     // K blocks per CTA
    int* err;
};

constexpr int WG_THREADS = 256;

__global__ void __launch_bounds__(WG_THREADS, 1) wgrad_kernel(const WgParams P, const __grid_constant__ WgMaps maps)
{
    extern __shared__ unsigned char raw_sm[];
    unsigned char* sm = aligned_base(raw_sm);
    const int layer = blockIdx.z;          // 0..3
    const uint32_t kb0 = blockIdx.x * P.kb_per;
    const uint32_t nkb = min(P.kb_per, P.kb_total > kb0 ? P.kb_total - kb0 : 0u);
    const int N = layer == 0 ? 64 : 256;
    const uint32_t bbytes = layer == 0 ? 8192u : WG_B_BYTES;
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + WG_STAGES * (WG_A_BYTES + WG_B_BYTES));
    uint64_t* empty = full + WG_STAGES;
    uint64_t* done = empty + WG_STAGES;
    uint32_t* taddr = reinterpret_cast<uint32_t*>(done + 1);
    if (threadIdx.x == 0) {
        for (int s = 0; s < WG_STAGES; ++s) {
            tc::mbar_init(full + s, 1);
            tc::mbar_init(empty + s, 1);
        }
        tc::mbar_init(done, 1);
        tc::fence_mbar_init();
    }
    if (threadIdx.x < 32) tc::tmem_alloc(taddr, 512);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *taddr;
    auto a_buf = [&](int s) { return sm + s * (WG_A_BYTES + WG_B_BYTES); };
    auto b_buf = [&](int s) { return sm + s * (WG_A_BYTES + WG_B_BYTES) + WG_A_BYTES; };
    auto load = [&](int s, uint32_t kb) {
        tc::mbar_arrive_expect_tx(full + s, WG_A_BYTES + bbytes);
        tc::tma_load_2d(a_buf(s), &maps.dz[layer], (int)(kb * 64), 0, full + s);
        tc::tma_load_2d(a_buf(s) + WG_A_BYTES / 2, &maps.dz[layer], (int)(kb * 64), 128, full + s);
        tc::tma_load_2d(b_buf(s), &maps.h[layer], (int)(kb * 64), 0, full + s);
    };
    if (threadIdx.x == 0 && nkb > 0) {
        const uint32_t idesc = tc::idesc_bf16(TILE, N);
        const int pro = (int)(nkb < (uint32_t)WG_STAGES ? nkb : (uint32_t)WG_STAGES);
        for (int s = 0; s < pro; ++s) load(s, kb0 + s);
        bool ok = true;
        for (uint32_t it = 0; it < nkb; ++it) {
            const int s = (int)(it % WG_STAGES);
            ok = ok && tc::mbar_wait(full + s, (it / WG_STAGES) & 1u, WAIT_NS);
            tc::fence_after_sync();
            for (int k = 0; k < 4; ++k) {
                const uint64_t bd = tc::desc_sw128(tc::smem_u32(b_buf(s)) + k * 32);
                const uint64_t a0 = tc::desc_sw128(tc::smem_u32(a_buf(s)) + k * 32);
                const uint64_t a1 = tc::desc_sw128(tc::smem_u32(a_buf(s) + WG_A_BYTES / 2) + k * 32);
                tc::mma_bf16(tmem, a0, bd, idesc, (it | k) ? 1u : 0u);
                tc::mma_bf16(tmem + 256u, a1, bd, idesc, (it | k) ? 1u : 0u);
            }
            tc::mma_commit(empty + s);
            // refill the stage used one iteration ago (its MMAs are done or nearly)
            if (it >= 1) {
                const uint32_t prev = it - 1;
                const int ps = (int)(prev % WG_STAGES);
                const uint32_t next = prev + WG_STAGES;
                if (next < nkb) {
                    ok = ok && tc::mbar_wait(empty + ps, (prev / WG_STAGES) & 1u, WAIT_NS);
                    load(ps, kb0 + next);
                }
            }
        }
        tc::mma_commit(done);
        if (!ok) atomicExch(P.err, 5);
    }
    __syncthreads();
    if (nkb > 0) {
        if (!tc::mbar_wait(done, 0, WAIT_NS)) atomicExch(P.err, 6);
        tc::fence_after_sync();
        const int m = row_of_thread(), h = (int)(threadIdx.x >> 7);   // 256 threads: two column halves
        const int ncols = N / 2;                 // columns per thread
        const int off = layer == 0 ? OFF_W1 : (layer == 1 ? OFF_W2 : (layer == 2 ? OFF_W3 : OFF_W4));
        const uint32_t lane_base = (uint32_t)(32 * ((threadIdx.x >> 5) & 3)) << 16;
        for (int hh = 0; hh < 2; ++hh) {
            float* g = P.grad + off + (size_t)(hh * 128 + m) * N;
            for (int ch = 0; ch < ncols / 32; ++ch) {
                const int col0 = h * ncols + 32 * ch;
                float v[32];
                tc::tmem_ld32(tmem + lane_base + (uint32_t)(hh * 256 + col0), v);
                // 16-byte vector reductions (four element-wise FP32 atomic adds
                // each): the gradient rows and col0 are multiples of 4 floats
#pragma unroll
                for (int j = 0; j < 32; j += 4)
                    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(g + col0 + j), "f"(v[j]),
                                 "f"(v[j + 1]), "f"(v[j + 2]), "f"(v[j + 3])
                                 : "memory");
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x < 32) tc::tmem_dealloc(tmem, 512);
}

// Row reductions of the backward pass: db2..db4 (row sums of dZ_2..4^T),
// dw5 = sum_b dout_b h4_b, db5 = sum_b dout_b. One CTA per output.
__device__ __forceinline__ float bf16_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t u) { return __uint_as_float(u & 0xFFFF0000u); }

// batch is a multiple of 128, so every row is 16-byte aligned and reads as
// uint4 (8 BF16) / float4 vectors. FP32 sums of 8, Kahan-compensated per
// thread, then an FP64 tree over the block (the FP64 pipe is slow on this
// part: only the final combination uses it).
__global__ void __launch_bounds__(256) rowsum_kernel(float* grad, const __nv_bfloat16* dz2,
                                                     const __nv_bfloat16* dz3, const __nv_bfloat16* dz4,
                                                     const __nv_bfloat16* ht4, const float* dout, uint32_t batch)
{
    const int r = blockIdx.x;   // 0..767: db2..db4; 768..1023: dw5; 1024: db5
    const uint32_t n8 = batch / 8;
    float s = 0.f, comp = 0.f;
    auto add = [&](float v) {
        const float y = v - comp;
        const float t = s + y;
        comp = (t - s) - y;
        s = t;
    };
    const float4* d4 = reinterpret_cast<const float4*>(dout);
    if (r < 768) {
        const __nv_bfloat16* dz = r < 256 ? dz2 : (r < 512 ? dz3 : dz4);
        const uint4* row = reinterpret_cast<const uint4*>(dz + (size_t)(r % 256) * batch);
        for (uint32_t i = threadIdx.x; i < n8; i += blockDim.x) {
            const uint4 u = row[i];
            add(((bf16_lo(u.x) + bf16_hi(u.x)) + (bf16_lo(u.y) + bf16_hi(u.y))) +
                ((bf16_lo(u.z) + bf16_hi(u.z)) + (bf16_lo(u.w) + bf16_hi(u.w))));
        }
    } else if (r < 1024) {
        const uint4* row = reinterpret_cast<const uint4*>(ht4 + (size_t)(r - 768) * batch);
        for (uint32_t i = threadIdx.x; i < n8; i += blockDim.x) {
            const uint4 u = row[i];
            const float4 a = d4[2 * i], b = d4[2 * i + 1];
            float p = a.x * bf16_lo(u.x);
            p = fmaf(a.y, bf16_hi(u.x), p);
            p = fmaf(a.z, bf16_lo(u.y), p);
            p = fmaf(a.w, bf16_hi(u.y), p);
            p = fmaf(b.x, bf16_lo(u.z), p);
            p = fmaf(b.y, bf16_hi(u.z), p);
            p = fmaf(b.z, bf16_lo(u.w), p);
            p = fmaf(b.w, bf16_hi(u.w), p);
            add(p);
        }
    } else {
        for (uint32_t i = threadIdx.x; i < n8; i += blockDim.x) {
            const float4 a = d4[2 * i], b = d4[2 * i + 1];
            add(((a.x + a.y) + (a.z + a.w)) + ((b.x + b.y) + (b.z + b.w)));
        }
    }
    double t = (double)s - (double)comp;
    __shared__ double red[8];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        if (r < 768) grad[OFF_B1 + 256 + r] = (float)tot;        // b2, b3, b4
        else if (r < 1024) grad[OFF_W5 + (r - 768)] = (float)tot;
        else grad[OFF_B5] = (float)tot;
    }
}

struct AdamParams {
    float* p;
    float* g;
    float* m;
    float* v;
    uint32_t* step;
    float lr0;
    uint32_t total_steps;
    __nv_bfloat16* w1;
    __nv_bfloat16* w[3];
    __nv_bfloat16* wt[3];
    float* epi;              // epilogue constants of the trace: b_l / 2, w5, b5
};

// Adam (beta 0.9 / 0.999, eps 1e-8, cosine learning-rate decay) on the FP32
// master copy; writes the BF16 weights and their transposes, zeroes the
// gradient. The last CTA to finish advances the step counter.
__global__ void adam_kernel(AdamParams A, unsigned int* done_ctr)
{
    const uint32_t t = *A.step + 1;
    const float lr = A.lr0 * 0.5f * (1.0f + cospif(fminf((float)(t - 1) / (float)max(A.total_steps, 1u), 1.0f)));
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NPARAM; i += gridDim.x * blockDim.x) {
        const float g = A.g[i];
        const float mm = b1 * A.m[i] + (1.0f - b1) * g;
        const float vv = b2 * A.v[i] + (1.0f - b2) * g * g;
        A.m[i] = mm;
        A.v[i] = vv;
        float p = A.p[i] - lr * (mm / c1) / (sqrtf(vv / c2) + 1e-8f);
        if (i >= OFF_B1 && i < OFF_B1 + 256) p = 0.0f;   // layer-1 bias lives in W1[:, 63]
        A.p[i] = p;
        A.g[i] = 0.0f;
        const __nv_bfloat16 pb = __float2bfloat16_rn(p);
        if (i < OFF_W2) {
            A.w1[i] = pb;
        } else if (i < OFF_B1) {
            const int l = (i - OFF_W2) / NPARAM_W, k = (i - OFF_W2) % NPARAM_W;
            const int out = k / H, in = k % H;
            A.w[l][k] = pb;
            A.wt[l][in * H + out] = pb;
        } else {
            A.epi[i - OFF_B1] = i < OFF_W5 ? 0.5f * p : p;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(done_ctr, 1u) == gridDim.x - 1) {
            *done_ctr = 0u;
            *A.step = t;
        }
    }
}

// Deterministic initialisation: uniform(-1, 1) * sqrt(6 / fan_in) for
// hidden weights (Philox), zero biases, small output layer.
__global__ void init_kernel(float* p, uint64_t seed)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NPARAM; i += gridDim.x * blockDim.x) {
        const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
        const uint4 r = philox(make_uint4(6u, 0x80000002u, (uint32_t)i, 0u), key);
        const float u = 2.0f * u01<float>(r.x) - 1.0f;
        float v = 0.0f;
        if (i < OFF_W2) v = ((i % KIN) == 63) ? 0.0f : u * sqrtf(6.0f / 16.0f);
        else if (i < OFF_B1) v = u * sqrtf(6.0f / (float)H);
        else if (i >= OFF_W5 && i < OFF_B5) v = u * sqrtf(6.0f / (float)H) * 0.1f;
        p[i] = v;
    }
}

}  // namespace sur
}  // namespace sas

// ------------------------------------------------------------ host side

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 2D BF16 tensor [outer][inner] (inner contiguous), 128-byte swizzle.
bool make_map(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint32_t box_inner,
              uint32_t box_outer)
{
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {inner * 2};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

struct sas_surrogate {
    sas_surrogate_box box;
    sur::Box dbox;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    float* d_p = nullptr;
    float* d_g = nullptr;
    float* d_m = nullptr;
    float* d_v = nullptr;
    uint32_t* d_step = nullptr;
    unsigned int* d_ctr = nullptr;
    __nv_bfloat16* d_w1 = nullptr;
    __nv_bfloat16* d_w[3] = {nullptr, nullptr, nullptr};
    __nv_bfloat16* d_wt[3] = {nullptr, nullptr, nullptr};
    float* d_epi = nullptr;   // [NPARAM - OFF_B1] trace epilogue constants
    Maps maps;
    float* d_tab = nullptr;
    sur::Tables tabs;
    std::vector<float> bucket_sp;
    sur::Raw* d_raw = nullptr;
    float* d_y = nullptr;
    uint64_t n_data = 0, cap_data = 0;
    uint32_t batch = 0;
    __nv_bfloat16* d_xt = nullptr;
    __nv_bfloat16* d_zt[4] = {};
    __nv_bfloat16* d_ht[4] = {};
    __nv_bfloat16* d_dzt[4] = {};
    float* d_pred = nullptr;
    float* d_dout = nullptr;
    sur::WgMaps wg;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t gx = nullptr;
    float g_lr = 0.f;
    uint32_t g_total = 0;
    int* d_err = nullptr;
    cudaStream_t cap = nullptr;
    cudaStream_t side = nullptr;        // the row sums, beside the weight gradients
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    uint64_t stall_ns = 0;   // test hook for the next sas_surrogate_eval
};

namespace {

void free_batch_buffers(sas_surrogate* s)
{
    cudaFree(s->d_xt);
    s->d_xt = nullptr;
    for (int l = 0; l < 4; ++l) {
        cudaFree(s->d_zt[l]);
        cudaFree(s->d_ht[l]);
        cudaFree(s->d_dzt[l]);
        s->d_zt[l] = s->d_ht[l] = s->d_dzt[l] = nullptr;
    }
    cudaFree(s->d_pred);
    cudaFree(s->d_dout);
    s->d_pred = s->d_dout = nullptr;
    if (s->gx) cudaGraphExecDestroy(s->gx);
    if (s->g) cudaGraphDestroy(s->g);
    s->gx = nullptr;
    s->g = nullptr;
    s->batch = 0;
}

sas_status ensure_batch(sas_surrogate* s, uint32_t batch)
{
    if (batch == s->batch) return SAS_OK;
    if (batch == 0 || batch % TILE != 0 || batch > (1u << 22))
        return set_error(SAS_ERR_ARG, "batch must be a positive multiple of 128 (<= 4194304)");
    SAS_CUDA_S(cudaStreamSynchronize(s->stream), "sync");
    free_batch_buffers(s);
    const size_t hb = (size_t)H * batch * sizeof(__nv_bfloat16);
    SAS_CUDA_S(cudaMalloc(&s->d_xt, (size_t)KIN * batch * sizeof(__nv_bfloat16)), "alloc xt");
    SAS_CUDA_S(cudaMemset(s->d_xt, 0, (size_t)KIN * batch * sizeof(__nv_bfloat16)), "zero xt");
    for (int l = 0; l < 4; ++l) {
        SAS_CUDA_S(cudaMalloc(&s->d_zt[l], hb), "alloc zt");
        SAS_CUDA_S(cudaMalloc(&s->d_ht[l], hb), "alloc ht");
        SAS_CUDA_S(cudaMalloc(&s->d_dzt[l], hb), "alloc dzt");
    }
    SAS_CUDA_S(cudaMalloc(&s->d_pred, batch * sizeof(float)), "alloc pred");
    SAS_CUDA_S(cudaMalloc(&s->d_dout, batch * sizeof(float)), "alloc dout");
    bool ok = true;
    for (int l = 0; l < 4; ++l) ok = ok && make_map(&s->wg.dz[l], s->d_dzt[l], batch, H, 64, 128);
    ok = ok && make_map(&s->wg.h[0], s->d_xt, batch, KIN, 64, 64);
    for (int l = 1; l < 4; ++l) ok = ok && make_map(&s->wg.h[l], s->d_ht[l - 1], batch, H, 64, 256);
    if (!ok) return set_error(SAS_ERR_CUDA, "cuTensorMapEncodeTiled failed (activation maps)");
    s->batch = batch;
    return SAS_OK;
}

// forward (training) + backward + weight gradients + row sums on the rows
// of the current step; adam = false leaves the gradient in d_g.
sas_status enqueue_step(sas_surrogate* s, const sur::Raw* raw, const float* y, uint64_t n_data, bool adam,
                        cudaStream_t st)
{
    const uint32_t B = s->batch;
    const uint32_t ntiles = B / TILE;
    const int grid = std::min<int>((int)ntiles, s->sm_count);
    sur::FwdParams F;
    std::memset(&F, 0, sizeof(F));
    F.box = s->dbox;
    F.raw = raw;
    F.n_data = n_data;
    F.step = s->d_step;
    F.batch = B;
    F.params = s->d_p;
    F.out = s->d_pred;
    F.xt = s->d_xt;
    for (int l = 0; l < 4; ++l) {
        F.zt[l] = s->d_zt[l];
        F.ht[l] = s->d_ht[l];
    }
    F.err = s->d_err;
    if (B % 256u == 0u) {
        // the warp-specialised kernel (two 128-row tiles in flight per SM,
        // weights streamed through a ring) in its training mode
        sur::STParams S;
        std::memset(&S, 0, sizeof(S));
        S.box = s->dbox;
        S.epi = s->d_epi;
        S.n_pairs = B / 256u;
        S.err = s->d_err;
        S.raw = raw;
        S.n_data = n_data;
        S.step = s->d_step;
        S.batch = B;
        S.out = s->d_pred;
        S.xt = s->d_xt;
        for (int l = 0; l < 4; ++l) {
            S.zt[l] = s->d_zt[l];
            S.ht[l] = s->d_ht[l];
        }
        const int g2 = (int)std::min<uint32_t>((uint32_t)s->sm_count, S.n_pairs);
        sur::sur_trace_kernel<sur::MODE_TRAIN><<<g2, sur::ST_THREADS, sur::S2_SMEM, st>>>(S, s->maps);
    } else {
        sur::mlp_fwd_kernel<true><<<grid, THREADS, SMEM_BYTES, st>>>(F, s->maps);
    }
    sur::BwdParams Bp;
    std::memset(&Bp, 0, sizeof(Bp));
    Bp.params = s->d_p;
    Bp.pred = s->d_pred;
    Bp.y = y;
    Bp.step = s->d_step;
    Bp.n_data = n_data;
    Bp.batch = B;
    Bp.scale = 2.0f / (float)B;      // mean squared error of log P
    Bp.dout = s->d_dout;
    for (int l = 0; l < 4; ++l) {
        Bp.zt[l] = s->d_zt[l];
        Bp.dzt[l] = s->d_dzt[l];
    }
    Bp.err = s->d_err;
    if (B % 256u == 0u) {
        sur::STParams S;
        std::memset(&S, 0, sizeof(S));
        S.epi = s->d_epi;
        S.n_pairs = B / 256u;
        S.err = s->d_err;
        S.n_data = n_data;
        S.step = s->d_step;
        S.batch = B;
        S.pred = s->d_pred;
        S.y = y;
        S.scale = Bp.scale;
        S.dout = s->d_dout;
        for (int l = 0; l < 4; ++l) {
            S.zt[l] = s->d_zt[l];
            S.dzt[l] = s->d_dzt[l];
        }
        const int g2 = (int)std::min<uint32_t>((uint32_t)s->sm_count, S.n_pairs);
        sur::sur_trace_kernel<sur::MODE_BWD><<<g2, sur::ST_THREADS, sur::S2_SMEM, st>>>(S, s->maps);
    } else {
        sur::mlp_bwd_kernel<<<grid, THREADS, SMEM_BYTES, st>>>(Bp, s->maps);
    }
    sur::WgParams W;
    W.grad = s->d_g;
    W.kb_total = B / 64;
    // enough K splits to cover the SMs across the 4 layers
    uint32_t splits = std::max<uint32_t>(1, (uint32_t)((s->sm_count + 3) / 4));
    splits = std::min<uint32_t>(splits, W.kb_total);
    W.kb_per = (W.kb_total + splits - 1) / splits;
    splits = (W.kb_total + W.kb_per - 1) / W.kb_per;
    W.err = s->d_err;
    // The row sums (b2..b4, w5, b5) and the weight gradients (W1..W4) read
    // the backward's outputs and write disjoint parts of the gradient: the
    // row sums run on a side stream (a parallel branch of the captured
    // graph), so their HBM reads overlap the weight-gradient GEMMs.
    cudaError_t fe = cudaEventRecord(s->ev_fork, st);
    if (fe == cudaSuccess) fe = cudaStreamWaitEvent(s->side, s->ev_fork, 0);
    if (fe != cudaSuccess) return set_cuda_error(fe, "fork");
    sur::rowsum_kernel<<<1025, 256, 0, s->side>>>(s->d_g, s->d_dzt[1], s->d_dzt[2], s->d_dzt[3], s->d_ht[3],
                                                  s->d_dout, B);
    fe = cudaEventRecord(s->ev_join, s->side);
    if (fe != cudaSuccess) return set_cuda_error(fe, "join");
    sur::wgrad_kernel<<<dim3(splits, 1, 4), sur::WG_THREADS, sur::WG_SMEM, st>>>(W, s->wg);
    fe = cudaStreamWaitEvent(st, s->ev_join, 0);
    if (fe != cudaSuccess) return set_cuda_error(fe, "join");
    if (adam) {
        sur::AdamParams A;
        A.p = s->d_p;
        A.g = s->d_g;
        A.m = s->d_m;
        A.v = s->d_v;
        A.step = s->d_step;
        A.lr0 = s->g_lr;
        A.total_steps = s->g_total;
        A.w1 = s->d_w1;
        A.epi = s->d_epi;
        for (int l = 0; l < 3; ++l) {
            A.w[l] = s->d_w[l];
            A.wt[l] = s->d_wt[l];
        }
        sur::adam_kernel<<<(NPARAM + 255) / 256, 256, 0, st>>>(A, s->d_ctr);
    }
    const cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) return set_cuda_error(le, "training launch");
    return SAS_OK;
}

// Write the BF16 weights (and transposes) of the current FP32 parameters.
// Also the trace's epilogue constants: halved biases, w5, b5.
__global__ void publish_weights_kernel(const float* p, __nv_bfloat16* w1, __nv_bfloat16* w2, __nv_bfloat16* w3,
                                       __nv_bfloat16* w4, __nv_bfloat16* t2, __nv_bfloat16* t3, __nv_bfloat16* t4,
                                       float* epi)
{
    __nv_bfloat16* w[3] = {w2, w3, w4};
    __nv_bfloat16* t[3] = {t2, t3, t4};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NPARAM; i += gridDim.x * blockDim.x) {
        if (i >= OFF_B1) {
            epi[i - OFF_B1] = i < OFF_W5 ? 0.5f * p[i] : p[i];
            continue;
        }
        const __nv_bfloat16 b = __float2bfloat16_rn(p[i]);
        if (i < OFF_W2) {
            w1[i] = b;
        } else {
            const int l = (i - OFF_W2) / NPARAM_W, k = (i - OFF_W2) % NPARAM_W;
            w[l][k] = b;
            t[l][(k % H) * H + k / H] = b;
        }
    }
}

sas_status publish(sas_surrogate* s)
{
    publish_weights_kernel<<<256, 256, 0, s->stream>>>(s->d_p, s->d_w1, s->d_w[0], s->d_w[1], s->d_w[2],
                                                      s->d_wt[0], s->d_wt[1], s->d_wt[2], s->d_epi);
    SAS_CUDA_S(cudaGetLastError(), "publish weights");
    return SAS_OK;
}

sas_status check_err(sas_surrogate* s)
{
    int e = 0;
    SAS_CUDA_S(cudaMemcpyAsync(&e, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->stream), "read error flag");
    SAS_CUDA_S(cudaStreamSynchronize(s->stream), "sync");
    if (e != 0) {
        cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream);
        return set_error(SAS_ERR_TIMEOUT, "a bounded wait in a tensor-core kernel gave up (code " +
                                              std::to_string(e) + ")");
    }
    return SAS_OK;
}

sur::Box device_box(const sas_surrogate_box& b)
{
    sur::Box d;
    d.q_max = (float)b.q_max;
    d.r_min = (float)b.r_min;
    d.r_max = (float)b.r_max;
    d.l_min = (float)b.l_min;
    d.l_max = (float)b.l_max;
    d.so_min = (float)b.sigma_orient_min;
    d.so_max = (float)b.sigma_orient_max;
    d.sp_min = (float)b.poly_min;
    d.sp_max = (float)b.poly_max;
    d.u_max = (float)(0.5 * b.q_max * b.l_max);
    d.v_max = (float)(b.q_max * b.r_max);
    d.la_min = (float)std::log(0.5 * b.l_min / b.r_max);
    d.la_max = (float)std::log(0.5 * b.l_max / b.r_min);
    if (d.la_max <= d.la_min) d.la_max = d.la_min + 1.0f;   // a single aspect ratio
    d.n_four = b.n_fourier;
    d.four_w = 0.5f;
    d.n_buckets = b.n_buckets;
    d.n_poly = b.n_poly;
    d.n_gamma = b.n_gamma;
    d.n_psi = b.n_psi;
    d.kind = b.model == SAS_ELLIPSOID ? SAS_ELLIPSOID : SAS_CYLINDER;
    return d;
}

}  // namespace

// exposed to sas_api.cu / sas_batch.cu
namespace sas {

int surrogate_kind(const sas_surrogate* s) { return s->dbox.kind; }

// The body's length along its axis: the cylinder's L, the ellipsoid's 2 R_p.
static double axial_length(const sas_model_desc& m)
{
    return m.kind == SAS_ELLIPSOID ? 2.0 * m.radius_polar : m.length;
}

bool surrogate_covers(const sas_surrogate* s, const sas_model_desc& m)
{
    if (!s || m.kind != s->dbox.kind || m.precision != SAS_FP32 || m.isotropic) return false;
    if (m.sampling != SAS_QUADRATURE || m.poly_dist != SAS_POLY_SCHULZ) return false;   // trained on Schulz averages
    if (m.self_attenuation) return false;   // the surrogate trace attenuates with the instrument's mu only
    const sas_surrogate_box& b = s->box;
    if (m.n_poly != b.n_poly || m.n_gamma != b.n_gamma || m.n_psi != b.n_psi) return false;
    const double L = axial_length(m);
    return m.radius >= b.r_min && m.radius <= b.r_max && L >= b.l_min && L <= b.l_max &&
           m.sigma_orient >= b.sigma_orient_min && m.sigma_orient <= b.sigma_orient_max && m.poly >= b.poly_min &&
           m.poly <= b.poly_max && m.sld != m.sld_solvent;
}

sur::SurExp surrogate_exp(const sas_model_desc& m, bool in_box)
{
    sur::SurExp e;
    std::memset(&e, 0, sizeof(e));
    e.nx = (float)(std::sin(m.axis_theta) * std::cos(m.axis_phi));
    e.ny = (float)(std::sin(m.axis_theta) * std::sin(m.axis_phi));
    e.nz = (float)std::cos(m.axis_theta);
    e.R = (float)m.radius;
    e.L = (float)axial_length(m);
    e.so = (float)m.sigma_orient;
    e.sp = (float)m.poly;
    // <V^2> / <V> of the Schulz distribution of the radius r: c <r^4> / <r^2>
    // with V = c r^2 (c = pi L for the cylinder, 4 pi R_p / 3 for the
    // ellipsoid), <r^k> = R^k prod_{j=1..k} (z + j) / (z + 1)^k, z = 1/p^2 - 1
    double r2 = m.radius * m.radius, r4 = r2 * r2;
    if (m.poly > 0.0) {
        const double z = 1.0 / (m.poly * m.poly) - 1.0;
        r2 *= (z + 2.0) / (z + 1.0);
        r4 *= (z + 2.0) * (z + 3.0) * (z + 4.0) / ((z + 1.0) * (z + 1.0) * (z + 1.0));
    }
    const double drho = m.sld - m.sld_solvent;
    const double c = m.kind == SAS_ELLIPSOID ? 4.0 * M_PI * m.radius_polar / 3.0 : M_PI * m.length;
    e.scale_p = (float)(m.volume_fraction * drho * drho * c * r4 / r2);
    e.in_box = in_box ? 1 : 0;
    return e;
}

cudaError_t launch_sur_trace(const sas_surrogate* s, const sur::STParams& P, int sm_count, cudaStream_t st)
{
    if (P.n_pairs == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(sur::sur_trace_kernel<sur::MODE_TRACE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sur::S2_SMEM);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<uint32_t>((uint32_t)sm_count, P.n_pairs);
    sur::sur_trace_kernel<sur::MODE_TRACE><<<grid, sur::ST_THREADS, sur::S2_SMEM, st>>>(P, s->maps);
    return cudaGetLastError();
}

uint64_t surrogate_pair_prefix(const std::vector<WorkItem>& items, std::vector<uint32_t>& prefix)
{
    prefix.resize(items.size());
    uint64_t n = 0;
    for (size_t i = 0; i < items.size(); ++i) {
        prefix[i] = (uint32_t)std::min<uint64_t>(n, 0xFFFFFFFFull);
        n += (items[i].n + 255u) / 256u;
    }
    return n;
}

const float* surrogate_epi(const sas_surrogate* s) { return s->d_epi; }
sur::Box surrogate_dbox(const sas_surrogate* s) { return s->dbox; }
int* surrogate_err(const sas_surrogate* s) { return s->d_err; }

sas_status surrogate_take_error(const sas_surrogate* s, cudaStream_t st)
{
    int e = 0;
    cudaError_t ce = cudaMemcpyAsync(&e, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) return set_cuda_error(ce, "read surrogate error flag");
    if (e == 0) return SAS_OK;
    cudaMemsetAsync(s->d_err, 0, sizeof(int), st);
    return set_error(SAS_ERR_TIMEOUT, "a bounded wait in the surrogate trace gave up (code " + std::to_string(e) +
                                          "); the detector is incomplete");
}

}  // namespace sas

extern "C" {

sas_status sas_create_surrogate(const sas_surrogate_box* box, uint64_t seed, void* stream, sas_surrogate** out)
{
    if (!out || !box) return set_error(SAS_ERR_ARG, "NULL argument");
    *out = nullptr;
    const sas_surrogate_box& b = *box;
    if (!(b.q_max > 0 && b.r_min > 0 && b.r_max >= b.r_min && b.l_min > 0 && b.l_max >= b.l_min &&
          b.sigma_orient_min > 0 && b.sigma_orient_max >= b.sigma_orient_min && b.poly_min > 0 &&
          b.poly_max >= b.poly_min && b.poly_max < 1.0))
        return set_error(SAS_ERR_ARG, "invalid surrogate box");
    if (b.model != 0 && b.model != SAS_CYLINDER && b.model != SAS_ELLIPSOID)
        return set_error(SAS_ERR_ARG, "surrogate model must be SAS_CYLINDER or SAS_ELLIPSOID");
    if (b.n_poly < 1 || b.n_poly > sur::MAX_POLY || b.n_gamma < 1 || b.n_gamma > sur::MAX_GL || b.n_psi < 1 ||
        b.n_psi > sur::MAX_GL || b.n_buckets < 1 || b.n_buckets > sur::MAX_BUCKETS || b.n_fourier < 0 ||
        b.n_fourier > 13)
        return set_error(SAS_ERR_ARG, "invalid surrogate quadrature sizes");
    if (!encode_fn()) return set_error(SAS_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    sas_surrogate* s = new (std::nothrow) sas_surrogate();
    if (!s) return set_error(SAS_ERR_OOM, "host allocation failed");
    auto bail = [&](sas_status st) { sas_destroy_surrogate(s); return st; };
    s->box = b;
    s->dbox = device_box(b);
    s->stream = (cudaStream_t)stream;
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming);
    const size_t pb = (size_t)NPARAM * sizeof(float);
    if (ce == cudaSuccess) ce = cudaMalloc(&s->d_p, pb);
    if (ce == cudaSuccess) ce = cudaMalloc(&s->d_g, pb);
    if (ce == cudaSuccess) ce = cudaMalloc(&s->d_m, pb);
    if (ce == cudaSuccess) ce = cudaMalloc(&s->d_v, pb);
    if (ce == cudaSuccess) ce = cudaMalloc(&s->d_step, sizeof(uint32_t));
    if (ce == cudaSuccess) ce = cudaMalloc(&s->d_ctr, sizeof(unsigned int));
    if (ce == cudaSuccess) ce = cudaMalloc(&s->d_err, sizeof(int));
    if (ce == cudaSuccess) ce = cudaMalloc(&s->d_w1, (size_t)NPARAM_W1 * 2);
    if (ce == cudaSuccess) ce = cudaMalloc(&s->d_epi, (size_t)(NPARAM - OFF_B1) * sizeof(float));
    for (int l = 0; l < 3 && ce == cudaSuccess; ++l) {
        ce = cudaMalloc(&s->d_w[l], (size_t)NPARAM_W * 2);
        if (ce == cudaSuccess) ce = cudaMalloc(&s->d_wt[l], (size_t)NPARAM_W * 2);
    }
    if (ce != cudaSuccess) return bail(set_cuda_error(ce, "sas_create_surrogate allocation"));
    cudaMemset(s->d_g, 0, pb);
    cudaMemset(s->d_m, 0, pb);
    cudaMemset(s->d_v, 0, pb);
    cudaMemset(s->d_step, 0, sizeof(uint32_t));
    cudaMemset(s->d_ctr, 0, sizeof(unsigned int));
    cudaMemset(s->d_err, 0, sizeof(int));
    bool ok = make_map(&s->maps.w1, s->d_w1, KIN, H, 64, 256);
    for (int l = 0; l < 3; ++l) {
        ok = ok && make_map(&s->maps.w[l], s->d_w[l], H, H, 64, 256);
        ok = ok && make_map(&s->maps.wt[l], s->d_wt[l], H, H, 64, 256);
    }
    if (!ok) return bail(set_error(SAS_ERR_CUDA, "cuTensorMapEncodeTiled failed (weight maps)"));
    // quadrature tables of the exact targets (FP64 on the host, FP32 on the device)
    std::vector<double> xg(b.n_gamma), wg(b.n_gamma), xp(b.n_psi), wp(b.n_psi);
    gauss_legendre(b.n_gamma, xg.data(), wg.data());
    gauss_legendre(b.n_psi, xp.data(), wp.data());
    std::vector<float> tab;
    auto push = [&](const std::vector<double>& v) {
        for (double x : v) tab.push_back((float)x);
    };
    push(xg);
    push(wg);
    push(xp);
    push(wp);
    s->bucket_sp.resize(b.n_buckets);
    std::vector<double> px((size_t)b.n_buckets * b.n_poly, 1.0), pw((size_t)b.n_buckets * b.n_poly, 0.0);
    for (int k = 0; k < b.n_buckets; ++k) {
        const double sp = b.n_buckets == 1 ? 0.5 * (b.poly_min + b.poly_max)
                                           : b.poly_min + (b.poly_max - b.poly_min) * k / (b.n_buckets - 1);
        s->bucket_sp[k] = (float)sp;
        std::vector<double> r(b.n_poly), w(b.n_poly);
        schulz_nodes(1.0, (double)(float)sp, b.n_poly, r.data(), w.data());
        double norm = 0.0;
        for (int i = 0; i < b.n_poly; ++i) norm += w[i] * std::pow(r[i], 4);
        for (int i = 0; i < b.n_poly; ++i) {
            px[(size_t)k * b.n_poly + i] = r[i];
            pw[(size_t)k * b.n_poly + i] = w[i] * std::pow(r[i], 4) / norm;
        }
    }
    for (float v : s->bucket_sp) tab.push_back(v);
    push(px);
    push(pw);
    // (x^2, w) pairs of every bucket for one 8-byte load per radial term
    if (tab.size() % 2) tab.push_back(0.f);
    const size_t off_x2w = tab.size();
    for (size_t i = 0; i < px.size(); ++i) {
        tab.push_back((float)(px[i] * px[i]));
        tab.push_back((float)pw[i]);
    }
    // (cos, sin) of the psi nodes
    const size_t off_psi = tab.size();
    for (int k = 0; k < b.n_psi; ++k) {
        const double psi = M_PI * (xp[k] + 1.0);
        tab.push_back((float)std::cos(psi));
        tab.push_back((float)std::sin(psi));
    }
    ce = cudaMalloc(&s->d_tab, tab.size() * sizeof(float));
    if (ce == cudaSuccess) ce = cudaMemcpy(s->d_tab, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) return bail(set_cuda_error(ce, "surrogate tables"));
    const float* t = s->d_tab;
    s->tabs.gl_g = t;
    s->tabs.glw_g = t + b.n_gamma;
    s->tabs.gl_p = t + 2 * b.n_gamma;
    s->tabs.glw_p = t + 2 * b.n_gamma + b.n_psi;
    s->tabs.bucket_sp = t + 2 * b.n_gamma + 2 * b.n_psi;
    s->tabs.poly_x = s->tabs.bucket_sp + b.n_buckets;
    s->tabs.poly_w = s->tabs.poly_x + (size_t)b.n_buckets * b.n_poly;
    s->tabs.poly_x2w = reinterpret_cast<const float2*>(t + off_x2w);
    s->tabs.psi_cs = reinterpret_cast<const float2*>(t + off_psi);
    sur::init_kernel<<<256, 256, 0, s->stream>>>(s->d_p, seed);
    sas_status st = publish(s);
    if (st != SAS_OK) return bail(st);
    SAS_CUDA_S(cudaFuncSetAttribute(sur::mlp_fwd_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES), "attr");
    SAS_CUDA_S(cudaFuncSetAttribute(sur::mlp_fwd_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES), "attr");
    SAS_CUDA_S(cudaFuncSetAttribute(sur::mlp_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES), "attr");
    SAS_CUDA_S(cudaFuncSetAttribute(sur::wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sur::WG_SMEM), "attr");
    SAS_CUDA_S(cudaFuncSetAttribute(sur::sur_trace_kernel<sur::MODE_TRAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sur::S2_SMEM), "attr");
    SAS_CUDA_S(cudaFuncSetAttribute(sur::sur_trace_kernel<sur::MODE_BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sur::S2_SMEM), "attr");
    SAS_CUDA_S(cudaStreamSynchronize(s->stream), "sync");
    *out = s;
    return SAS_OK;
}

sas_status sas_surrogate_generate(sas_surrogate* s, uint64_t n, uint64_t seed)
{
    if (!s || n == 0) return set_error(SAS_ERR_ARG, "bad arguments");
    if (n > s->cap_data) {
        SAS_CUDA_S(cudaStreamSynchronize(s->stream), "sync");
        cudaFree(s->d_raw);
        cudaFree(s->d_y);
        s->d_raw = nullptr;
        s->d_y = nullptr;
        SAS_CUDA_S(cudaMalloc(&s->d_raw, n * sizeof(sur::Raw)), "alloc dataset");
        SAS_CUDA_S(cudaMalloc(&s->d_y, n * sizeof(float)), "alloc dataset");
        s->cap_data = n;
    }
    s->n_data = n;
    const int blocks = s->sm_count * 8;
    sur::data_kernel<<<blocks, 256, 0, s->stream>>>(s->dbox, s->tabs, seed, 0, n, s->d_raw, s->d_y, 1);
    SAS_CUDA_S(cudaGetLastError(), "data kernel");
    return SAS_OK;
}

sas_status sas_surrogate_exact(sas_surrogate* s, const void* raw, size_t n, float* log_p)
{
    if (!s || !raw || !log_p) return set_error(SAS_ERR_ARG, "NULL argument");
    if (n == 0) return SAS_OK;
    sur::data_kernel<<<s->sm_count * 8, 256, 0, s->stream>>>(s->dbox, s->tabs, 0, 0, n,
                                                             (sur::Raw*)const_cast<void*>(raw), log_p, 0);
    SAS_CUDA_S(cudaGetLastError(), "exact kernel");
    return SAS_OK;
}

sas_status sas_surrogate_dataset(const sas_surrogate* s, const void** raw, const float** log_p, uint64_t* n)
{
    if (!s) return set_error(SAS_ERR_ARG, "NULL argument");
    if (raw) *raw = s->d_raw;
    if (log_p) *log_p = s->d_y;
    if (n) *n = s->n_data;
    return SAS_OK;
}

sas_status sas_surrogate_eval(sas_surrogate* s, const void* raw, size_t n, float* log_p)
{
    if (!s || !raw || !log_p) return set_error(SAS_ERR_ARG, "NULL argument");
    if (n == 0) return SAS_OK;
    if (n > 0xFFFFFFFFull) return set_error(SAS_ERR_ARG, "too many rows");
    sur::FwdParams F;
    std::memset(&F, 0, sizeof(F));
    F.box = s->dbox;
    F.raw = (const sur::Raw*)raw;
    F.n_data = n;
    F.step = nullptr;
    F.batch = (uint32_t)n;
    F.first = 0;
    F.params = s->d_p;
    F.out = log_p;
    F.err = s->d_err;
    F.stall_ns = s->stall_ns;
    s->stall_ns = 0;
    const uint32_t ntiles = (uint32_t)((n + TILE - 1) / TILE);
    const int grid = (int)std::min<uint32_t>(ntiles, (uint32_t)s->sm_count);
    sur::mlp_fwd_kernel<false><<<grid, THREADS, SMEM_BYTES, s->stream>>>(F, s->maps);
    SAS_CUDA_S(cudaGetLastError(), "eval kernel");
    return check_err(s);
}

sas_status sas_surrogate_grad(sas_surrogate* s, const void* raw, const float* log_p, uint32_t n, float* grad_host,
                              size_t n_params)
{
    if (!s || !raw || !log_p || !grad_host) return set_error(SAS_ERR_ARG, "NULL argument");
    if (n_params != (size_t)NPARAM) return set_error(SAS_ERR_ARG, "n_params mismatch");
    sas_status st = ensure_batch(s, n);
    if (st != SAS_OK) return st;
    uint32_t saved = 0;
    SAS_CUDA_S(cudaMemcpyAsync(&saved, s->d_step, 4, cudaMemcpyDeviceToHost, s->stream), "read step");
    SAS_CUDA_S(cudaMemsetAsync(s->d_step, 0, 4, s->stream), "zero step");
    SAS_CUDA_S(cudaMemsetAsync(s->d_g, 0, (size_t)NPARAM * 4, s->stream), "zero grad");
    st = enqueue_step(s, (const sur::Raw*)raw, log_p, n, false, s->stream);
    if (st != SAS_OK) return st;
    SAS_CUDA_S(cudaMemcpyAsync(grad_host, s->d_g, (size_t)NPARAM * 4, cudaMemcpyDeviceToHost, s->stream), "read grad");
    SAS_CUDA_S(cudaMemsetAsync(s->d_g, 0, (size_t)NPARAM * 4, s->stream), "zero grad");
    SAS_CUDA_S(cudaMemcpyAsync(s->d_step, &saved, 4, cudaMemcpyHostToDevice, s->stream), "restore step");
    return check_err(s);
}

sas_status sas_surrogate_train(sas_surrogate* s, uint32_t n_steps, uint32_t batch, double lr, uint32_t total_steps)
{
    if (!s) return set_error(SAS_ERR_ARG, "NULL argument");
    if (s->n_data == 0) return set_error(SAS_ERR_STATE, "no training data: call sas_surrogate_generate");
    if (!(lr > 0.0)) return set_error(SAS_ERR_ARG, "lr must be > 0");
    sas_status st = ensure_batch(s, batch);
    if (st != SAS_OK) return st;
    if (!s->gx || s->g_lr != (float)lr || s->g_total != total_steps) {
        if (s->gx) cudaGraphExecDestroy(s->gx);
        if (s->g) cudaGraphDestroy(s->g);
        s->gx = nullptr;
        s->g = nullptr;
        s->g_lr = (float)lr;
        s->g_total = total_steps;
        SAS_CUDA_S(cudaStreamSynchronize(s->stream), "sync");
        SAS_CUDA_S(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
        sas_status e = enqueue_step(s, s->d_raw, s->d_y, s->n_data, true, s->cap);
        cudaError_t ce = cudaStreamEndCapture(s->cap, &s->g);
        if (e != SAS_OK) return e;
        if (ce != cudaSuccess) return set_cuda_error(ce, "end capture");
        SAS_CUDA_S(cudaGraphInstantiate(&s->gx, s->g, 0), "graph instantiate");
    }
    for (uint32_t i = 0; i < n_steps; ++i) SAS_CUDA_S(cudaGraphLaunch(s->gx, s->stream), "graph launch");
    return check_err(s);
}

sas_status sas_surrogate_get_params(const sas_surrogate* s, float* host, size_t n)
{
    if (!s || !host || n != (size_t)NPARAM) return set_error(SAS_ERR_ARG, "bad arguments");
    SAS_CUDA_S(cudaMemcpyAsync(host, s->d_p, n * 4, cudaMemcpyDeviceToHost, s->stream), "read params");
    SAS_CUDA_S(cudaStreamSynchronize(s->stream), "sync");
    return SAS_OK;
}

sas_status sas_surrogate_set_params(sas_surrogate* s, const float* host, size_t n)
{
    if (!s || !host || n != (size_t)NPARAM) return set_error(SAS_ERR_ARG, "bad arguments");
    SAS_CUDA_S(cudaMemcpyAsync(s->d_p, host, n * 4, cudaMemcpyHostToDevice, s->stream), "write params");
    sas_status st = publish(s);
    if (st != SAS_OK) return st;
    SAS_CUDA_S(cudaStreamSynchronize(s->stream), "sync");
    return SAS_OK;
}

sas_status sas_surrogate_test_stall(sas_surrogate* s, uint64_t wait_ns)
{
    if (!s) return set_error(SAS_ERR_ARG, "NULL argument");
    if (wait_ns > 1000000000ull) return set_error(SAS_ERR_ARG, "wait_ns above 1 s");
    s->stall_ns = wait_ns;
    return SAS_OK;
}

sas_status sas_surrogate_info(const sas_surrogate* s, size_t* n_params, uint32_t* steps_done)
{
    if (!s) return set_error(SAS_ERR_ARG, "NULL argument");
    if (n_params) *n_params = (size_t)NPARAM;
    if (steps_done) {
        SAS_CUDA_S(cudaMemcpyAsync(steps_done, s->d_step, 4, cudaMemcpyDeviceToHost, s->stream), "read step");
        SAS_CUDA_S(cudaStreamSynchronize(s->stream), "sync");
    }
    return SAS_OK;
}

sas_status sas_destroy_surrogate(sas_surrogate* s)
{
    if (!s) return SAS_OK;
    cudaStreamSynchronize(s->stream);
    free_batch_buffers(s);
    cudaFree(s->d_p);
    cudaFree(s->d_g);
    cudaFree(s->d_m);
    cudaFree(s->d_v);
    cudaFree(s->d_step);
    cudaFree(s->d_ctr);
    cudaFree(s->d_err);
    cudaFree(s->d_w1);
    cudaFree(s->d_epi);
    for (int l = 0; l < 3; ++l) {
        cudaFree(s->d_w[l]);
        cudaFree(s->d_wt[l]);
    }
    cudaFree(s->d_tab);
    cudaFree(s->d_raw);
    cudaFree(s->d_y);
    if (s->cap) cudaStreamDestroy(s->cap);
    if (s->side) cudaStreamDestroy(s->side);
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    if (s->ev_join) cudaEventDestroy(s->ev_join);
    delete s;
    return SAS_OK;
}

}  // extern "C"
