// Learned surrogate of the orientation- and polydispersity-averaged
// cylinder form factor: an MLP 5 (padded to 64) -> 4 x 256 (SiLU) -> 1 that
// outputs log P, with BF16 weights and FP32 accumulation on the tcgen05
// tensor cores.
//
// One CTA of 256 threads (8 warps) works on tiles of 128 rows (neutrons or
// training samples). The accumulator of a layer is a 128 x 256 FP32 block
// of tensor memory: TMEM lane m holds row m. Warp w reads lanes
// 32 (w % 4) .. 32 (w % 4) + 31 and columns 128 (w / 4) .. + 127, so every
// thread owns one row and half of its columns in the epilogues. Layer by
// layer: one thread loads the layer's weights into shared memory with TMA
// and issues the MMAs (A = activations of the tile in shared memory, B =
// weights, both K-major, 128-byte swizzle); the epilogue adds the bias,
// applies SiLU and writes the BF16 activations back as the next A operand.
//
// SiLU(z) = z s(z) with s(z) = 1/2 + tanh(z/2)/2 (hardware tanh
// approximation); training and inference use the same definition, its
// derivative is s (1 + z (1 - s)).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include "sas_tc.cuh"

namespace sas {
namespace mlp {

constexpr int H = 256;          // hidden width
constexpr int KIN = 64;         // padded input width (one 64-element K block)
constexpr int NF = 5;           // features used
constexpr int TILE = 128;       // rows per tile (MMA M)
constexpr int THREADS = 512;    // tile kernels: 16 warps, a quarter of the columns each
constexpr int NGROUP = THREADS / TILE;   // column groups (warps w, w + 4, ... share TMEM lanes)
constexpr int GCOLS = H / NGROUP;        // accumulator columns per thread
constexpr int NPARAM_W1 = H * KIN;
constexpr int NPARAM_W = H * H;
// flat FP32 parameter layout: W1 [256][64] | W2 | W3 | W4 [256][256] |
// b1 | b2 | b3 | b4 [256] | w5 [256] | b5
constexpr int OFF_W1 = 0;
constexpr int OFF_W2 = OFF_W1 + NPARAM_W1;
constexpr int OFF_W3 = OFF_W2 + NPARAM_W;
constexpr int OFF_W4 = OFF_W3 + NPARAM_W;
constexpr int OFF_B1 = OFF_W4 + NPARAM_W;
constexpr int OFF_W5 = OFF_B1 + 4 * H;
constexpr int OFF_B5 = OFF_W5 + H;
constexpr int NPARAM = OFF_B5 + 1;

// shared memory layout of the fused tile kernels (offsets from a
// 1024-byte aligned base)
constexpr uint32_t SM_A0 = 0;              // 128 x 64 bf16 input tile (16 KB)
constexpr uint32_t SM_A = 16384;           // 128 x 256 bf16 activations (64 KB)
constexpr uint32_t SM_B = 81920;           // 256 x 256 bf16 weights (128 KB)
constexpr uint32_t SM_BIAS = 212992;       // 4 x 256 f32 biases
constexpr uint32_t SM_W5 = SM_BIAS + 4096; // 256 f32
constexpr uint32_t SM_ROW = SM_W5 + 1024;  // NGROUP x 128 f32 per-row scratch
constexpr uint32_t SM_BAR = SM_ROW + 4 * TILE * NGROUP; // mbarriers + TMEM address
constexpr uint32_t SM_TOTAL = SM_BAR + 64;
constexpr size_t SMEM_BYTES = SM_TOTAL + 1024;   // + alignment slack

constexpr uint64_t WAIT_NS = 2000000000ull;      // 2 s limit on any wait

struct Maps {
    CUtensorMap w1;      // [256][64] bf16
    CUtensorMap w[3];    // W2..W4 [256 out][256 in] bf16
    CUtensorMap wt[3];   // W2^T..W4^T [256 in][256 out] bf16
};

__device__ __forceinline__ float tanh_approx(float x)
{
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(x));
    return t;
}
__device__ __forceinline__ float sig_(float z) { return fmaf(0.5f, tanh_approx(0.5f * z), 0.5f); }

// tanh of two values through one half-precision MUFU operation (inputs
// rounded to f16; about 2^-11 relative error, like tanh.approx.f32)
__device__ __forceinline__ float2 tanh2_f16(float2 x)
{
    const __half2 h = __floats2half2_rn(x.x, x.y);
    uint32_t r;
    asm("tanh.approx.f16x2 %0, %1;" : "=r"(r) : "r"(*reinterpret_cast<const uint32_t*>(&h)));
    return __half22float2(*reinterpret_cast<const __half2*>(&r));
}
__device__ __forceinline__ float silu(float z) { return z * sig_(z); }
__device__ __forceinline__ float dsilu(float z)
{
    const float s = sig_(z);
    return s * fmaf(z, 1.0f - s, 1.0f);
}

struct Ctx {
    unsigned char* sm;
    uint32_t tmem;
    uint64_t* bar_tma;
    uint64_t* bar_mma;
    uint32_t ph_tma, ph_mma;
    int* err;
};

__device__ __forceinline__ unsigned char* aligned_base(unsigned char* raw)
{
    const uint32_t a = tc::smem_u32(raw);
    return raw + (((a + 1023u) & ~1023u) - a);
}

// CTA set-up: barriers, TMEM (256 columns, allocated by warp 0).
__device__ __forceinline__ void ctx_init(Ctx& c, unsigned char* raw, int* err)
{
    c.sm = aligned_base(raw);
    c.bar_tma = reinterpret_cast<uint64_t*>(c.sm + SM_BAR);
    c.bar_mma = c.bar_tma + 1;
    uint32_t* taddr = reinterpret_cast<uint32_t*>(c.sm + SM_BAR + 16);
    c.err = err;
    c.ph_tma = c.ph_mma = 0;
    if (threadIdx.x == 0) {
        tc::mbar_init(c.bar_tma, 1);
        tc::mbar_init(c.bar_mma, 1);
        tc::fence_mbar_init();
    }
    if (threadIdx.x < 32) tc::tmem_alloc(taddr, 256);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    c.tmem = *taddr;
}

__device__ __forceinline__ void ctx_finish(Ctx& c)
{
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x < 32) tc::tmem_dealloc(c.tmem, 256);
}

// one thread: TMA nkb 64-wide K blocks of a [256 x 64*nkb] weight map into B
__device__ __forceinline__ void load_weights(Ctx& c, const CUtensorMap* map, int nkb)
{
    if (threadIdx.x == 0) {
        tc::mbar_arrive_expect_tx(c.bar_tma, (uint32_t)nkb * 32768u);
        for (int kb = 0; kb < nkb; ++kb) tc::tma_load_2d(c.sm + SM_B + kb * 32768, map, kb * 64, 0, c.bar_tma);
    }
}

// one thread: wait for the weights, issue the layer's MMAs, commit.
__device__ __forceinline__ void issue_layer(Ctx& c, uint32_t a_off, int nkb)
{
    if (threadIdx.x == 0) {
        if (!tc::mbar_wait(c.bar_tma, c.ph_tma, WAIT_NS)) atomicExch(c.err, 1);
        tc::fence_after_sync();
        const uint32_t idesc = tc::idesc_bf16(TILE, H);
        for (int kb = 0; kb < nkb; ++kb)
            for (int k = 0; k < 4; ++k) {
                const uint64_t ad = tc::desc_sw128(tc::smem_u32(c.sm + a_off + kb * 16384) + k * 32);
                const uint64_t bd = tc::desc_sw128(tc::smem_u32(c.sm + SM_B + kb * 32768) + k * 32);
                tc::mma_bf16(c.tmem, ad, bd, idesc, (kb | k) ? 1u : 0u);
            }
        tc::mma_commit(c.bar_mma);
    }
    c.ph_tma ^= 1u;
}

__device__ __forceinline__ void wait_layer(Ctx& c)
{
    if (!tc::mbar_wait(c.bar_mma, c.ph_mma, WAIT_NS)) atomicExch(c.err, 2);
    c.ph_mma ^= 1u;
    tc::fence_after_sync();
}

// make the generic-proxy shared-memory writes of the epilogue visible to
// the tensor cores and order them before the next MMA
__device__ __forceinline__ void publish_smem()
{
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
}

__device__ __forceinline__ int row_of_thread() { return 32 * ((threadIdx.x >> 5) & 3) + (threadIdx.x & 31); }
__device__ __forceinline__ int group_of_thread() { return (threadIdx.x >> 5) >> 2; }

__device__ __forceinline__ uint32_t tmem_addr(const Ctx& c, int col)
{
    return c.tmem + ((uint32_t)(32 * ((threadIdx.x >> 5) & 3)) << 16) + (uint32_t)col;
}

// write 8 bf16 values (columns col..col+7, col % 8 == 0) of row m into a
// swizzled 64-wide-K-block operand buffer
__device__ __forceinline__ void st_row8(unsigned char* buf, int m, int col, const float* v)
{
    const int kb = col >> 6, c = (col & 63) >> 3;
    uint4 p;
    p.x = tc::pack_bf16(v[0], v[1]);
    p.y = tc::pack_bf16(v[2], v[3]);
    p.z = tc::pack_bf16(v[4], v[5]);
    p.w = tc::pack_bf16(v[6], v[7]);
    *reinterpret_cast<uint4*>(buf + kb * 16384 + tc::sw128_chunk(m, c)) = p;
}

// Hidden-layer epilogue: z = acc + b, a = SiLU(z) -> A operand; when zt/ht
// are given (training) also z and a into [256][ld] transposed global arrays
// at column `col_g` (this row's sample index). With dot != nullptr the
// activations are instead reduced against w5 (last hidden layer).
__device__ __forceinline__ float epi_hidden(Ctx& c, const float* bias, __nv_bfloat16* zt, __nv_bfloat16* ht,
                                            size_t ld, size_t col_g, bool row_valid, const float* w5)
{
    const int m = row_of_thread(), h = group_of_thread();
    float dot = 0.f;
    for (int ch = 0; ch < GCOLS / 32; ++ch) {
        const int col0 = GCOLS * h + 32 * ch;
        float v[32];
        tc::tmem_ld32(tmem_addr(c, col0), v);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const float z = v[j] + bias[col0 + j];
            const float a = silu(z);
            if (zt && row_valid) {
                zt[(size_t)(col0 + j) * ld + col_g] = __float2bfloat16_rn(z);
                ht[(size_t)(col0 + j) * ld + col_g] = __float2bfloat16_rn(a);
            }
            if (w5) dot = fmaf(__bfloat162float(__float2bfloat16_rn(a)), w5[col0 + j], dot);
            v[j] = a;
        }
        if (!w5) {
#pragma unroll
            for (int q = 0; q < 4; ++q) st_row8(c.sm + SM_A, m, col0 + 8 * q, v + 8 * q);
        }
    }
    return dot;
}

// Forward pass of one tile. The input tile (A0) must already hold the
// features; layer-1 weights must have been requested with load_weights(w1).
// Returns this thread's half of the output dot product (rows: see
// row_of_thread). On return the layer-1 weights are being loaded again for
// the next tile.
template <bool TRAIN>
__device__ __forceinline__ float forward_tile(Ctx& c, const Maps& maps, __nv_bfloat16* const* zt,
                                              __nv_bfloat16* const* ht, size_t ld, size_t col_g, bool row_valid)
{
    const float* bias = reinterpret_cast<const float*>(c.sm + SM_BIAS);
    const float* w5 = reinterpret_cast<const float*>(c.sm + SM_W5);
    publish_smem();
    issue_layer(c, SM_A0, 1);                       // layer 1: K = 64
    float dot = 0.f;
    for (int l = 0; l < 4; ++l) {
        wait_layer(c);
        // the weights of the next layer (or layer 1 of the next tile) can now
        // overwrite B while the epilogue runs
        if (l < 3) load_weights(c, &maps.w[l], 4);
        else load_weights(c, &maps.w1, 1);
        const bool last = (l == 3);
        dot = epi_hidden(c, bias + 256 * l, TRAIN ? zt[l] : nullptr, TRAIN ? ht[l] : nullptr, ld, col_g,
                         row_valid, last ? w5 : nullptr);
        if (!last) {
            publish_smem();
            issue_layer(c, SM_A, 4);
        }
    }
    tc::fence_before_sync();
    return dot;
}

// Stage biases and w5 of the FP32 master parameters into shared memory.
__device__ __forceinline__ void stage_params(Ctx& c, const float* P)
{
    float* b = reinterpret_cast<float*>(c.sm + SM_BIAS);
    for (int i = threadIdx.x; i < 4 * H; i += blockDim.x) b[i] = P[OFF_B1 + i];
    float* w5 = reinterpret_cast<float*>(c.sm + SM_W5);
    for (int i = threadIdx.x; i < H; i += blockDim.x) w5[i] = P[OFF_W5 + i];
}

}  // namespace mlp
}  // namespace sas
