// Cylinder trace through the learned surrogate: warp-specialised, two
// 128-history tiles ("slots") in flight per SM.
//
// 9 warps per CTA. Warp 8 is the producer: one lane streams the weight
// K blocks (64 wide, 32 KB) through a 3-stage TMA ring and issues the
// tcgen05 MMAs of slot 0 and slot 1 alternately into two TMEM accumulators
// (columns 0..255 and 256..511). Warps 0..7 are the epilogue: warps 0..3
// trace the histories of a slot and write its features; for every layer all
// eight read the slot's accumulator (row m = TMEM lane m, warps 0..3 columns
// 0..127, warps 4..7 columns 128..255), add the bias, apply SiLU and write
// the BF16 activations back as the next layer's A operand, or, after the
// last layer, reduce against w5, weight and tally the histories. While the
// epilogue works on one slot the tensor cores work on the other.
//
// Synchronisation (mbarriers):
//   full[st]   TMA of ring stage st landed                  (producer waits)
//   empty[st]  MMAs reading stage st's block finished        (producer waits)
//   acc[s]     the layer MMAs of slot s finished             (epilogue waits)
//   ready[s]   slot s's A operand written, TMEM read (256)   (producer waits)
//   drain      every MMA issued finished                    (producer, at exit)
// Every wait gives up after WAIT_NS or once another thread has given up
// (a shared abort flag); the loops keep their trip counts so that the
// epilogue's named barrier stays matched, the producer drains its copies and
// MMAs in flight, and the kernel reports the failure in P.err.
//
// Work: the histories are cut into 256-history pairs (two slots); CTA c
// takes pairs c, c + G, c + 2G, ... (G = grid size), and a prefix array
// over the work items maps a pair to its item, so producer and epilogue
// walk the same sequence without exchanging messages.
#pragma once

#include "sas_surrogate.cuh"

namespace sas {
namespace sur {

constexpr int ST_THREADS = 288;
constexpr int RING = 3;                        // weight ring stages (32 KB each)
constexpr uint32_t S2_A = 0;                   // 2 x 64 KB activation slots (K block 0 = features)
constexpr uint32_t S2_W = 131072;              // RING x 32 KB weight ring
constexpr uint32_t S2_DOT = S2_W + RING * 32768u;   // [2][128] f32: second half of the output dot
constexpr uint32_t S2_BAR = S2_DOT + 1024;     // 11 mbarriers, TMEM address, abort flag
constexpr size_t S2_SMEM = (size_t)S2_BAR + 128 + 1024;
constexpr int UNITS_PER_PAIR = 26;             // layer 1: 2 slots x 1 K block; layers 2..4: 2 slots x 4
constexpr int LOADS_PER_PAIR = 16;

// Static schedule of one pair. A unit is the 4 MMAs (K = 64) of one layer,
// slot and weight K block. Slot 1 walks the K blocks of a layer in reverse
// so that it finds three of slot 0's four blocks still in the ring; only
// the fourth (K block 0) is fetched again. 16 loads per pair instead of 26.
// Ring stages play three roles X, Y, Z, ordered by when their last block of
// the previous pair is released (units 23, 24, 25); roles Y and Z swap
// physical stages from one pair to the next. Every load is issued after the
// MMAs of its stage's previous block finished (unit free_after, negative:
// the previous pair) and at least two units before its first use.
enum : uint8_t { U_FIRST = 1, U_LAST = 2, U_RELEASE = 4 };
struct SchedUnit {
    uint8_t l, s, kb, load, flags;   // flags: first / last unit of (l, s), last use of the load
};
struct SchedLoad {
    uint8_t l, kb, role;
    int8_t free_after;
};
static __constant__ SchedUnit kUnits[UNITS_PER_PAIR] = {
    {0, 0, 0, 0, U_FIRST | U_LAST}, {0, 1, 0, 0, U_FIRST | U_LAST | U_RELEASE},
    {1, 0, 0, 1, U_FIRST | U_RELEASE}, {1, 0, 1, 2, 0}, {1, 0, 2, 3, 0}, {1, 0, 3, 4, U_LAST},
    {1, 1, 3, 4, U_FIRST | U_RELEASE}, {1, 1, 2, 3, U_RELEASE}, {1, 1, 1, 2, U_RELEASE},
    {1, 1, 0, 5, U_LAST | U_RELEASE},
    {2, 0, 0, 6, U_FIRST | U_RELEASE}, {2, 0, 1, 7, 0}, {2, 0, 2, 8, 0}, {2, 0, 3, 9, U_LAST},
    {2, 1, 3, 9, U_FIRST | U_RELEASE}, {2, 1, 2, 8, U_RELEASE}, {2, 1, 1, 7, U_RELEASE},
    {2, 1, 0, 10, U_LAST | U_RELEASE},
    {3, 0, 0, 11, U_FIRST | U_RELEASE}, {3, 0, 1, 12, 0}, {3, 0, 2, 13, 0}, {3, 0, 3, 14, U_LAST},
    {3, 1, 3, 14, U_FIRST | U_RELEASE}, {3, 1, 2, 13, U_RELEASE}, {3, 1, 1, 12, U_RELEASE},
    {3, 1, 0, 15, U_LAST | U_RELEASE},
};
static __constant__ SchedLoad kLoads[LOADS_PER_PAIR] = {
    {0, 0, 0, -3}, {1, 0, 1, -2}, {1, 1, 2, -1}, {1, 2, 0, 1}, {1, 3, 1, 2}, {1, 0, 1, 6},
    {2, 0, 0, 7}, {2, 1, 2, 8}, {2, 2, 1, 9}, {2, 3, 0, 10}, {2, 0, 0, 14},
    {3, 0, 1, 15}, {3, 1, 2, 16}, {3, 2, 0, 17}, {3, 3, 1, 18}, {3, 0, 1, 22},
};

__device__ __forceinline__ uint32_t ring_stage(uint32_t pair, uint32_t role)
{
    return role == 0 ? 0u : ((pair & 1u) ? 3u - role : role);
}

// History data a row keeps in the registers of its epilogue thread
// (warps 0..3) from the features to the tally.
struct RowRec {
    float pref, q0, q1, q2, wt;
    int pix_flags;   // (pixel + 1) << 2 | in_box << 1 | valid
};

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

// Bounded wait that also gives up once *abort is set; sets it on timeout.
__device__ __forceinline__ bool wait_ab(uint64_t* bar, uint32_t parity, volatile int* abort)
{
    if (tc::mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = tc::globaltimer();
    for (uint32_t i = 1; i < 0x7FFFFFFFu; ++i) {
        if (tc::mbar_try_wait(bar, parity)) return true;
        if ((i & 63u) == 0u) {
            if (*abort) return false;
            if (tc::globaltimer() - t0 > mlp::WAIT_NS) break;
        }
    }
    *abort = 1;
    return false;
}

struct PairInfo {
    uint64_t first;
    uint32_t exp;
    uint32_t n;      // histories in the pair (1..256)
};

__device__ __forceinline__ PairInfo pair_info(const STParams& P, uint32_t p)
{
    // last item i with pair_prefix[i] <= p
    uint32_t lo = 0, hi = P.n_items;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (P.pair_prefix[mid] <= p) lo = mid;
        else hi = mid;
    }
    const WorkItem w = P.items[lo];
    const uint32_t off = (p - P.pair_prefix[lo]) * 256u;
    PairInfo r;
    r.first = w.first + off;
    r.exp = w.exp;
    r.n = min(256u, w.n - off);
    return r;
}

// Trace the history of row m of slot s and write its features into the
// slot's A operand (warps 0..3).
__device__ __forceinline__ RowRec slot_features(const STParams& P, unsigned char* sm, int s, int m,
                                                const PairInfo& pi)
{
    float f[64];
#pragma unroll
    for (int k = 0; k < 64; ++k) f[k] = 0.f;
    RowRec r;
    r.pref = r.q0 = r.q1 = r.q2 = r.wt = 0.f;
    r.pix_flags = 0;
    const uint32_t j = (uint32_t)s * 128u + (uint32_t)m;
    if (j < pi.n) {
        const History<float> hs = history<float>(P.in, *P.seed, P.philox_base + pi.exp, pi.first + j);
        r.wt = hs.wt;
        int flags = 1 | ((hs.pixel + 1) << 2);
        if (hs.pixel >= 0) {
            const SurExp e = P.sexp[pi.exp];
            const float qp = hs.q[0] * e.nx + hs.q[1] * e.ny + hs.q[2] * e.nz;
            const float q2 = hs.q[0] * hs.q[0] + hs.q[1] * hs.q[1] + hs.q[2] * hs.q[2];
            const float qt = sqrtf(fmaxf(q2 - qp * qp, 0.0f));
            const bool inb = e.in_box && sqrtf(q2) <= P.box.q_max;
            if (inb) features(P.box, fabsf(qp), qt, e.R, e.L, e.so, e.sp, f);
            flags |= inb ? 2 : 0;
            r.pref = hs.pref;
            r.q0 = hs.q[0];
            r.q1 = hs.q[1];
            r.q2 = hs.q[2];
        }
        r.pix_flags = flags;
    }
    unsigned char* a = sm + S2_A + (uint32_t)s * 65536u;
#pragma unroll
    for (int q = 0; q < 8; ++q) mlp::st_row8(a, m, 8 * q, f + 8 * q);
    return r;
}

// After the last layer: weight and tally one row; returns its transmitted weight.
__device__ __forceinline__ float row_finish(const STParams& P, const RowRec& r, const PairInfo& pi, float out)
{
    if (!(r.pix_flags & 1)) return 0.f;
    const int pix = (r.pix_flags >> 2) - 1;
    if (pix >= 0) {
        float ds;
        if (r.pix_flags & 2) {
            ds = P.sexp[pi.exp].scale_p * __expf(out);
        } else {
            const BatchExp& be = P.bexp[pi.exp];
            const float q[3] = {r.q0, r.q1, r.q2};
            ds = dsigma<float, SAS_CYLINDER>(q, be.mc, P.poly + be.poly_off, P.orient + be.orient_off);
            atomicAdd(P.fallbacks, 1ull);
        }
        const float w = r.pref * ds;
        const size_t o = (size_t)pi.exp * P.npix + pix;
        atomicAdd(P.sum_w + o, (double)w);
        atomicAdd(P.sum_w2 + o, (double)w * (double)w);
        atomicAdd(P.count + o, 1ull);
    }
    return r.wt;
}

// Warp-uniform flush of the transmitted weight accumulated for experiment `exp`.
__device__ __forceinline__ void flush_trans(const STParams& P, double& t, uint32_t exp)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if ((threadIdx.x & 31) == 0 && t != 0.0 && exp != 0xFFFFFFFFu) atomicAdd(P.trans + exp, t);
    t = 0.0;
}

__global__ void __launch_bounds__(ST_THREADS, 1) sur_trace_kernel(const STParams P, const __grid_constant__ mlp::Maps maps)
{
    extern __shared__ unsigned char raw_sm[];
    unsigned char* sm = mlp::aligned_base(raw_sm);
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + S2_BAR);   // [RING]
    uint64_t* empty = full + RING;                                // [RING]
    uint64_t* acc = empty + RING;                                 // [2]
    uint64_t* ready = acc + 2;                                    // [2]
    uint64_t* drain = ready + 2;
    uint32_t* taddr = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort = reinterpret_cast<volatile int*>(taddr + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < RING; ++i) {
            tc::mbar_init(full + i, 1);
            tc::mbar_init(empty + i, 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(acc + i, 1);
            tc::mbar_init(ready + i, 256);
        }
        tc::mbar_init(drain, 1);
        *abort = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(taddr, 512);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *taddr;
    const uint32_t my_pairs = blockIdx.x < P.n_pairs ? (P.n_pairs - 1u - blockIdx.x) / gridDim.x + 1u : 0u;

    if (warp == 8) {
        // ---------------------------------------------------------- producer
        if (lane == 0 && my_pairs > 0) {
            const uint32_t total = my_pairs * UNITS_PER_PAIR;
            const uint32_t n_loads = my_pairs * LOADS_PER_PAIR;
            const uint32_t idesc = tc::idesc_bf16(mlp::TILE, mlp::H);
            uint32_t nld[RING] = {0u, 0u, 0u};    // loads issued per stage
            uint8_t ld_stage[32], ld_par[32];     // stage and full-barrier parity of load g (mod 32)
            uint32_t g_next = 0;                   // next load (over all pairs of this CTA)
            uint32_t rd_ph[2] = {0u, 0u};
            uint32_t issued = 0;                   // units whose MMAs were issued
            bool ok = true;
            // issue, in order, every load whose stage was released by unit <= v_done
            auto issue_loads = [&](int64_t v_done) {
                while (ok && g_next < n_loads) {
                    const uint32_t pair = g_next / LOADS_PER_PAIR;
                    const SchedLoad L = kLoads[g_next % LOADS_PER_PAIR];
                    if ((int64_t)pair * UNITS_PER_PAIR + L.free_after > v_done) break;
                    const uint32_t k = ring_stage(pair, L.role);
                    if (nld[k] > 0) {
                        ok = wait_ab(empty + k, (nld[k] - 1u) & 1u, abort);
                        if (!ok) break;
                    }
                    const CUtensorMap* map = L.l == 0 ? &maps.w1 : &maps.w[L.l - 1];
                    tc::mbar_arrive_expect_tx(full + k, 32768u);
                    tc::tma_load_2d(sm + S2_W + k * 32768u, map, L.kb * 64, 0, full + k);
                    ld_stage[g_next & 31u] = (uint8_t)k;
                    ld_par[g_next & 31u] = (uint8_t)(nld[k] & 1u);
                    ++nld[k];
                    ++g_next;
                }
            };
            issue_loads(-1);
            for (uint32_t v = 0; v < total && ok; ++v) {
                const uint32_t pair = v / UNITS_PER_PAIR;
                const SchedUnit U = kUnits[v % UNITS_PER_PAIR];
                if (U.flags & U_FIRST) {
                    ok = wait_ab(ready + U.s, rd_ph[U.s], abort);
                    rd_ph[U.s] ^= 1u;
                    if (!ok) break;
                }
                const uint32_t g = pair * LOADS_PER_PAIR + U.load;   // issued: its stage was released >= 2 units ago
                const uint32_t k = ld_stage[g & 31u];
                ok = wait_ab(full + k, ld_par[g & 31u], abort);
                if (!ok) break;
                tc::fence_after_sync();
                const uint32_t a0 = tc::smem_u32(sm + S2_A + (uint32_t)U.s * 65536u + (uint32_t)U.kb * 16384u);
                const uint32_t b0 = tc::smem_u32(sm + S2_W + k * 32768u);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    tc::mma_bf16(tmem + 256u * (uint32_t)U.s, tc::desc_sw128(a0 + kk * 32),
                                 tc::desc_sw128(b0 + kk * 32), idesc, ((U.flags & U_FIRST) && kk == 0) ? 0u : 1u);
                if (U.flags & U_RELEASE) tc::mma_commit(empty + k);
                if (U.flags & U_LAST) tc::mma_commit(acc + U.s);
                issued = v + 1;
                issue_loads((int64_t)v - 1);
            }
            // drain: the last load of each stage, then every MMA issued
            bool drained = true;
            for (int k = 0; k < RING; ++k)
                if (nld[k] > 0) drained = tc::mbar_wait(full + k, (nld[k] - 1u) & 1u, mlp::WAIT_NS) && drained;
            if (issued > 0) {
                tc::mma_commit(drain);
                drained = tc::mbar_wait(drain, 0u, mlp::WAIT_NS) && drained;
            }
            if (!ok || !drained) {
                *abort = 1;
                atomicExch(P.err, 8);
            }
        }
    } else {
        // ---------------------------------------------------------- epilogue
        const int h = warp >> 2;
        const int m = 32 * (warp & 3) + lane;
        const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
        const float* bias = P.params + mlp::OFF_B1;
        const float* w5 = P.params + mlp::OFF_W5;
        float* dot1 = reinterpret_cast<float*>(sm + S2_DOT);
        const float b5 = __ldg(P.params + mlp::OFF_B5);
        uint32_t acc_ph[2] = {0u, 0u};
        bool ok = true;
        double t_acc = 0.0;
        uint32_t t_exp = 0xFFFFFFFFu;
        RowRec rec[2];
        PairInfo cur = my_pairs > 0 ? pair_info(P, blockIdx.x) : PairInfo{0, 0, 0};
        if (my_pairs > 0) {
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                if (h == 0) rec[s] = slot_features(P, sm, s, m, cur);
                tc::fence_proxy_async_smem();
                mbar_arrive(ready + s);
            }
        }
        for (uint32_t it = 0; it < my_pairs; ++it) {
            const bool more = it + 1 < my_pairs;
            const PairInfo nxt = more ? pair_info(P, blockIdx.x + (it + 1) * gridDim.x) : cur;
            for (int l = 0; l < 4; ++l) {
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    ok = wait_ab(acc + s, acc_ph[s], abort) && ok;
                    acc_ph[s] ^= 1u;
                    tc::fence_after_sync();
                    const uint32_t tbase = tmem + lane_base + 256u * (uint32_t)s;
                    unsigned char* a = sm + S2_A + (uint32_t)s * 65536u;
                    float dot = 0.f;
#pragma unroll 1
                    for (int ch = 0; ch < 4; ++ch) {
                        const int col0 = 128 * h + 32 * ch;
                        float v[32];
                        tc::tmem_ld32(tbase + col0, v);
                        const float4* b4 = reinterpret_cast<const float4*>(bias + 256 * l + col0);
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const float4 bb = __ldg(b4 + q);
                            v[4 * q + 0] = mlp::silu(v[4 * q + 0] + bb.x);
                            v[4 * q + 1] = mlp::silu(v[4 * q + 1] + bb.y);
                            v[4 * q + 2] = mlp::silu(v[4 * q + 2] + bb.z);
                            v[4 * q + 3] = mlp::silu(v[4 * q + 3] + bb.w);
                        }
                        if (l < 3) {
#pragma unroll
                            for (int q = 0; q < 4; ++q) mlp::st_row8(a, m, col0 + 8 * q, v + 8 * q);
                        } else {
                            const float4* w4 = reinterpret_cast<const float4*>(w5 + col0);
#pragma unroll
                            for (int q = 0; q < 8; ++q) {
                                const float4 ww = __ldg(w4 + q);
                                dot = fmaf(__bfloat162float(__float2bfloat16_rn(v[4 * q + 0])), ww.x, dot);
                                dot = fmaf(__bfloat162float(__float2bfloat16_rn(v[4 * q + 1])), ww.y, dot);
                                dot = fmaf(__bfloat162float(__float2bfloat16_rn(v[4 * q + 2])), ww.z, dot);
                                dot = fmaf(__bfloat162float(__float2bfloat16_rn(v[4 * q + 3])), ww.w, dot);
                            }
                        }
                    }
                    tc::fence_before_sync();
                    if (l < 3) {
                        tc::fence_proxy_async_smem();
                        mbar_arrive(ready + s);
                    } else {
                        if (h == 1) dot1[s * 128 + m] = dot;
                        epi_sync();
                        if (h == 0) {
                            if (cur.exp != t_exp) {
                                flush_trans(P, t_acc, t_exp);
                                t_exp = cur.exp;
                            }
                            t_acc += (double)row_finish(P, rec[s], cur, b5 + dot + dot1[s * 128 + m]);
                            if (more) rec[s] = slot_features(P, sm, s, m, nxt);
                        }
                        if (more) {
                            tc::fence_proxy_async_smem();
                            mbar_arrive(ready + s);
                        }
                    }
                }
            }
            cur = nxt;
        }
        if (h == 0) flush_trans(P, t_acc, t_exp);
        if (!ok) atomicExch(P.err, 9);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

}  // namespace sur
}  // namespace sas
