// Cylinder trace through the learned surrogate: warp-specialised, two
// 128-history tiles ("slots") in flight per SM. The same pipeline runs the
// training step's forward pass (MODE_TRAIN: rows of the data set instead of
// traced histories; Z^T, H^T and X^T stored for the backward pass) and its
// backward pass through the hidden layers (MODE_BWD: the first step forms
// dZ4 from d loss / d out, a placeholder first-layer MMA keeps the static
// schedule, then dH = dZ W^T with W4^T, W3^T, W2^T and dZ = dH SiLU'(z),
// dZ^T stored for the weight gradients).
//
// 22 warps per CTA, in four roles:
// - MMA warp (0): one lane issues the tcgen05 MMAs of slot 0 and slot 1
//   alternately into two TMEM accumulators (columns 0..255, 256..511);
// - TMA warp (1): one lane streams the weight K blocks (64 wide, 32 KB)
//   through a 3-stage ring in a static order;
// - SiLU warps (4..19): each reads a quarter of a slot's accumulator (row m
//   = TMEM lane m; lanes 32 (w % 4).., columns 64 ((w - 4) / 4)..), adds the
//   bias, applies SiLU and writes the BF16 activations back as the next
//   layer's A operand, or after the last layer reduces against w5; sixteen
//   warps keep the MUFU (tanh) pipe, their bound, busy;
// - history warps (2, 3, 20, 21): thread m traces row m of both slots one
//   pair ahead, writes the features and tallies the weighted histories.
// While the SiLU warps work on one slot the tensor cores work on the other.
//
// Synchronisation (mbarriers):
//   full[st]   TMA of ring stage st landed                     (MMA warp waits)
//   empty[st]  MMAs reading stage st's block finished          (TMA warp waits)
//   acc[s]     the layer MMAs of slot s finished               (SiLU warps wait)
//   ready[s]   activations of slot s written, TMEM read (16)   (MMA warp waits)
//   dots[s]    output partials of slot s written, TMEM read (16) (history warps)
//   feat[s]    features of slot s's next pair written (4)      (MMA warp waits)
//   drain      every MMA issued finished                       (MMA warp, at exit)
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

// Warp roles. The single-lane MMA and TMA issuers take the oldest warps 0
// and 1 (measured faster than placing them last); the SiLU warps 4..19 keep
// warp % 4 equal to their TMEM lane group; history warps 2, 3, 20, 21.
constexpr int MMA_WARP = 0;
constexpr int TMA_WARP = 1;
constexpr int EPI_WARP0 = 4;                   // SiLU warps 4..19
constexpr int EPI_WARPS = 16;
constexpr int HIST_WARPS = 4;
constexpr int ST_THREADS = 32 * 22;

__device__ __forceinline__ int hist_index(int warp)   // 0..3 for history warps, else -1
{
    return warp == 2 ? 0 : warp == 3 ? 1 : (warp == 20 || warp == 21) ? warp - 18 : -1;
}
constexpr int RING = 3;                        // weight ring stages (32 KB each)
constexpr uint32_t S2_A = 0;                   // 2 x 64 KB activation slots (K block 0 = features)
constexpr uint32_t S2_W = 131072;              // RING x 32 KB weight ring
constexpr uint32_t S2_BAR = S2_W + RING * 32768u;   // 15 mbarriers, TMEM address, abort flag
constexpr uint32_t S2_DOUT = S2_BAR + 256;     // MODE_BWD: 2 x 128 floats of d loss / d out
constexpr size_t S2_SMEM = (size_t)S2_DOUT + 1024 + 1024;
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
    uint8_t l, kb, role, ord;   // ord: loads of the same role before this one in the pair
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
    {0, 0, 0, 0, -3}, {1, 0, 1, 0, -2}, {1, 1, 2, 0, -1}, {1, 2, 0, 1, 1}, {1, 3, 1, 1, 2}, {1, 0, 1, 2, 6},
    {2, 0, 0, 2, 7}, {2, 1, 2, 1, 8}, {2, 2, 1, 3, 9}, {2, 3, 0, 3, 10}, {2, 0, 0, 4, 14},
    {3, 0, 1, 4, 15}, {3, 1, 2, 2, 16}, {3, 2, 0, 5, 17}, {3, 3, 1, 5, 18}, {3, 0, 1, 6, 22},
};

__device__ __forceinline__ uint32_t ring_stage(uint32_t pair, uint32_t role)
{
    return role == 0 ? 0u : ((pair & 1u) ? 3u - role : role);
}

// Phase parity of a load's full barrier (and of its release on empty). Per
// pair role X takes 6 loads (even) and stays on stage 0; roles Y and Z take
// 7 and 3 loads and swap stages 1 and 2 every pair, so each of those stages
// has seen an odd number of loads before every odd pair.
__device__ __forceinline__ uint32_t ring_parity(uint32_t pair, const SchedLoad& L)
{
    return ((L.role == 0 ? 0u : (pair & 1u)) + L.ord) & 1u;
}

// History data a history-warp thread keeps in registers from the trace of a
// history to its tally.
struct RowRec {
    float pref, q0, q1, q2, wt;
    int pix_flags;   // (pixel + 1) << 2 | in_box << 1 | valid
    float qp, qt;    // |Q . axis| and |Q x axis|: the features are made from these
};

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

// Trace the history of row m of slot s of a pair.
__device__ __forceinline__ RowRec trace_row(const STParams& P, int s, int m, const PairInfo& pi)
{
    RowRec r;
    r.pref = r.q0 = r.q1 = r.q2 = r.wt = r.qp = r.qt = 0.f;
    r.pix_flags = 0;
    const uint32_t j = (uint32_t)s * 128u + (uint32_t)m;
    if (j < pi.n) {
        // the surrogate covers models without self-attenuation only
        const AttTable<float> no_att{};
        const History<float> hs = history<float>(P.in, no_att, *P.seed, P.philox_base + pi.exp, pi.first + j);
        r.wt = hs.wt;
        int flags = 1 | ((hs.pixel + 1) << 2);
        if (hs.pixel >= 0) {
            const SurExp e = P.sexp[pi.exp];
            const float qp = hs.q[0] * e.nx + hs.q[1] * e.ny + hs.q[2] * e.nz;
            const float q2 = hs.q[0] * hs.q[0] + hs.q[1] * hs.q[1] + hs.q[2] * hs.q[2];
            r.qp = fabsf(qp);
            r.qt = sqrtf(fmaxf(q2 - qp * qp, 0.0f));
            flags |= (e.in_box && sqrtf(q2) <= P.box.q_max) ? 2 : 0;
            r.pref = hs.pref;
            r.q0 = hs.q[0];
            r.q1 = hs.q[1];
            r.q2 = hs.q[2];
        }
        r.pix_flags = flags;
    }
    return r;
}

// Features of a traced row into K block 0 of its slot's A operand.
__device__ __forceinline__ void put_features(const STParams& P, unsigned char* sm, int s, int m, const RowRec& r,
                                             const PairInfo& pi)
{
    const SurExp e = P.sexp[pi.exp];
    write_features(P.box, (r.pix_flags & 2) != 0, r.qp, r.qt, e.R, e.L, e.so, e.sp,
                   sm + S2_A + (uint32_t)s * 65536u, m);
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
            ds = P.box.kind == SAS_ELLIPSOID
                     ? dsigma<float, SAS_ELLIPSOID>(q, be.mc, P.poly + be.poly_off, P.orient + be.orient_off)
                     : dsigma<float, SAS_CYLINDER>(q, be.mc, P.poly + be.poly_off, P.orient + be.orient_off);
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

// ------------------------------------------------------ training forward
// MODE_TRAIN: the history warps load the minibatch's data set rows instead
// of tracing histories (R, L, sigma_orient, sigma_poly travel in the
// record's pref, q0, q1, q2; pix_flags holds the row + 1), write their
// features into the slot and X^T into global memory, and store the output.
enum { MODE_TRACE = 0, MODE_TRAIN = 1, MODE_BWD = 2 };

__device__ __forceinline__ RowRec train_row(const STParams& P, uint32_t pair, int s, int m)
{
    RowRec r;
    const uint32_t i = pair * 256u + (uint32_t)s * 128u + (uint32_t)m;
    const uint64_t row = ((uint64_t)(*P.step) * P.batch + i) % P.n_data;
    const Raw x = P.raw[row];
    r.qp = x.qpar;
    r.qt = x.qperp;
    r.pref = x.R;
    r.q0 = x.L;
    r.q1 = x.so;
    r.q2 = x.sp;
    r.wt = 0.f;
    r.pix_flags = (int)(((i + 1u) << 2) | 3u);
    return r;
}

__device__ __forceinline__ void train_features(const STParams& P, unsigned char* sm, int s, int m, const RowRec& r)
{
    unsigned char* kb = sm + S2_A + (uint32_t)s * 65536u;
    write_features(P.box, true, r.qp, r.qt, r.pref, r.q0, r.q1, r.q2, kb, m);
    // X^T for the layer-1 weight gradient: the row just written, read back
    const size_t i = (size_t)((r.pix_flags >> 2) - 1);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const uint4 v = *reinterpret_cast<const uint4*>(kb + tc::sw128_chunk(m, c));
        const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            __stcs(reinterpret_cast<unsigned short*>(P.xt + (size_t)(8 * c + 2 * j) * P.batch + i),
                   (unsigned short)(w4[j] & 0xFFFFu));
            __stcs(reinterpret_cast<unsigned short*>(P.xt + (size_t)(8 * c + 2 * j + 1) * P.batch + i),
                   (unsigned short)(w4[j] >> 16));
        }
    }
}

// Four columns c .. c + 3 of one row into a transposed BF16 array [col][ld]
// (bf16x2 words v01 = columns c, c + 1 and v23 = c + 2, c + 3 of this row).
// Lanes 2k and 2k + 1 hold adjacent rows: they swap half their words, so
// that the even lane stores columns c, c + 1 and the odd lane c + 2, c + 3,
// each as 32-bit words holding both rows (half the store instructions of
// 2-byte stores). Called by all 32 lanes of the warp.
__device__ __forceinline__ void store_pair_t(__nv_bfloat16* dst, uint32_t ld, int c, uint32_t row, uint32_t v01,
                                             uint32_t v23, int lane)
{
    const bool odd = lane & 1;
    const uint32_t r = __shfl_xor_sync(0xffffffffu, odd ? v01 : v23, 1);
    const uint32_t lo = odd ? r : v01, hi = odd ? v23 : r;   // words of the even row, then the odd row
    const uint32_t w0 = __byte_perm(lo, hi, 0x5410), w1 = __byte_perm(lo, hi, 0x7632);
    uint32_t* p = reinterpret_cast<uint32_t*>(dst + (size_t)(c + (odd ? 2 : 0)) * ld + (row & ~1u));
    // streaming stores (evict first): the activations pass through L2 once,
    // and must not push the weights the TMA ring reads out of it
    __stcs(reinterpret_cast<unsigned int*>(p), w0);
    __stcs(reinterpret_cast<unsigned int*>(p + (ld >> 1)), w1);
}

// MODE_BWD: the history warps form d loss / d out = scale (pred - y) of each
// row (kept in the record's wt) for the SiLU warps' first step.
__device__ __forceinline__ RowRec bwd_row(const STParams& P, uint32_t pair, int s, int m)
{
    RowRec r = {};
    const uint32_t i = pair * 256u + (uint32_t)s * 128u + (uint32_t)m;
    const uint64_t row = ((uint64_t)(*P.step) * P.batch + i) % P.n_data;
    r.wt = P.scale * (P.pred[i] - P.y[row]);
    r.pix_flags = (int)(((i + 1u) << 2) | 3u);
    return r;
}

// Warp-uniform flush of the transmitted weight accumulated for experiment `exp`.
__device__ __forceinline__ void flush_trans(const STParams& P, double& t, uint32_t exp)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if ((threadIdx.x & 31) == 0 && t != 0.0 && exp != 0xFFFFFFFFu) atomicAdd(P.trans + exp, t);
    t = 0.0;
}

template <int MODE>
__global__ void __launch_bounds__(ST_THREADS, 1) sur_trace_kernel(const STParams P, const __grid_constant__ mlp::Maps maps)
{
    extern __shared__ unsigned char raw_sm[];
    unsigned char* sm = mlp::aligned_base(raw_sm);
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + S2_BAR);   // [RING] weight block landed
    uint64_t* empty = full + RING;                                // [RING] weight block released
    uint64_t* acc = empty + RING;                                 // [2] layer MMAs done
    uint64_t* ready = acc + 2;                                    // [2] activations written (16 SiLU warps)
    uint64_t* feat = ready + 2;                                   // [2] features written (4 history warps)
    uint64_t* dots = feat + 2;                                    // [2] output partials written (16 SiLU warps)
    uint64_t* drain = dots + 2;
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
            tc::mbar_init(ready + i, EPI_WARPS);
            tc::mbar_init(feat + i, HIST_WARPS);
            tc::mbar_init(dots + i, EPI_WARPS);
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

    if (warp == TMA_WARP) {
        // ------------------------------------------------------------ loads
        // The static load sequence, each load as soon as its ring stage's
        // previous block is released.
        if (lane == 0 && my_pairs > 0) {
            const uint32_t n_loads = my_pairs * LOADS_PER_PAIR;
            uint32_t last0 = 0, last1 = 0, last2 = 0;   // latest load + 1 per stage
            bool ok = true;
            for (uint32_t g = 0; g < n_loads && ok; ++g) {
                const uint32_t pair = g / LOADS_PER_PAIR;
                const SchedLoad L = kLoads[g % LOADS_PER_PAIR];
                const uint32_t k = ring_stage(pair, L.role);
                if (pair > 0 || L.ord > 0) ok = wait_ab(empty + k, ring_parity(pair, L) ^ 1u, abort);
                if (!ok) break;
                // MODE_BWD walks the layers backward: W4^T, W3^T, W2^T after the
                // placeholder first layer (its MMA result is not read)
                const CUtensorMap* map = L.l == 0 ? &maps.w1
                                                  : (MODE == MODE_BWD ? &maps.wt[3 - L.l] : &maps.w[L.l - 1]);
                tc::mbar_arrive_expect_tx(full + k, 32768u);
                tc::tma_load_2d(sm + S2_W + k * 32768u, map, L.kb * 64, 0, full + k);
                if (k == 0) last0 = g + 1;
                else if (k == 1) last1 = g + 1;
                else last2 = g + 1;
            }
            // the latest load of each stage may still be in flight
            bool drained = true;
#pragma unroll
            for (int k = 0; k < RING; ++k) {
                const uint32_t g1 = k == 0 ? last0 : (k == 1 ? last1 : last2);
                if (g1 == 0) continue;
                const uint32_t pr = (g1 - 1u) / LOADS_PER_PAIR;
                const SchedLoad L = kLoads[(g1 - 1u) % LOADS_PER_PAIR];
                drained = tc::mbar_wait(full + k, ring_parity(pr, L), mlp::WAIT_NS) && drained;
            }
            if (!ok || !drained) {
                *abort = 1;
                atomicExch(P.err, 8);
            }
        }
    } else if (warp == MMA_WARP) {
        // ------------------------------------------------------------- MMAs
        if (lane == 0 && my_pairs > 0) {
            const uint32_t idesc = tc::idesc_bf16(mlp::TILE, mlp::H);
            // operand descriptors, computed once: advancing K by 16 elements
            // (32 bytes) adds 2 to the start-address field
            const uint64_t dA = tc::desc_sw128(tc::smem_u32(sm + S2_A));
            const uint64_t dW0 = tc::desc_sw128(tc::smem_u32(sm + S2_W));
            const uint64_t dW1 = dW0 + (32768u >> 4), dW2 = dW0 + (65536u >> 4);
            uint32_t rd0 = 0u, rd1 = 0u, ft0 = 0u, ft1 = 0u;   // phases of ready[] and feat[]
            bool ok = true, issued = false;
            for (uint32_t pair = 0; pair < my_pairs && ok; ++pair) {
                const uint32_t pb = pair & 1u;
                const uint64_t dY = pb ? dW2 : dW1, dZ = pb ? dW1 : dW2;   // stages of roles Y, Z
#pragma unroll
                for (int u = 0; u < UNITS_PER_PAIR; ++u) {
                    if (!ok) break;
                    const SchedUnit U = kUnits[u];
                    if (U.flags & U_FIRST) {
                        if (U.l == 0) {
                            ok = wait_ab(feat + U.s, U.s ? ft1 : ft0, abort);
                            if (U.s) ft1 ^= 1u;
                            else ft0 ^= 1u;
                        } else {
                            ok = wait_ab(ready + U.s, U.s ? rd1 : rd0, abort);
                            if (U.s) rd1 ^= 1u;
                            else rd0 ^= 1u;
                        }
                        if (!ok) break;
                    }
                    const SchedLoad L = kLoads[U.load];
                    const uint32_t k = ring_stage(pair, L.role);
                    ok = wait_ab(full + k, ring_parity(pair, L), abort);
                    if (!ok) break;
                    tc::fence_after_sync();
                    const uint64_t da = dA + (((uint32_t)U.s * 65536u + (uint32_t)U.kb * 16384u) >> 4);
                    const uint64_t db = L.role == 0 ? dW0 : (L.role == 1 ? dY : dZ);
                    const uint32_t dtm = tmem + 256u * (uint32_t)U.s;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        tc::mma_bf16(dtm, da + 2 * kk, db + 2 * kk, idesc, ((U.flags & U_FIRST) && kk == 0) ? 0u : 1u);
                    issued = true;
                    if (U.flags & U_RELEASE) tc::mma_commit(empty + k);
                    if (U.flags & U_LAST) tc::mma_commit(acc + U.s);
                }
            }
            bool drained = true;
            if (issued) {
                tc::mma_commit(drain);
                drained = tc::mbar_wait(drain, 0u, mlp::WAIT_NS);
            }
            if (!ok || !drained) {
                *abort = 1;
                atomicExch(P.err, 8);
            }
        }
    } else if (hist_index(warp) >= 0) {
        // ---------------------------------------------------------- histories
        // Thread m traces row m of both slots one pair ahead of the tensor
        // cores: at the end of pair p it reads the output partials of each
        // slot, writes that slot's features of pair p + 1 (traced earlier)
        // and tallies pair p; then it traces pair p + 2.
        const int m = 32 * hist_index(warp) + lane;
        const float b5 = __ldg(P.epi + 5 * mlp::H);
        uint32_t dt0 = 0u, dt1 = 0u;   // phases of dots[]
        bool ok = true;
        double t_acc = 0.0;
        uint32_t t_exp = 0xFFFFFFFFu;
        RowRec cur0 = {}, cur1 = {}, nx0 = {}, nx1 = {};
        const bool train = MODE != MODE_TRACE;
        PairInfo pc = (my_pairs > 0 && !train) ? pair_info(P, blockIdx.x) : PairInfo{0, 0, 0};
        PairInfo pn = (my_pairs > 1 && !train) ? pair_info(P, blockIdx.x + gridDim.x) : pc;
        auto get_row = [&](int s, uint32_t k, const PairInfo& pi) {   // row of slot s of my k-th pair
            if constexpr (MODE == MODE_BWD) return bwd_row(P, blockIdx.x + k * gridDim.x, s, m);
            else return train ? train_row(P, blockIdx.x + k * gridDim.x, s, m) : trace_row(P, s, m, pi);
        };
        auto put_row = [&](int s, const RowRec& r, const PairInfo& pi) {
            if constexpr (MODE == MODE_BWD) {
                reinterpret_cast<float*>(sm + S2_DOUT)[s * 128 + m] = r.wt;
                P.dout[(r.pix_flags >> 2) - 1] = r.wt;
            } else if (train) {
                train_features(P, sm, s, m, r);
            } else {
                put_features(P, sm, s, m, r, pi);
            }
        };
        if (my_pairs > 0) {
            cur0 = get_row(0, 0, pc);
            put_row(0, cur0, pc);
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(feat + 0);
            cur1 = get_row(1, 0, pc);
            put_row(1, cur1, pc);
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(feat + 1);
            if (my_pairs > 1) {
                nx0 = get_row(0, 1, pn);
                nx1 = get_row(1, 1, pn);
            }
        }
        for (uint32_t it = 0; it < my_pairs; ++it) {
            const bool more = it + 1 < my_pairs, more2 = it + 2 < my_pairs;
            const PairInfo pn2 = (more2 && !train) ? pair_info(P, blockIdx.x + (it + 2) * gridDim.x) : pn;
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                ok = wait_ab(dots + s, s ? dt1 : dt0, abort) && ok;
                if (s) dt1 ^= 1u;
                else dt0 ^= 1u;
                // partial output dots of the 4 column quarters, in K block 1
                const float* d = reinterpret_cast<const float*>(sm + S2_A + (uint32_t)s * 65536u + 16384u);
                const float out = b5 + d[m] + d[128 + m] + d[256 + m] + d[384 + m];
                if (more) {
                    put_row(s, s ? nx1 : nx0, pn);
                    tc::fence_proxy_async_smem();
                }
                __syncwarp();
                if (more && lane == 0) mbar_arrive(feat + s);
                if (MODE == MODE_TRAIN) {
                    P.out[((s ? cur1 : cur0).pix_flags >> 2) - 1] = out;
                } else if (MODE == MODE_TRACE) {
                    if (pc.exp != t_exp) {
                        flush_trans(P, t_acc, t_exp);
                        t_exp = pc.exp;
                    }
                    t_acc += (double)row_finish(P, s ? cur1 : cur0, pc, out);
                }
            }
            // both slots handed over: trace pair p + 2 while the tensor cores
            // and SiLU warps run pair p + 1
            cur0 = nx0;
            cur1 = nx1;
            if (more2) {
                nx0 = get_row(0, it + 2, pn2);
                nx1 = get_row(1, it + 2, pn2);
            }
            pc = pn;
            pn = pn2;
        }
        if (!train) flush_trans(P, t_acc, t_exp);
        if (!ok) atomicExch(P.err, 9);
    } else {
        // -------------------------------------------------------- SiLU warps
        // Warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows m) and columns
        // 64 ((w - 4) / 4) .. + 63 of every accumulator.
        const int q = (warp - EPI_WARP0) >> 2;
        const int m = 32 * (warp & 3) + lane;
        const int col_q = 64 * q;
        const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
        const float* hbias = P.epi;                        // b_l / 2
        const float* w5 = P.epi + 4 * mlp::H;
        uint32_t ac0 = 0u, ac1 = 0u;
        uint32_t fe0 = 0u, fe1 = 0u;   // MODE_BWD: phases of feat[] (d loss / d out written)
        bool ok = true;
        const float2 half2 = make_float2(0.5f, 0.5f);
        for (uint32_t it = 0; it < my_pairs; ++it) {
            const uint32_t row0 = (blockIdx.x + it * gridDim.x) * 256u + (uint32_t)m;   // MODE_TRAIN: slot 0's row
            for (int l = 0; l < 4; ++l) {
                const float* hb = hbias + 256 * l + col_q;
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    ok = wait_ab(acc + s, s ? ac1 : ac0, abort) && ok;
                    if (s) ac1 ^= 1u;
                    else ac0 ^= 1u;
                    tc::fence_after_sync();
                    unsigned char* a = sm + S2_A + (uint32_t)s * 65536u;
                    if constexpr (MODE == MODE_BWD) {
                        // Step l: l = 0 forms dZ4 = dout w5 SiLU'(z4) (the
                        // placeholder MMA is not read); l = 1..3 form
                        // dZ_{4-l} = dH SiLU'(z_{4-l}) from the accumulator of
                        // dH = dZ_{5-l} W_{5-l}. dZ^T goes to global memory and,
                        // but for the last step, into the slot as the next A.
                        const int zl = 3 - l;   // stored layer of Z and dZ: 3, 2, 1, 0
                        const size_t i = (size_t)row0 + (uint32_t)s * 128u;
                        float dval = 0.f;
                        if (l == 0) {
                            ok = wait_ab(feat + s, s ? fe1 : fe0, abort) && ok;
                            if (s) fe1 ^= 1u;
                            else fe0 ^= 1u;
                            dval = reinterpret_cast<const float*>(sm + S2_DOUT)[s * 128 + m];
                        }
#pragma unroll 1
                        for (int half = 0; half < 2; ++half) {
                            const int col0 = col_q + 32 * half;
                            float v[32];
                            if (l > 0) {
                                uint32_t r[32];
                                tc::tmem_ld32_nowait(tmem + lane_base + 256u * (uint32_t)s + col0, r);
                                tc::tmem_wait_ld();
#pragma unroll
                                for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
                            } else {
#pragma unroll
                                for (int j = 0; j < 32; ++j) v[j] = dval * __ldg(w5 + col0 + j);
                            }
                            // every load of the chunk's Z before any store (a store
                            // could alias a later load and serialise them)
                            __nv_bfloat16 zpre[32];
                            const __nv_bfloat16* zsrc = P.zt[zl] + (size_t)col0 * P.batch + i;
#pragma unroll
                            for (int j = 0; j < 32; ++j)
                                zpre[j] = __ushort_as_bfloat16(
                                    __ldcs(reinterpret_cast<const unsigned short*>(zsrc + (size_t)j * P.batch)));
                            uint32_t w[16];   // bf16x2 of columns (2t, 2t + 1) of this row
#pragma unroll
                            for (int t = 0; t < 16; ++t) {
                                const float a0 = v[2 * t] * mlp::dsilu(__bfloat162float(zpre[2 * t]));
                                const float a1 = v[2 * t + 1] * mlp::dsilu(__bfloat162float(zpre[2 * t + 1]));
                                w[t] = tc::pack_bf16(a0, a1);
                            }
#pragma unroll
                            for (int g = 0; g < 8; ++g)
                                store_pair_t(P.dzt[zl], P.batch, col0 + 4 * g, (uint32_t)i, w[2 * g], w[2 * g + 1], lane);
                            if (l < 3) {
#pragma unroll
                                for (int j = 0; j < 4; ++j)
                                    *reinterpret_cast<uint4*>(a + (col0 >> 6) * 16384 +
                                                              tc::sw128_chunk(m, ((col0 & 63) >> 3) + j)) =
                                        make_uint4(w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]);
                            }
                        }
                        tc::fence_before_sync();
                        if (l < 3) {
                            tc::fence_proxy_async_smem();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(ready + s);
                        } else {
                            __syncwarp();
                            if (lane == 0) mbar_arrive(dots + s);
                        }
                        continue;
                    }
                    float2 dot2 = make_float2(0.f, 0.f);
#pragma unroll 1
                    for (int half = 0; half < 2; ++half) {
                        const int col0 = col_q + 32 * half;
                        uint32_t r[32];
                        tc::tmem_ld32_nowait(tmem + lane_base + 256u * (uint32_t)s + col0, r);
                        tc::tmem_wait_ld();
                        const float4* b4 = reinterpret_cast<const float4*>(hb + 32 * half);
                        uint32_t pk[16];
#pragma unroll
                        for (int g = 0; g < 8; ++g) {
                            const float4 bb = __ldg(b4 + g);
                            // SiLU(z) = h (1 + tanh h), h = z / 2 = acc / 2 + b / 2
                            const float2 h01 = __ffma2_rn(make_float2(__uint_as_float(r[4 * g]), __uint_as_float(r[4 * g + 1])),
                                                          half2, make_float2(bb.x, bb.y));
                            const float2 h23 = __ffma2_rn(make_float2(__uint_as_float(r[4 * g + 2]), __uint_as_float(r[4 * g + 3])),
                                                          half2, make_float2(bb.z, bb.w));
                            const float2 t01 = make_float2(mlp::tanh_approx(h01.x), mlp::tanh_approx(h01.y));
                            const float2 t23 = make_float2(mlp::tanh_approx(h23.x), mlp::tanh_approx(h23.y));
                            const float2 s01 = __ffma2_rn(h01, t01, h01);
                            const float2 s23 = __ffma2_rn(h23, t23, h23);
                            pk[2 * g] = tc::pack_bf16(s01.x, s01.y);
                            pk[2 * g + 1] = tc::pack_bf16(s23.x, s23.y);
                            if constexpr (MODE == MODE_TRAIN) {
                                // Z^T and H^T of the four columns for the backward pass
                                const uint32_t z01 = tc::pack_bf16(h01.x + h01.x, h01.y + h01.y);
                                const uint32_t z23 = tc::pack_bf16(h23.x + h23.x, h23.y + h23.y);
                                store_pair_t(P.zt[l], P.batch, col0 + 4 * g, row0 + (uint32_t)s * 128u, z01, z23, lane);
                                store_pair_t(P.ht[l], P.batch, col0 + 4 * g, row0 + (uint32_t)s * 128u, pk[2 * g],
                                             pk[2 * g + 1], lane);
                            }
                        }
                        if (l < 3) {
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                *reinterpret_cast<uint4*>(a + (col0 >> 6) * 16384 +
                                                          tc::sw128_chunk(m, ((col0 & 63) >> 3) + j)) =
                                    make_uint4(pk[4 * j], pk[4 * j + 1], pk[4 * j + 2], pk[4 * j + 3]);
                        } else {
                            // output: the BF16 activations against w5
                            const float2* w2 = reinterpret_cast<const float2*>(w5 + col0);
#pragma unroll
                            for (int g = 0; g < 16; ++g) {
                                const float2 ab = make_float2(__uint_as_float(pk[g] << 16),
                                                              __uint_as_float(pk[g] & 0xFFFF0000u));
                                dot2 = __ffma2_rn(ab, __ldg(w2 + g), dot2);
                            }
                        }
                    }
                    tc::fence_before_sync();
                    if (l < 3) {
                        tc::fence_proxy_async_smem();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(ready + s);
                    } else {
                        // partial output dots meet in K block 1 of the slot's A
                        // buffer (free once its last layer's MMAs are done; the
                        // next writer there is the next pair's layer-1 epilogue)
                        reinterpret_cast<float*>(a + 16384)[q * 128 + m] = dot2.x + dot2.y;
                        __syncwarp();
                        if (lane == 0) mbar_arrive(dots + s);
                    }
                }
            }
        }
        if (!ok) atomicExch(P.err, 9);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

}  // namespace sur
}  // namespace sas
