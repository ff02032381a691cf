// Surrogate box, feature map and the exact quadrature that generates the
// training targets (device side).
#pragma once

#include "sas_batch.cuh"
#include "sas_device.cuh"
#include "sas_mlp.cuh"

namespace sas {
namespace sur {

constexpr int MAX_BUCKETS = 64;
constexpr int MAX_POLY = 64;
constexpr int MAX_GL = 128;
constexpr uint32_t DATA_EXP_ID = 0x80000001u;   // Philox experiment id of the training draws

// Box and feature scaling in the trace precision (FP32).
struct Box {
    float q_max, r_min, r_max, l_min, l_max, so_min, so_max, sp_min, sp_max;
    float u_max, v_max, la_min, la_max;  // feature ranges (la: ln a)
    float four_w;                        // angular step of the Fourier features of u and v
    int n_four;                          // Fourier pairs of u, and as many of v
    int n_buckets, n_poly, n_gamma, n_psi;
    int kind;                            // SAS_CYLINDER or SAS_ELLIPSOID (L = 2 R_p)
};

// Raw parameters of one evaluation: q_par, q_perp (1/A), R, L (A), sigma_orient
// (rad), sigma_poly, bucket index (as float), pad.
struct Raw {
    float qpar, qperp, R, L, so, sp, bucket, pad;
};

// Feature vector (64 wide). With u = q_par L / 2, v = q_perp R, a = L / (2R):
//   0..4   u, v, ln a, sigma_orient, sigma_poly, each scaled to [-1, 1]
//          over the box;
//   5..7   the envelopes ln(1 + u^2) / 4 - 1, ln(1 + v^2) / 4 - 1,
//          ln(1 + (u / a)^2) / 4 - 1 (u / a = q_par R);
//   8..    n_four (sin, cos) pairs of k w u, then n_four pairs of k w v
//          (k = 1..n_four, w = four_w = 1/2);
//   63     1 (the bias of layer 1); the columns between are 0.
constexpr int FEAT_FOURIER0 = 8;

// The eight scaled inputs and envelopes (columns 0..7).
__device__ __forceinline__ void feature_head(const Box& b, float u, float v, float R, float L, float so, float sp,
                                             float* h8)
{
    const float a = 0.5f * L / R;
    const float ua = u / a;
    h8[0] = 2.f * u / b.u_max - 1.f;
    h8[1] = 2.f * v / b.v_max - 1.f;
    h8[2] = 2.f * (__logf(a) - b.la_min) / (b.la_max - b.la_min) - 1.f;
    h8[3] = 2.f * (so - b.so_min) / (b.so_max - b.so_min) - 1.f;
    h8[4] = 2.f * (sp - b.sp_min) / (b.sp_max - b.sp_min) - 1.f;
    h8[5] = 0.25f * __logf(fmaf(u, u, 1.f)) - 1.f;
    h8[6] = 0.25f * __logf(fmaf(v, v, 1.f)) - 1.f;
    h8[7] = 0.25f * __logf(fmaf(ua, ua, 1.f)) - 1.f;
}

// Column col (>= FEAT_FOURIER0) of the Fourier block: walks the u pairs,
// then the v pairs, advancing the running (sin, cos) after each cosine.
struct FourierWalk {
    float su1, cu1, sv1, cv1, su, cu, sv, cv;
    int end_u, end_v;
    __device__ __forceinline__ FourierWalk(const Box& b, bool on, float u, float v)
    {
        su1 = 0.f, cu1 = 1.f, sv1 = 0.f, cv1 = 1.f;
        if (on) {
            sas_sincosf(b.four_w * u, su1, cu1);
            sas_sincosf(b.four_w * v, sv1, cv1);
        }
        su = su1, cu = cu1, sv = sv1, cv = cv1;
        const int nf = on ? b.n_four : 0;
        end_u = FEAT_FOURIER0 + 2 * nf;
        end_v = end_u + 2 * nf;
    }
    __device__ __forceinline__ float next(int col)
    {
        float x = 0.f;
        if (col < end_u) {
            const bool odd = (col - FEAT_FOURIER0) & 1;
            x = odd ? cu : su;
            if (odd) {
                const float sn = fmaf(su, cu1, cu * su1);
                const float cn = fmaf(cu, cu1, -(su * su1));
                su = sn;
                cu = cn;
            }
        } else if (col < end_v) {
            const bool odd = (col - end_u) & 1;
            x = odd ? cv : sv;
            if (odd) {
                const float sn = fmaf(sv, cv1, cv * sv1);
                const float cn = fmaf(cv, cv1, -(sv * sv1));
                sv = sn;
                cv = cn;
            }
        }
        return x;
    }
};

// The feature vector in registers (the training and evaluation kernels);
// every column index is a compile-time constant, so f64 stays in registers.
__device__ __forceinline__ void features(const Box& b, float qpar, float qperp, float R, float L, float so,
                                         float sp, float* f64)
{
    const float u = qpar * 0.5f * L;
    const float v = qperp * R;
    feature_head(b, u, v, R, L, so, sp, f64);
    FourierWalk fw(b, true, u, v);
#pragma unroll
    for (int col = FEAT_FOURIER0; col < 63; ++col) f64[col] = fw.next(col);
    f64[63] = 1.f;
}

// The same feature vector written straight into row m of a swizzled 64-wide
// BF16 K block, 8 columns at a time (nothing beyond one chunk is live);
// `on` false writes a zero row. NF > 0 fixes the number of Fourier pairs at
// compile time (no per-column selects); NF = 0 reads it from the box.
template <int NF>
__device__ __forceinline__ void write_features_n(const Box& b, bool on, float qpar, float qperp, float R, float L,
                                                 float so, float sp, unsigned char* kblock, int m)
{
    const float u = qpar * 0.5f * L;
    const float v = qperp * R;
    float head[8];
    feature_head(b, u, v, R, L, so, sp, head);
    FourierWalk fw(b, on, u, v);
    if constexpr (NF > 0) {
        fw.end_u = FEAT_FOURIER0 + 2 * NF;
        fw.end_v = FEAT_FOURIER0 + 4 * NF;
    }
#pragma unroll
    for (int chunk = 0; chunk < 8; ++chunk) {
        float x8[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int col = 8 * chunk + j;
            float x;
            if (chunk == 0) x = on ? head[j] : 0.f;
            else if (col == 63) x = on ? 1.f : 0.f;
            else if (NF > 0 && col >= FEAT_FOURIER0 + 4 * NF) x = 0.f;
            else x = (NF > 0 && !on) ? 0.f : fw.next(col);
            x8[j] = x;
        }
        uint4 pk;
        pk.x = tc::pack_bf16(x8[0], x8[1]);
        pk.y = tc::pack_bf16(x8[2], x8[3]);
        pk.z = tc::pack_bf16(x8[4], x8[5]);
        pk.w = tc::pack_bf16(x8[6], x8[7]);
        *reinterpret_cast<uint4*>(kblock + tc::sw128_chunk(m, chunk)) = pk;
    }
}

__device__ __forceinline__ void write_features(const Box& b, bool on, float qpar, float qperp, float R, float L,
                                               float so, float sp, unsigned char* kblock, int m)
{
    if (b.n_four == 12) write_features_n<12>(b, on, qpar, qperp, R, L, so, sp, kblock, m);
    else write_features_n<0>(b, on, qpar, qperp, R, L, so, sp, kblock, m);
}

__device__ __forceinline__ bool in_box(const Box& b, float q, float R, float L, float so, float sp)
{
    return q <= b.q_max && R >= b.r_min && R <= b.r_max && L >= b.l_min && L <= b.l_max && so >= b.so_min &&
           so <= b.so_max && sp >= b.sp_min && sp <= b.sp_max;
}

// Tables for the exact quadrature of the training targets.
struct Tables {
    const float* gl_g;      // [n_gamma] Gauss-Legendre nodes on [-1, 1]
    const float* glw_g;     // [n_gamma] weights
    const float* gl_p;      // [n_psi]
    const float* glw_p;     // [n_psi]
    const float* bucket_sp; // [n_buckets] sigma_poly of each bucket
    const float* poly_x;    // [n_buckets][n_poly] Schulz nodes r_i / R
    const float* poly_w;    // [n_buckets][n_poly] w_i x_i^4 / sum(w x^4)
    const float2* poly_x2w; // [n_buckets][n_poly] (x_i^2, w_i x_i^4 / sum(w x^4))
    const float2* psi_cs;   // [n_psi] (cos, sin) of the psi nodes pi (gl_p + 1)
};

// Normalised averaged form factor P = <|F|^2> / (drho^2 <V^2>) of the
// box's body at (q_par, q_perp) about the mean axis z, by the same
// quadrature as the trace (Gaussian cap of width so truncated at 3 so, GL
// in gamma and psi, Schulz nodes of the bucket on the radius). Cylinder:
// sinc(Q_C L / 2)^2 a(Q_AB r)^2; ellipsoid of revolution (R_p = L / 2 fixed,
// r polydisperse, V^2 ~ r^4 as for the cylinder): (3 g(x))^2 with
// x^2 = r^2 Q_AB^2 + R_p^2 Q_C^2. Computed by one warp; every lane returns it.
__device__ __forceinline__ double exact_pbar_warp(const Box& b, const Tables& t, const Raw& r)
{
    const int lane = threadIdx.x & 31;
    const int bk = (int)r.bucket;
    const float* px = t.poly_x + bk * b.n_poly;
    const float* pw = t.poly_w + bk * b.n_poly;
    const float gmax = fminf(3.0f * r.so, 3.14159265f);
    const float inv2s2 = 0.5f / (r.so * r.so);
    const float q2 = r.qpar * r.qpar + r.qperp * r.qperp;
    const float R2 = r.R * r.R;
    // the warp shares the sample: |Q x c| <= |Q| bounds every argument, so
    // the (ascending) radius nodes split once into the tiers of 2 J1(x)/x
    const float qm = q2 * R2;
    auto tier_end = [&](int lo, float smax) {
        int hi = b.n_poly;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (px[mid] * px[mid] * qm <= smax) lo = mid + 1;
            else hi = mid;
        }
        return lo;
    };
    const int t4 = tier_end(0, SAS_J1R_SMAX);
    const int t6 = tier_end(t4, SAS_J1V_SMAX);
    const int t8 = tier_end(t6, SAS_J1P_SMAX);
    const int no = b.n_gamma * b.n_psi;
    Kahan<float> num, den;
    int i = lane / b.n_psi, k = lane - i * b.n_psi;    // node o = i n_psi + k, stepped by 32
    for (int o = lane; o < no; o += 32) {
        const float g = 0.5f * gmax * (t.gl_g[i] + 1.0f);
        float sg, cg;
        __sincosf(g, &sg, &cg);
        const float cp = t.psi_cs[k].x;   // Q lies in the plane of the axis and e_1: only cos(psi) enters
        const float wo = t.glw_g[i] * sg * __expf(-g * g * inv2s2) * t.glw_p[k];
        const float qc = r.qperp * sg * cp + r.qpar * cg;
        const float qab2 = fmaxf(q2 - qc * qc, 0.0f);
        if (b.kind == SAS_ELLIPSOID) {
            const float pol = 0.25f * r.L * r.L * (qc * qc);
            const float qabR2 = qab2 * R2;
            const float2* xw = t.poly_x2w + bk * b.n_poly;
            float inner = 0.f;
#pragma unroll 4
            for (int j = 0; j < b.n_poly; ++j) {
                const float2 v = xw[j];
                // floored so that Q = 0 takes the series branch
                const float x2 = fmaxf(fmaf(qabR2, v.x, pol), 1e-30f);
                const float inv = rsqrtf(x2);
                const float g = 3.0f * M<float>::sphere_g(x2 * inv, inv);
                inner = fmaf(v.y, g * g, inner);
            }
            num.add(wo * inner);
            den.add(wo);
            for (k += 32; k >= b.n_psi; k -= b.n_psi) ++i;
            continue;
        }
        const float y = fabsf(qc) * 0.5f * r.L;
        const float sn = M<float>::sinc(y, __fdividef(1.0f, y));
        const float qabR2 = qab2 * R2;
        const float2* xw = t.poly_x2w + bk * b.n_poly;
        float inner = 0.f;
#pragma unroll 4
        for (int j = 0; j < t4; ++j) {
            const float2 v = xw[j];
            const float a = sas_cyl_a_r(qabR2 * v.x);
            inner = fmaf(v.y, a * a, inner);
        }
#pragma unroll 4
        for (int j = t4; j < t6; ++j) {
            const float2 v = xw[j];
            const float a = sas_cyl_a_v(qabR2 * v.x);
            inner = fmaf(v.y, a * a, inner);
        }
#pragma unroll 2
        for (int j = t6; j < t8; ++j) {
            const float2 v = xw[j];
            const float a = sas_cyl_a_s(qabR2 * v.x);
            inner = fmaf(v.y, a * a, inner);
        }
        if (t8 < b.n_poly) {
            const float qabR = M<float>::sqrt_(qabR2);
            for (int j = t8; j < b.n_poly; ++j) {
                const float x = px[j];
                const float sx = qabR2 * (x * x);
                float a;
                if (sx <= SAS_J1P_SMAX) {
                    a = sas_cyl_a_s(sx);
                } else {
                    const float xx = qabR * x;
                    a = sas_cyl_a_large(xx, __frcp_rn(xx), rsqrtf(xx));
                }
                inner = fmaf(pw[j], a * a, inner);
            }
        }
        num.add(wo * sn * sn * inner);
        den.add(wo);
        for (k += 32; k >= b.n_psi; k -= b.n_psi) ++i;
    }
    double n = (double)num.s - (double)num.c, d = (double)den.s - (double)den.c;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        n += __shfl_xor_sync(0xffffffffu, n, s);
        d += __shfl_xor_sync(0xffffffffu, d, s);
    }
    return n / d;
}

struct SurExp {
    float nx, ny, nz;      // mean axis
    float R, L, so, sp;    // cylinder parameters
    float scale_p;         // phi drho^2 <V^2> / <V> (1/angstrom): dSigma = scale_p P
    int in_box;
    int pad[3];
};

struct STParams {
    InstConst<float> in;
    Box box;
    const float* epi;        // [1281]: b_l / 2 (l = 1..4, 4 x 256), w5 (256), b5
    const uint64_t* seed;    // device scalar
    uint32_t philox_base;    // Philox experiment id = philox_base + item experiment
    // single experiment or batch items; item i holds pairs (256 histories)
    // pair_prefix[i] .. pair_prefix[i + 1] - 1 (every item but the last of an
    // experiment is a multiple of 256 long)
    const WorkItem* items;
    const uint32_t* pair_prefix;   // [n_items]
    uint32_t n_items;
    uint32_t n_pairs;
    const SurExp* sexp;
    const BatchExp* bexp;    // exact fallback (model constants and table offsets)
    const float* poly;
    const float* orient;
    double* sum_w;
    double* sum_w2;
    unsigned long long* count;
    double* trans;
    int npix;
    unsigned long long* fallbacks;
    int* err;
    // training forward (MODE_TRAIN of the warp-specialised kernel): pair p
    // holds rows [256 p, 256 p + 256) of the minibatch; row i reads data set
    // row (step * batch + i) mod n_data and stores the BF16 features X^T
    // [64][batch], pre-activations Z_l^T and activations H_l^T [256][batch]
    // and the output log P [batch]
    const Raw* raw;
    uint64_t n_data;
    const uint32_t* step;
    uint32_t batch;
    float* out;
    __nv_bfloat16* xt;
    __nv_bfloat16* zt[4];
    __nv_bfloat16* ht[4];
    // training backward (MODE_BWD): d loss / d out = scale (pred - y) into
    // dout [batch]; dZ_l^T [256][batch] from the stored Z_l^T
    const float* pred;
    const float* y;
    float scale;
    float* dout;
    __nv_bfloat16* dzt[4];
};

}  // namespace sur
}  // namespace sas
