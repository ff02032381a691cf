// Batched form: thousands of experiments (different models, parameters and
// neutron counts) traced by one persistent kernel launch.
//
// The host cuts every experiment's index range into work items whose cost
// (histories x FLOP per history) is close to a target and orders them
// longest-first. Persistent CTAs (a multiple of the SM count) take items
// from a global atomic counter; a CTA works on one item at a time with all
// its warps (one history per lane, batches of 32 consecutive indices), so
// the model kind is uniform per CTA. Cheap models tally into a per-CTA
// shared-memory histogram flushed into the experiment's FP64 detector at
// the end of each item; models with an orientation average stage their
// orientation table in shared memory instead and tally with FP64 atomics.
#pragma once

#include "sas_kernels.cuh"

namespace sas {

struct BatchExp {
    ModelConst<float> mc;
    uint32_t poly_off;     // float offset into the concatenated poly tables
    uint32_t orient_off;   // float offset into the concatenated orient tables
    int use_hist;          // tally through the shared-memory histogram
    int stage_orient;      // copy the orientation table into shared memory
};

struct WorkItem {
    uint64_t first;        // first neutron index
    uint32_t exp;          // experiment (also its Philox experiment id)
    uint32_t n;            // histories in the item
};

struct BatchParams {
    InstConst<float> in;
    const BatchExp* exps;
    const WorkItem* items;
    uint32_t n_items;
    const float* poly;
    const float* orient;
    const uint64_t* seed;          // device scalar (updated between graph launches)
    unsigned int* queue;           // device work counter, zeroed in the graph
    double* sum_w;                 // [n_exp][npix]
    double* sum_w2;
    unsigned long long* count;
    double* trans;                 // [n_exp]
    int npix;
};

template <int KIND, int HIST, bool ATT>
__device__ __forceinline__ void batch_item(const BatchParams& P, const ModelConst<float>& mc,
                                           const float* poly, const float* orient,
                                           const WorkItem& w, const SmemHist& h, uint64_t seed,
                                           Kahan<float>& tr)
{
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    double* sw = P.sum_w + (size_t)w.exp * P.npix;
    double* sw2 = P.sum_w2 + (size_t)w.exp * P.npix;
    unsigned long long* cnt = P.count + (size_t)w.exp * P.npix;
    for (uint32_t base = (threadIdx.x >> 5) * 32u; base < w.n; base += (uint32_t)wpb * 32u) {
        const uint32_t j = base + lane;
        int pix = -1;
        float wt = 0.f;
        if (j < w.n) {
            const History<float> hs = history<float, ATT>(P.in, mc.att, seed, w.exp, w.first + j);
            tr.add(hs.wt);
            if (hs.pixel >= 0) {
                wt = hs.pref * dsigma_history<float, KIND, true>(hs.q, mc, poly, orient, seed, w.exp, w.first + j);
                pix = hs.pixel;
            }
        }
        if (HIST) {
            if (pix >= 0) h.add(cnt, pix, wt, wt * wt, 1u);
        } else if (pix >= 0) {
            atomicAdd(sw + pix, (double)wt);
            atomicAdd(sw2 + pix, (double)wt * (double)wt);
            atomicAdd(cnt + pix, 1ull);
        }
    }
}

// FULL: every kind a batch takes (the shape-independent laws are refused on
// the host). The histogram kernel (batch_kernel<1>) is compiled without the
// elliptical cylinder and the hollow prism, whose code would push its
// register allocation into spills; the host launches batch_kernel<0> for
// any batch that holds one of them.
template <int HIST, bool ATT, bool FULL>
__device__ __forceinline__ void batch_dispatch(const BatchParams& P, const ModelConst<float>& mc, const float* poly,
                                               const float* orient, const WorkItem& w, const SmemHist& h,
                                               uint64_t seed, Kahan<float>& tr)
{
    if constexpr (FULL) {
        if (mc.kind == SAS_ELLIPTICAL_CYLINDER) {
            batch_item<SAS_ELLIPTICAL_CYLINDER, HIST, ATT>(P, mc, poly, orient, w, h, seed, tr);
            return;
        }
        if (mc.kind == SAS_HOLLOW_RECTANGULAR_PRISM) {
            batch_item<SAS_HOLLOW_RECTANGULAR_PRISM, HIST, ATT>(P, mc, poly, orient, w, h, seed, tr);
            return;
        }
    }
    switch (mc.kind) {
    case SAS_SPHERE: batch_item<SAS_SPHERE, HIST, ATT>(P, mc, poly, orient, w, h, seed, tr); break;
    case SAS_CORE_SHELL: batch_item<SAS_CORE_SHELL, HIST, ATT>(P, mc, poly, orient, w, h, seed, tr); break;
    case SAS_CYLINDER: batch_item<SAS_CYLINDER, HIST, ATT>(P, mc, poly, orient, w, h, seed, tr); break;
    case SAS_TRIAXIAL_ELLIPSOID: batch_item<SAS_TRIAXIAL_ELLIPSOID, HIST, ATT>(P, mc, poly, orient, w, h, seed, tr); break;
    case SAS_PARALLELEPIPED: batch_item<SAS_PARALLELEPIPED, HIST, ATT>(P, mc, poly, orient, w, h, seed, tr); break;
    case SAS_CAPPED_CYLINDER: batch_item<SAS_CAPPED_CYLINDER, HIST, ATT>(P, mc, poly, orient, w, h, seed, tr); break;
    case SAS_BARBELL: batch_item<SAS_BARBELL, HIST, ATT>(P, mc, poly, orient, w, h, seed, tr); break;
    case SAS_CORE_SHELL_CYLINDER: batch_item<SAS_CORE_SHELL_CYLINDER, HIST, ATT>(P, mc, poly, orient, w, h, seed, tr); break;
    case SAS_HOLLOW_CYLINDER: batch_item<SAS_HOLLOW_CYLINDER, HIST, ATT>(P, mc, poly, orient, w, h, seed, tr); break;
    case SAS_CORE_SHELL_ELLIPSOID: batch_item<SAS_CORE_SHELL_ELLIPSOID, HIST, ATT>(P, mc, poly, orient, w, h, seed, tr); break;
    case SAS_CORE_SHELL_BICELLE: batch_item<SAS_CORE_SHELL_BICELLE, HIST, ATT>(P, mc, poly, orient, w, h, seed, tr); break;
    default: batch_item<SAS_ELLIPSOID, HIST, ATT>(P, mc, poly, orient, w, h, seed, tr); break;
    }
}

template <int HIST_OK>
__global__ void __launch_bounds__(1024) batch_kernel(const BatchParams P)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned int s_item;
    __shared__ ModelConst<float> s_mc;
    __shared__ BatchExp s_e;
    const uint64_t seed = *P.seed;
    float* s_poly = reinterpret_cast<float*>(smem);
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(P.queue, 1u);
        __syncthreads();
        const unsigned int it = s_item;
        if (it >= P.n_items) break;
        const WorkItem w = P.items[it];
        if (threadIdx.x == 0) {
            s_e = P.exps[w.exp];
            s_mc = s_e.mc;
        }
        __syncthreads();
        const ModelConst<float> mc = s_mc;
        const int np = mc.n_poly * SAS_POLY_STRIDE;
        for (int i = threadIdx.x; i < np; i += blockDim.x) s_poly[i] = P.poly[s_e.poly_off + i];
        const float* orient = P.orient + s_e.orient_off;
        if (s_e.stage_orient) {
            float* s_or = s_poly + np;
            const int no = mc.n_orient * SAS_ORIENT_STRIDE;
            for (int i = threadIdx.x; i < no; i += blockDim.x) s_or[i] = orient[i];
            orient = s_or;
        }
        SmemHist h;
        h.bind(smem + table_bytes<float>(mc.n_poly, 0, 0), P.npix);
        const bool hist = HIST_OK && s_e.use_hist;
        if (hist) h.clear();
        __syncthreads();
        Kahan<float> tr;
        if (mc.att.n > 0) {
            if (hist) batch_dispatch<HIST_OK, true, HIST_OK == 0>(P, mc, s_poly, orient, w, h, seed, tr);
            else batch_dispatch<0, true, HIST_OK == 0>(P, mc, s_poly, orient, w, h, seed, tr);
        } else {
            if (hist) batch_dispatch<HIST_OK, false, HIST_OK == 0>(P, mc, s_poly, orient, w, h, seed, tr);
            else batch_dispatch<0, false, HIST_OK == 0>(P, mc, s_poly, orient, w, h, seed, tr);
        }
        double t = (double)tr.s - (double)tr.c;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if ((threadIdx.x & 31) == 0 && t != 0.0) atomicAdd(P.trans + w.exp, t);
        __syncthreads();
        if (hist) {   // FP64 per-bin reduction of this item into its detector
            h.flush(P.sum_w + (size_t)w.exp * P.npix, P.sum_w2 + (size_t)w.exp * P.npix,
                    P.count + (size_t)w.exp * P.npix);
            __syncthreads();
        }
    }
}

}  // namespace sas
