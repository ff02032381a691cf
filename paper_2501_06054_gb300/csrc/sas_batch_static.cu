// Batched trace for callers that cannot allocate device memory.
//
// sas_trace_batch_static runs the same persistent batch kernel as
// sas_trace_batch, but everything it needs besides the caller's inputs and
// outputs (per-experiment model constants, quadrature tables, work items,
// the work counter and the seed) lives in one file-scope device array of
// fixed size. The array exists on every GPU that loads the library, from
// load until process exit. The entry point calls no device allocator.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "sas_batch.cuh"
#include "sas_host.h"

namespace sas {
sas_status set_error(sas_status s, const std::string& msg);
sas_status set_cuda_error(cudaError_t e, const char* what);
double host_flops_per_history(const sas_model_desc& m, int n_poly, int n_orient);
}  // namespace sas

using namespace sas;

#define SAS_STATIC_SCRATCH_BYTES (8u << 20)   // 8 MiB

// The scratch. Host code must not pass this name to a kernel: on the host it
// is only a stand-in for the symbol. Its device address comes from
// cudaGetSymbolAddress in the caller's current context (scratch_base below).
static __device__ __align__(256) unsigned char g_batch_scratch[SAS_STATIC_SCRATCH_BYTES];

namespace {

// Device address of the scratch in the current CUDA context, looked up on
// every call with the caller's device current. The address belongs to the
// module loaded in that context, not to the device: a second context on the
// same GPU (a plugin host's own driver-API context) or the primary context
// re-created after cudaDeviceReset gets its own copy of the array at its
// own address, so nothing is cached across calls. The lookup is a host-side
// table query once the module is loaded (the first call in a context loads
// it).
sas_status scratch_base(unsigned char** out)
{
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_batch_scratch);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaGetSymbolAddress(static batch scratch)");
    *out = static_cast<unsigned char*>(p);
    return SAS_OK;
}

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" {

sas_status sas_trace_batch_static(const sas_instrument* inst, const sas_model_desc* models,
                                  const uint64_t* counts, size_t n_exp, uint64_t seed, double* sum_w,
                                  double* sum_w2, uint64_t* count, double* transmitted, void* stream)
{
    if (!models || !counts || n_exp == 0) return set_error(SAS_ERR_ARG, "empty batch");
    if (!sum_w || !sum_w2 || !count || !transmitted) return set_error(SAS_ERR_ARG, "NULL output buffer");
    if (n_exp > 0x7FFFFFFFull) return set_error(SAS_ERR_ARG, "too many experiments");
    sas_status st = validate_instrument(inst);
    if (st != SAS_OK) return st;
    const cudaStream_t s = (cudaStream_t)stream;
    const int npix = (int)(inst->nx * inst->ny);
    int dev = 0, sms = 0, optin = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (ce != cudaSuccess) return set_cuda_error(ce, "device query");

    // tables, tally choice and work items (as sas_create_batch, fixed config)
    std::vector<BatchExp> exps(n_exp);
    std::vector<float> poly, orient;
    std::vector<WorkItem> items;
    std::vector<double> icost;
    size_t smem = 0;
    int any_hist = 0;
    const double target = 2e9;
    // the histogram kernel is built without these two kinds
    bool full = false;
    for (size_t e = 0; e < n_exp; ++e)
        full |= models[e].kind == SAS_ELLIPTICAL_CYLINDER || models[e].kind == SAS_HOLLOW_RECTANGULAR_PRISM;
    for (size_t e = 0; e < n_exp; ++e) {
        const sas_model_desc& m = models[e];
        st = validate_model(&m);
        if (st != SAS_OK) return st;
        if (m.precision != SAS_FP32) return set_error(SAS_ERR_ARG, "batched experiments are FP32");
        if (m.kind == SAS_SHAPE_INDEPENDENT)
            return set_error(SAS_ERR_ARG, "shape-independent laws are traced one by one (sas_trace), not batched");
        if (m.sq_kind == SAS_SQ_HAYTER_MSA)
            return set_error(SAS_ERR_ARG, "the Hayter MSA S(Q) is traced one by one (sas_trace), not batched");
        if (m.self_attenuation)
            return set_error(SAS_ERR_ARG, "the allocation-free batch does not build self-attenuation tables; "
                                          "use sas_create_batch");
        ModelTables t;
        st = build_model_tables(m, t, instrument_q_max(*inst));
        if (st != SAS_OK) return st;
        BatchExp& x = exps[e];
        std::memset(&x, 0, sizeof(x));
        x.mc = model_const<float>(m, t);
        x.poly_off = (uint32_t)poly.size();
        x.orient_off = (uint32_t)orient.size();
        for (double v : t.poly) poly.push_back((float)v);
        for (double v : t.orient) orient.push_back((float)v);
        const bool hist = !full && t.n_orient <= 1 &&
                          table_bytes<float>(t.n_poly, 0, 0) + hist_bytes(npix) <= (size_t)optin;
        x.use_hist = hist ? 1 : 0;
        x.stage_orient = (!hist && t.n_orient > 1 && table_bytes<float>(t.n_poly, t.n_orient, 1) <= (size_t)optin)
                             ? 1 : 0;
        size_t need = hist ? table_bytes<float>(t.n_poly, 0, 0) + hist_bytes(npix)
                           : table_bytes<float>(t.n_poly, t.n_orient, x.stage_orient);
        smem = std::max(smem, need);
        any_hist |= x.use_hist;
        const double cost = host_flops_per_history(m, t.n_poly, std::max(t.n_orient, 1));
        const uint64_t c = (uint64_t)std::min(std::max(std::floor(target / cost), 1024.0), 1073741824.0);
        for (uint64_t f = 0; f < counts[e]; f += c) {
            WorkItem w;
            w.first = f;
            w.exp = (uint32_t)e;
            w.n = (uint32_t)std::min<uint64_t>(c, counts[e] - f);
            items.push_back(w);
            icost.push_back(cost * (double)w.n);
        }
    }
    std::vector<size_t> idx(items.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t b) { return icost[a] > icost[b]; });
    std::vector<WorkItem> sorted(items.size());
    for (size_t i = 0; i < idx.size(); ++i) sorted[i] = items[idx[i]];

    // scratch layout: [control 256 B | experiments | items | poly | orient]
    const size_t off_exps = 256;
    const size_t off_items = off_exps + up256(n_exp * sizeof(BatchExp));
    const size_t off_poly = off_items + up256(sorted.size() * sizeof(WorkItem));
    const size_t off_orient = off_poly + up256(poly.size() * sizeof(float));
    const size_t total = off_orient + up256(orient.size() * sizeof(float));
    if (total > SAS_STATIC_SCRATCH_BYTES)
        return set_error(SAS_ERR_ARG, "this batch needs " + std::to_string(total) +
                                          " bytes of scratch; the static scratch holds " +
                                          std::to_string(SAS_STATIC_SCRATCH_BYTES));
    if (sorted.size() > 0xFFFFFFF0ull) return set_error(SAS_ERR_ARG, "too many work items");

    unsigned char* base = nullptr;
    st = scratch_base(&base);
    if (st != SAS_OK) return st;
    unsigned int* queue = reinterpret_cast<unsigned int*>(base);
    uint64_t* d_seed = reinterpret_cast<uint64_t*>(base + 8);
    // the work counter must start at zero on every call
    ce = cudaMemsetAsync(queue, 0, sizeof(unsigned int), s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(d_seed, &seed, sizeof(seed), cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(base + off_exps, exps.data(), n_exp * sizeof(BatchExp), cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess && !sorted.empty())
        ce = cudaMemcpyAsync(base + off_items, sorted.data(), sorted.size() * sizeof(WorkItem),
                             cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess && !poly.empty())
        ce = cudaMemcpyAsync(base + off_poly, poly.data(), poly.size() * sizeof(float), cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess && !orient.empty())
        ce = cudaMemcpyAsync(base + off_orient, orient.data(), orient.size() * sizeof(float),
                             cudaMemcpyHostToDevice, s);
    // outputs start at zero
    const size_t det = n_exp * (size_t)npix;
    if (ce == cudaSuccess) ce = cudaMemsetAsync(sum_w, 0, det * sizeof(double), s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(sum_w2, 0, det * sizeof(double), s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(count, 0, det * sizeof(uint64_t), s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(transmitted, 0, n_exp * sizeof(double), s);
    if (ce != cudaSuccess) return set_cuda_error(ce, "sas_trace_batch_static upload");
    if (sorted.empty()) return SAS_OK;

    BatchParams P;
    std::memset(&P, 0, sizeof(P));
    P.in = inst_const<float>(*inst);
    P.exps = reinterpret_cast<const BatchExp*>(base + off_exps);
    P.items = reinterpret_cast<const WorkItem*>(base + off_items);
    P.n_items = (uint32_t)sorted.size();
    P.poly = reinterpret_cast<const float*>(base + off_poly);
    P.orient = reinterpret_cast<const float*>(base + off_orient);
    P.seed = d_seed;
    P.queue = queue;
    P.sum_w = sum_w;
    P.sum_w2 = sum_w2;
    P.count = reinterpret_cast<unsigned long long*>(count);
    P.trans = transmitted;
    P.npix = npix;
    auto kern = any_hist ? batch_kernel<1> : batch_kernel<0>;
    const int block = 512;
    ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    if (ce == cudaSuccess) ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem);
    if (ce != cudaSuccess) return set_cuda_error(ce, "batch kernel set-up");
    if (per_sm < 1) return set_error(SAS_ERR_ARG, "batch launch shape does not fit on an SM");
    kern<<<sms * per_sm, block, smem, s>>>(P);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return set_cuda_error(ce, "batch kernel launch");
    return SAS_OK;
}

}  // extern "C"
