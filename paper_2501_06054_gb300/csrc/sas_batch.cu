// Host runtime of the batched form: tables of all experiments, LPT-ordered
// work items, one persistent kernel captured in a CUDA graph, autotuning of
// the launch shape and item size.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sas_batch.cuh"
#include "sas_host.h"
#include "sas_sur_host.h"

namespace sas {
sas_status set_error(sas_status s, const std::string& msg);
sas_status set_cuda_error(cudaError_t e, const char* what);
double host_flops_per_history(const sas_model_desc& m, int n_poly, int n_orient);
unsigned long long* experiment_fallback_counter(const sas_experiment* e);
cudaStream_t experiment_stream(const sas_experiment* e);
}  // namespace sas

using namespace sas;

#define SAS_CUDA_B(call, what)                                     \
    do {                                                           \
        cudaError_t _e = (call);                                   \
        if (_e != cudaSuccess) return set_cuda_error(_e, what);    \
    } while (0)

struct sas_batch {
    sas_instrument inst;
    InstConst<float> icf;
    int device = 0, sm_count = 0, smem_optin = 0;
    cudaStream_t stream = nullptr;     // caller's stream: graph launches go here
    cudaStream_t cap = nullptr;        // private stream used for graph capture
    size_t n_exp = 0;
    int npix = 0;
    std::vector<uint64_t> counts;
    std::vector<double> cost;          // FLOP per history (scheduling cost model)
    std::vector<BatchExp> h_exps;
    std::vector<int> hist_capable;     // the histogram fits and the model is cheap
    std::vector<int> orient_stageable;
    BatchExp* d_exps = nullptr;
    WorkItem* d_items = nullptr;
    size_t items_cap = 0;
    uint32_t n_items = 0;
    float* d_poly = nullptr;
    float* d_orient = nullptr;
    uint64_t* d_seed = nullptr;
    unsigned int* d_queue = nullptr;
    double* d_sum_w = nullptr;
    double* d_sum_w2 = nullptr;
    unsigned long long* d_count = nullptr;
    double* d_trans = nullptr;
    sas_batch_config cfg;
    size_t smem = 0;
    int hist_ok = 0;
    int grid = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t total_histories = 0;
    std::vector<sas_model_desc> models;
    // learned surrogates for the in-box experiments: slot 0 cylinders,
    // slot 1 ellipsoids; use_sur[e] = serving slot + 1, or 0 (exact)
    const sas_surrogate* sur[2] = {nullptr, nullptr};
    std::vector<int> use_sur;
    WorkItem* d_sur_items[2] = {nullptr, nullptr};
    uint32_t* d_sur_prefix[2] = {nullptr, nullptr};  // 256-history pairs before each surrogate item
    size_t sur_cap[2] = {0, 0};
    uint32_t n_sur_items[2] = {0, 0};
    uint32_t n_sur_pairs[2] = {0, 0};
    sur::SurExp* d_sexp = nullptr;
    unsigned long long* d_fallbacks = nullptr;
};

namespace {

void drop_graph(sas_batch* b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// Items of about cfg.target_item_flop each, longest first.
sas_status build_items(sas_batch* b)
{
    std::vector<WorkItem> items;
    std::vector<double> icost;
    const double target = b->cfg.target_item_flop > 0 ? b->cfg.target_item_flop : 2e9;
    std::vector<WorkItem> sitems[2];
    for (size_t e = 0; e < b->n_exp; ++e) {
        const uint64_t n = b->counts[e];
        if (n == 0) continue;
        if (!b->use_sur.empty() && b->use_sur[e]) {
            const uint64_t c = 1ull << 16;
            for (uint64_t f = 0; f < n; f += c) {
                WorkItem w;
                w.first = f;
                w.exp = (uint32_t)e;
                w.n = (uint32_t)std::min<uint64_t>(c, n - f);
                sitems[b->use_sur[e] - 1].push_back(w);
            }
            continue;
        }
        // at least four histories per thread of the CTA, in whole CTA passes,
        // so that every warp of the CTA has the same number of 32-history
        // batches even for the costly models (a 76 x 76 x 40 cylinder costs
        // 6.35 MFLOP per history, 315 histories per 2 GFLOP item)
        const double per_pass = (double)b->cfg.block;
        double chunk = std::floor(target / b->cost[e]);
        chunk = std::max(chunk, 4.0 * per_pass);
        chunk = std::ceil(chunk / per_pass) * per_pass;
        chunk = std::min(chunk, 1073741824.0);
        const uint64_t c = (uint64_t)chunk;
        for (uint64_t f = 0; f < n; f += c) {
            WorkItem w;
            w.first = f;
            w.exp = (uint32_t)e;
            w.n = (uint32_t)std::min<uint64_t>(c, n - f);
            items.push_back(w);
            icost.push_back(b->cost[e] * (double)w.n);
        }
    }
    std::vector<size_t> idx(items.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t c) { return icost[a] > icost[c]; });
    std::vector<WorkItem> sorted(items.size());
    for (size_t i = 0; i < idx.size(); ++i) sorted[i] = items[idx[i]];
    if (sorted.size() > 0xFFFFFFF0ull) return set_error(SAS_ERR_ARG, "too many work items");
    if (sorted.size() > b->items_cap) {
        cudaFree(b->d_items);
        b->d_items = nullptr;
        SAS_CUDA_B(cudaMalloc(&b->d_items, std::max<size_t>(sorted.size(), 1) * sizeof(WorkItem)), "cudaMalloc(items)");
        b->items_cap = sorted.size();
    }
    b->n_items = (uint32_t)sorted.size();
    if (!sorted.empty())
        SAS_CUDA_B(cudaMemcpy(b->d_items, sorted.data(), sorted.size() * sizeof(WorkItem), cudaMemcpyHostToDevice),
                   "upload items");
    for (int k = 0; k < 2; ++k) {
        const std::vector<WorkItem>& si = sitems[k];
        std::vector<uint32_t> sprefix;
        const uint64_t n_pairs = surrogate_pair_prefix(si, sprefix);
        if (n_pairs > 0xFFFFFFFFull) return set_error(SAS_ERR_ARG, "too many surrogate histories");
        if (si.size() > b->sur_cap[k]) {
            cudaFree(b->d_sur_items[k]);
            cudaFree(b->d_sur_prefix[k]);
            b->d_sur_items[k] = nullptr;
            b->d_sur_prefix[k] = nullptr;
            b->sur_cap[k] = 0;
            SAS_CUDA_B(cudaMalloc(&b->d_sur_items[k], si.size() * sizeof(WorkItem)), "cudaMalloc(items)");
            SAS_CUDA_B(cudaMalloc(&b->d_sur_prefix[k], si.size() * sizeof(uint32_t)), "cudaMalloc(items)");
            b->sur_cap[k] = si.size();
        }
        b->n_sur_items[k] = (uint32_t)si.size();
        b->n_sur_pairs[k] = (uint32_t)n_pairs;
        if (!si.empty()) {
            SAS_CUDA_B(cudaMemcpy(b->d_sur_items[k], si.data(), si.size() * sizeof(WorkItem), cudaMemcpyHostToDevice),
                       "upload items");
            SAS_CUDA_B(cudaMemcpy(b->d_sur_prefix[k], sprefix.data(), sprefix.size() * sizeof(uint32_t),
                                  cudaMemcpyHostToDevice),
                       "upload items");
        }
    }
    return SAS_OK;
}

// Per-experiment tally / staging choice and the kernel's shared memory.
sas_status plan(sas_batch* b)
{
    size_t smem = 0;
    int any_hist = 0;
    // the histogram kernel is built without these two kinds
    bool full = false;
    for (const sas_model_desc& m : b->models)
        full |= m.kind == SAS_ELLIPTICAL_CYLINDER || m.kind == SAS_HOLLOW_RECTANGULAR_PRISM;
    for (size_t e = 0; e < b->n_exp; ++e) {
        BatchExp& x = b->h_exps[e];
        x.use_hist = (b->cfg.use_hist && b->hist_capable[e] && !full) ? 1 : 0;
        x.stage_orient = (!x.use_hist && b->orient_stageable[e]) ? 1 : 0;
        size_t need = table_bytes<float>(x.mc.n_poly, x.mc.n_orient, x.stage_orient);
        if (x.use_hist) need = table_bytes<float>(x.mc.n_poly, 0, 0) + hist_bytes(b->npix);
        smem = std::max(smem, need);
        any_hist |= x.use_hist;
    }
    b->smem = smem;
    b->hist_ok = any_hist;
    SAS_CUDA_B(cudaMemcpy(b->d_exps, b->h_exps.data(), b->n_exp * sizeof(BatchExp), cudaMemcpyHostToDevice),
               "upload experiments");
    return SAS_OK;
}

sas_status capture(sas_batch* b)
{
    drop_graph(b);
    auto kern = b->hist_ok ? batch_kernel<1> : batch_kernel<0>;
    SAS_CUDA_B(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem),
               "cudaFuncSetAttribute");
    int per_sm = 0;
    SAS_CUDA_B(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, b->cfg.block, b->smem),
               "occupancy");
    if (per_sm < 1) return set_error(SAS_ERR_ARG, "batch launch shape does not fit on an SM");
    if (b->cfg.ctas_per_sm > 0 && b->cfg.ctas_per_sm < per_sm) per_sm = b->cfg.ctas_per_sm;
    b->grid = b->sm_count * per_sm;
    BatchParams P;
    std::memset(&P, 0, sizeof(P));
    P.in = b->icf;
    P.exps = b->d_exps;
    P.items = b->d_items;
    P.n_items = b->n_items;
    P.poly = b->d_poly;
    P.orient = b->d_orient;
    P.seed = b->d_seed;
    P.queue = b->d_queue;
    P.sum_w = b->d_sum_w;
    P.sum_w2 = b->d_sum_w2;
    P.count = b->d_count;
    P.trans = b->d_trans;
    P.npix = b->npix;
    const size_t det = b->n_exp * (size_t)b->npix;
    SAS_CUDA_B(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaMemsetAsync(b->d_sum_w, 0, det * sizeof(double), b->cap);
    cudaMemsetAsync(b->d_sum_w2, 0, det * sizeof(double), b->cap);
    cudaMemsetAsync(b->d_count, 0, det * sizeof(unsigned long long), b->cap);
    cudaMemsetAsync(b->d_trans, 0, b->n_exp * sizeof(double), b->cap);
    cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned int), b->cap);
    if (b->n_items > 0) kern<<<b->grid, b->cfg.block, b->smem, b->cap>>>(P);
    cudaError_t le = cudaGetLastError();
    for (int k = 0; k < 2; ++k) {
        if (le != cudaSuccess || !b->sur[k] || b->n_sur_items[k] == 0) continue;
        sur::STParams S;
        std::memset(&S, 0, sizeof(S));
        S.in = b->icf;
        S.box = surrogate_dbox(b->sur[k]);
        S.epi = surrogate_epi(b->sur[k]);
        S.seed = b->d_seed;
        S.philox_base = 0;
        S.items = b->d_sur_items[k];
        S.pair_prefix = b->d_sur_prefix[k];
        S.n_items = b->n_sur_items[k];
        S.n_pairs = b->n_sur_pairs[k];
        S.sexp = b->d_sexp;
        S.bexp = b->d_exps;
        S.poly = b->d_poly;
        S.orient = b->d_orient;
        S.sum_w = b->d_sum_w;
        S.sum_w2 = b->d_sum_w2;
        S.count = b->d_count;
        S.trans = b->d_trans;
        S.npix = b->npix;
        S.fallbacks = b->d_fallbacks;
        S.err = surrogate_err(b->sur[k]);
        le = launch_sur_trace(b->sur[k], S, b->sm_count, b->cap);
    }
    cudaError_t ce = cudaStreamEndCapture(b->cap, &b->graph);
    if (le != cudaSuccess) return set_cuda_error(le, "batch kernel launch (capture)");
    if (ce != cudaSuccess) return set_cuda_error(ce, "end capture");
    SAS_CUDA_B(cudaGraphInstantiate(&b->exec, b->graph, 0), "graph instantiate");
    return SAS_OK;
}

}  // namespace

extern "C" {

sas_status sas_create_batch(const sas_instrument* inst, const sas_model_desc* models, const uint64_t* counts,
                            size_t n_exp, void* stream, sas_batch** out)
{
    if (!out) return set_error(SAS_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!models || !counts || n_exp == 0) return set_error(SAS_ERR_ARG, "empty batch");
    if (n_exp > 0x7FFFFFFFull) return set_error(SAS_ERR_ARG, "too many experiments");
    sas_status st = validate_instrument(inst);
    if (st != SAS_OK) return st;
    sas_batch* b = new (std::nothrow) sas_batch();
    if (!b) return set_error(SAS_ERR_OOM, "host allocation failed");
    b->inst = *inst;
    b->icf = inst_const<float>(*inst);
    b->stream = (cudaStream_t)stream;
    b->n_exp = n_exp;
    b->npix = (int)(inst->nx * inst->ny);
    b->counts.assign(counts, counts + n_exp);
    b->cfg.block = 1024;   // 32 warps per SM with the one-CTA histogram layout
    b->cfg.ctas_per_sm = 0;
    b->cfg.use_hist = 1;
    b->cfg.reserved = 0;
    b->cfg.target_item_flop = 2e9;
    auto bail = [&](sas_status s) { sas_destroy_batch(b); return s; };
    cudaError_t ce = cudaGetDevice(&b->device);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device);
    if (ce == cudaSuccess)
        ce = cudaDeviceGetAttribute(&b->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device);
    if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (ce != cudaSuccess) return bail(set_cuda_error(ce, "sas_create_batch"));
    std::vector<float> poly, orient;
    std::vector<std::pair<size_t, ModelTables>> att_exps;   // experiments with self-attenuation
    b->h_exps.resize(n_exp);
    b->cost.resize(n_exp);
    b->hist_capable.resize(n_exp);
    b->orient_stageable.resize(n_exp);
    for (size_t e = 0; e < n_exp; ++e) {
        const sas_model_desc& m = models[e];
        st = validate_model(&m);
        if (st != SAS_OK) return bail(st);
        if (m.precision != SAS_FP32) return bail(set_error(SAS_ERR_ARG, "batched experiments are FP32"));
        if (m.kind == SAS_SHAPE_INDEPENDENT)
            return bail(set_error(SAS_ERR_ARG, "shape-independent laws are traced one by one (sas_trace), not batched"));
        if (m.sq_kind == SAS_SQ_HAYTER_MSA)
            return bail(set_error(SAS_ERR_ARG, "the Hayter MSA S(Q) is traced one by one (sas_trace), not batched"));
        ModelTables t;
        st = build_model_tables(m, t, instrument_q_max(*inst));
        if (st != SAS_OK) return bail(st);
        BatchExp& x = b->h_exps[e];
        std::memset(&x, 0, sizeof(x));
        x.mc = model_const<float>(m, t);
        x.poly_off = (uint32_t)poly.size();
        x.orient_off = (uint32_t)orient.size();
        for (double v : t.poly) poly.push_back((float)v);
        for (double v : t.orient) orient.push_back((float)v);
        if (poly.size() > 0xFFFFFFF0ull || orient.size() > 0xFFFFFFF0ull)
            return bail(set_error(SAS_ERR_ARG, "batch tables too large"));
        b->cost[e] = host_flops_per_history(m, t.n_poly, std::max(t.n_orient, 1));
        b->hist_capable[e] = (t.n_orient <= 1) &&
                             (table_bytes<float>(t.n_poly, 0, 0) + hist_bytes(b->npix) <= (size_t)b->smem_optin);
        b->orient_stageable[e] = (t.n_orient > 1) &&
                                 (table_bytes<float>(t.n_poly, t.n_orient, 1) <= (size_t)b->smem_optin);
        b->total_histories += counts[e];
        b->models.push_back(m);
        if (m.self_attenuation) att_exps.emplace_back(e, t);
    }
    const size_t det = n_exp * (size_t)b->npix;
    ce = cudaMalloc(&b->d_exps, n_exp * sizeof(BatchExp));
    if (ce == cudaSuccess) ce = cudaMalloc(&b->d_poly, std::max<size_t>(poly.size(), 1) * sizeof(float));
    if (ce == cudaSuccess) ce = cudaMalloc(&b->d_orient, std::max<size_t>(orient.size(), 1) * sizeof(float));
    if (ce == cudaSuccess) ce = cudaMalloc(&b->d_seed, sizeof(uint64_t));
    if (ce == cudaSuccess) ce = cudaMalloc(&b->d_queue, sizeof(unsigned int));
    if (ce == cudaSuccess) ce = cudaMalloc(&b->d_sum_w, det * sizeof(double));
    if (ce == cudaSuccess) ce = cudaMalloc(&b->d_sum_w2, det * sizeof(double));
    if (ce == cudaSuccess) ce = cudaMalloc(&b->d_count, det * sizeof(unsigned long long));
    if (ce == cudaSuccess) ce = cudaMalloc(&b->d_trans, n_exp * sizeof(double));
    if (ce == cudaSuccess && !poly.empty())
        ce = cudaMemcpy(b->d_poly, poly.data(), poly.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess && !orient.empty())
        ce = cudaMemcpy(b->d_orient, orient.data(), orient.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) return bail(set_cuda_error(ce, "sas_create_batch allocation"));
    // self-attenuation tables, from each experiment's tables now on the device
    for (auto& ea : att_exps) {
        const size_t e = ea.first;
        ModelTables& t = ea.second;
        AttRule r;
        att_rule(*inst, models[e], t, r);
        double mu[SAS_ATT_MAX];
        ce = att_nodes(models[e], t, (const float*)b->d_poly + b->h_exps[e].poly_off,
                       (const float*)b->d_orient + b->h_exps[e].orient_off, r, b->stream, mu);
        if (ce != cudaSuccess) return bail(set_cuda_error(ce, "self-attenuation table"));
        for (int j = 0; j < r.n_lambda; ++j)
            if (!std::isfinite(mu[j]) || mu[j] < 0.0)
                return bail(set_error(SAS_ERR_NUMERIC, "self-attenuation: non-finite or negative cross section"));
        att_fit(r, mu, t);
        b->h_exps[e].mc.att = model_const<float>(models[e], t).att;
    }
    st = plan(b);
    if (st == SAS_OK) st = build_items(b);
    if (st != SAS_OK) return bail(st);
    *out = b;
    return SAS_OK;
}

sas_status sas_batch_set_config(sas_batch* b, const sas_batch_config* cfg)
{
    if (!b || !cfg) return set_error(SAS_ERR_ARG, "NULL argument");
    if (cfg->block < 32 || cfg->block > 1024 || cfg->block % 32 != 0)
        return set_error(SAS_ERR_ARG, "block must be a multiple of 32 in [32, 1024]");
    if (cfg->ctas_per_sm < 0 || !(cfg->target_item_flop >= 0.0))
        return set_error(SAS_ERR_ARG, "bad batch config");
    SAS_CUDA_B(cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
    b->cfg = *cfg;
    drop_graph(b);
    sas_status st = plan(b);
    if (st == SAS_OK) st = build_items(b);
    return st;
}

sas_status sas_batch_get_config(const sas_batch* b, sas_batch_config* cfg)
{
    if (!b || !cfg) return set_error(SAS_ERR_ARG, "NULL argument");
    *cfg = b->cfg;
    return SAS_OK;
}

sas_status sas_batch_info(const sas_batch* b, uint32_t* n_items, int* grid, size_t* smem,
                          uint64_t* total_histories)
{
    if (!b) return set_error(SAS_ERR_ARG, "batch is NULL");
    if (n_items) *n_items = b->n_items;
    if (grid) *grid = b->grid;
    if (smem) *smem = b->smem;
    if (total_histories) *total_histories = b->total_histories;
    return SAS_OK;
}

sas_status sas_trace_batch(sas_batch* b, uint64_t seed)
{
    if (!b) return set_error(SAS_ERR_ARG, "batch is NULL");
    if (!b->exec) {
        sas_status st = capture(b);
        if (st != SAS_OK) return st;
    }
    SAS_CUDA_B(cudaMemcpyAsync(b->d_seed, &seed, sizeof(seed), cudaMemcpyHostToDevice, b->stream), "seed upload");
    SAS_CUDA_B(cudaGraphLaunch(b->exec, b->stream), "cudaGraphLaunch");
    return SAS_OK;
}

sas_status sas_read_batch_detector(const sas_batch* b, size_t exp, double* sum_w, double* sum_w2,
                                   uint64_t* count, size_t n_pixels, double* transmitted)
{
    if (!b) return set_error(SAS_ERR_ARG, "batch is NULL");
    if (exp >= b->n_exp) return set_error(SAS_ERR_ARG, "experiment index out of range");
    if ((sum_w || sum_w2 || count) && n_pixels != (size_t)b->npix)
        return set_error(SAS_ERR_ARG, "n_pixels does not match nx*ny");
    const size_t off = exp * (size_t)b->npix, bytes = (size_t)b->npix * 8;
    if (sum_w) SAS_CUDA_B(cudaMemcpyAsync(sum_w, b->d_sum_w + off, bytes, cudaMemcpyDeviceToHost, b->stream), "read");
    if (sum_w2) SAS_CUDA_B(cudaMemcpyAsync(sum_w2, b->d_sum_w2 + off, bytes, cudaMemcpyDeviceToHost, b->stream), "read");
    if (count) SAS_CUDA_B(cudaMemcpyAsync(count, b->d_count + off, bytes, cudaMemcpyDeviceToHost, b->stream), "read");
    if (transmitted)
        SAS_CUDA_B(cudaMemcpyAsync(transmitted, b->d_trans + exp, 8, cudaMemcpyDeviceToHost, b->stream), "read");
    SAS_CUDA_B(cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
    for (int k = 0; k < 2; ++k)
        if (b->sur[k]) {
            const sas_status st = surrogate_take_error(b->sur[k], b->stream);
            if (st != SAS_OK) return st;
        }
    return SAS_OK;
}

sas_status sas_batch_detector_device(const sas_batch* b, const double** sum_w, const double** sum_w2,
                                     const uint64_t** count, const double** transmitted)
{
    if (!b) return set_error(SAS_ERR_ARG, "batch is NULL");
    if (sum_w) *sum_w = b->d_sum_w;
    if (sum_w2) *sum_w2 = b->d_sum_w2;
    if (count) *count = (const uint64_t*)b->d_count;
    if (transmitted) *transmitted = b->d_trans;
    return SAS_OK;
}

// Time every candidate launch shape / item size on this batch (one traced
// batch each, CUDA events on the batch's stream) and keep the fastest.
sas_status sas_batch_autotune(sas_batch* b, uint64_t seed, sas_batch_config* best_out, double* best_ms)
{
    if (!b) return set_error(SAS_ERR_ARG, "batch is NULL");
    const int blocks[] = {256, 512, 1024};
    const double targets[] = {5e8, 2e9, 8e9};
    const int hists[] = {1, 0};
    cudaEvent_t e0, e1;
    SAS_CUDA_B(cudaEventCreate(&e0), "event");
    SAS_CUDA_B(cudaEventCreate(&e1), "event");
    sas_batch_config best = b->cfg;
    float best_t = 1e30f;
    sas_status st = SAS_OK;
    for (int hb : hists) {
        for (int blk : blocks) {
            for (double tg : targets) {
                sas_batch_config c = b->cfg;
                c.block = blk;
                c.target_item_flop = tg;
                c.use_hist = hb;
                c.ctas_per_sm = 0;
                st = sas_batch_set_config(b, &c);
                if (st != SAS_OK) continue;   // shape does not fit: skip it
                st = sas_trace_batch(b, seed);   // warm-up + capture
                if (st != SAS_OK) continue;
                cudaEventRecord(e0, b->stream);
                st = sas_trace_batch(b, seed);
                cudaEventRecord(e1, b->stream);
                if (cudaEventSynchronize(e1) != cudaSuccess || st != SAS_OK) continue;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best_t) {
                    best_t = ms;
                    best = c;
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_t >= 1e30f) return set_error(SAS_ERR_CUDA, "no batch launch shape ran");
    st = sas_batch_set_config(b, &best);
    if (st != SAS_OK) return st;
    if (best_out) *best_out = best;
    if (best_ms) *best_ms = best_t;
    return SAS_OK;
}

sas_status sas_batch_attach_surrogate(sas_batch* b, const sas_surrogate* s)
{
    if (!b) return set_error(SAS_ERR_ARG, "batch is NULL");
    SAS_CUDA_B(cudaStreamSynchronize(b->stream), "sync");
    drop_graph(b);
    if (s) b->sur[surrogate_kind(s) == SAS_ELLIPSOID ? 1 : 0] = s;
    else b->sur[0] = b->sur[1] = nullptr;
    b->use_sur.assign(b->n_exp, 0);
    if (b->sur[0] || b->sur[1]) {
        std::vector<sur::SurExp> se(b->n_exp);
        for (size_t e = 0; e < b->n_exp; ++e) {
            for (int k = 0; k < 2 && !b->use_sur[e]; ++k)
                if (surrogate_covers(b->sur[k], b->models[e])) b->use_sur[e] = k + 1;
            se[e] = surrogate_exp(b->models[e], b->use_sur[e] != 0);
        }
        if (!b->d_sexp) {
            SAS_CUDA_B(cudaMalloc(&b->d_sexp, b->n_exp * sizeof(sur::SurExp)), "alloc");
            SAS_CUDA_B(cudaMalloc(&b->d_fallbacks, sizeof(unsigned long long)), "alloc");
        }
        SAS_CUDA_B(cudaMemset(b->d_fallbacks, 0, sizeof(unsigned long long)), "memset");
        SAS_CUDA_B(cudaMemcpy(b->d_sexp, se.data(), b->n_exp * sizeof(sur::SurExp), cudaMemcpyHostToDevice),
                   "upload");
    }
    return build_items(b);
}

sas_status sas_batch_surrogate_share(const sas_batch* b, uint64_t* experiments, uint64_t* histories)
{
    if (!b) return set_error(SAS_ERR_ARG, "batch is NULL");
    uint64_t ne = 0, nh = 0;
    for (size_t e = 0; e < b->use_sur.size(); ++e)
        if (b->use_sur[e]) {
            ++ne;
            nh += b->counts[e];
        }
    if (experiments) *experiments = ne;
    if (histories) *histories = nh;
    return SAS_OK;
}

sas_status sas_surrogate_fallbacks(const sas_experiment* e, const sas_batch* b, uint64_t* count)
{
    if (!count) return set_error(SAS_ERR_ARG, "NULL argument");
    *count = 0;
    unsigned long long v = 0;
    if (e && experiment_fallback_counter(e)) {
        SAS_CUDA_B(cudaMemcpyAsync(&v, experiment_fallback_counter(e), 8, cudaMemcpyDeviceToHost,
                                   experiment_stream(e)), "read");
        SAS_CUDA_B(cudaStreamSynchronize(experiment_stream(e)), "sync");
        *count += v;
    }
    if (b && b->d_fallbacks) {
        SAS_CUDA_B(cudaMemcpyAsync(&v, b->d_fallbacks, 8, cudaMemcpyDeviceToHost, b->stream), "read");
        SAS_CUDA_B(cudaStreamSynchronize(b->stream), "sync");
        *count += v;
    }
    return SAS_OK;
}

sas_status sas_destroy_batch(sas_batch* b)
{
    if (!b) return SAS_OK;
    cudaStreamSynchronize(b->stream);
    if (b->cap) cudaStreamSynchronize(b->cap);
    drop_graph(b);
    cudaFree(b->d_exps);
    cudaFree(b->d_items);
    cudaFree(b->d_poly);
    cudaFree(b->d_orient);
    cudaFree(b->d_seed);
    cudaFree(b->d_queue);
    cudaFree(b->d_sum_w);
    cudaFree(b->d_sum_w2);
    cudaFree(b->d_count);
    cudaFree(b->d_trans);
    for (int k = 0; k < 2; ++k) {
        cudaFree(b->d_sur_items[k]);
        cudaFree(b->d_sur_prefix[k]);
    }
    cudaFree(b->d_sexp);
    cudaFree(b->d_fallbacks);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return SAS_OK;
}

}  // extern "C"
