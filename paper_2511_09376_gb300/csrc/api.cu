// C ABI of the library (declared in include/woodelf.h): context and ensemble
// lifetime, argument checks, device buffers, and the order of the kernel launches of
// Algorithm 3.  No kernel here; every step runs in the kernels of k_*.cu.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "launch.h"
#include "wdf_internal.h"
#include "woodelf.h"

namespace {

thread_local std::string g_err;

wdf_status fail(wdf_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

wdf_status cuda_fail(cudaError_t e, const char *where) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(WDF_ENOMEM, std::string(where) + ": " + cudaGetErrorString(e));
    }
    return fail(WDF_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define WDF_CUDA(call)                                     \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// Makes the context's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

template <typename T>
cudaError_t dalloc(T **p, size_t count, int64_t *bytes) {
    *p = nullptr;
    if (count == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e == cudaSuccess) *bytes += (int64_t)(count * sizeof(T));
    return e;
}

template <typename T>
void dfree(T *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

constexpr int64_t kStageRows = 1 << 19;  // rows per host<->device staging chunk

std::atomic<int64_t> g_launches{0};

}  // namespace

namespace wdf {
void count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
void set_last_error(const std::string &msg) { g_err = msg; }
TraceRange::TraceRange(const char *name) { nvtxRangePushA(name); }
TraceRange::~TraceRange() { nvtxRangePop(); }
}  // namespace wdf

#include "wdf_objects.h"

namespace {

void free_ensemble(wdf_ensemble *e) {
    dfree(e->d_nodes); dfree(e->d_keys); dfree(e->d_group_leaf); dfree(e->d_leaf_row);
    dfree(e->d_w_rows); dfree(e->d_tiles); dfree(e->d_t32);
    dfree(e->d_rec); dfree(e->d_meta); dfree(e->d_flfeat); dfree(e->d_xmask); dfree(e->d_cols); dfree(e->d_col_thr);
    dfree(e->d_apk); dfree(e->d_bpk); dfree(e->d_tiles128); dfree(e->d_err); dfree(e->d_A); dfree(e->d_ratio);
    dfree(e->d_hist); dfree(e->d_vc); dfree(e->d_scale); dfree(e->d_S); dfree(e->d_sfold); dfree(e->d_base);
    dfree(e->d_lines);
    for (int i = 0; i < 2; ++i) {
        dfree(e->d_codes[i]);
        dfree(e->d_stage_in[i]);
        dfree(e->d_stage_out[i]);
        if (e->ist[i]) cudaStreamDestroy(e->ist[i]);
        if (e->ev_join[i]) cudaEventDestroy(e->ev_join[i]);
        if (e->ev_enc[i]) cudaEventDestroy(e->ev_enc[i]);
        if (e->ev_cnt[i]) cudaEventDestroy(e->ev_cnt[i]);
        e->ist[i] = nullptr;
        e->ev_join[i] = nullptr;
        e->ev_enc[i] = e->ev_cnt[i] = nullptr;
    }
    if (e->ev_fork) cudaEventDestroy(e->ev_fork);
    e->ev_fork = nullptr;
}

// Double-buffered staging for host-memory calls: chunk i of the rows goes through
// buffer i % 2 on internal stream i % 2, so the copy engines of one chunk overlap the
// kernels of the other.  Grows to the largest chunk seen (at most kStageRows rows).
wdf_status ensure_streams(wdf_ensemble *e) {
    if (!e->ist[0]) {
        for (int i = 0; i < 2; ++i) {
            WDF_CUDA(cudaStreamCreateWithFlags(&e->ist[i], cudaStreamNonBlocking));
            WDF_CUDA(cudaEventCreateWithFlags(&e->ev_join[i], cudaEventDisableTiming));
            WDF_CUDA(cudaEventCreateWithFlags(&e->ev_enc[i], cudaEventDisableTiming));
            WDF_CUDA(cudaEventCreateWithFlags(&e->ev_cnt[i], cudaEventDisableTiming));
        }
        WDF_CUDA(cudaEventCreateWithFlags(&e->ev_fork, cudaEventDisableTiming));
    }
    return WDF_OK;
}

wdf_status ensure_staging(wdf_ensemble *e, int64_t rows, bool out) {
    rows = std::min(rows, kStageRows);
    wdf_status s0 = ensure_streams(e);
    if (s0 != WDF_OK) return s0;
    if (rows > e->stage_rows) {
        WDF_CUDA(cudaDeviceSynchronize());
        for (int i = 0; i < 2; ++i) {
            dfree(e->d_stage_in[i]);
            dfree(e->d_stage_out[i]);
        }
        e->stage_rows = 0;
        const size_t n = (size_t)rows * e->pk.F;
        for (int i = 0; i < 2; ++i) {
            WDF_CUDA(dalloc(&e->d_stage_in[i], n, &e->bytes));
            WDF_CUDA(dalloc(&e->d_stage_out[i], n, &e->bytes));
        }
        e->stage_rows = rows;
    }
    (void)out;
    return WDF_OK;
}

// Decision-code buffers for background chunks of up to `rows` rows (at most kCodeRows,
// a multiple of the largest background tile), nbuf of them.
constexpr int64_t kCodeRows = 1 << 20;
wdf_status ensure_codes(wdf_ensemble *e, int64_t rows, int nbuf) {
    const int64_t tile = wdf::kBgMaxTileRows;
    rows = std::min((rows + tile - 1) / tile * tile, kCodeRows);
    const size_t xb = e->pk.cols.size() * (size_t)e->pk.code_bytes;
    if (rows > e->code_rows) {
        WDF_CUDA(cudaDeviceSynchronize());
        for (int i = 0; i < 2; ++i) dfree(e->d_codes[i]);
        e->code_rows = rows;
    }
    for (int i = 0; i < nbuf; ++i)
        if (!e->d_codes[i]) WDF_CUDA(dalloc(&e->d_codes[i], (size_t)e->code_rows * xb, &e->bytes));
    return WDF_OK;
}

// Counts of device rows B (m rows) added into hist: with more than one chunk of codes,
// the encode of the next chunk overlaps the count of this one (two code buffers, the
// side stream ist[0]).
wdf_status count_device_rows(wdf_ensemble *ens, const float *B, int64_t m, int64_t ldb, uint32_t *hist,
                             cudaStream_t st) {
    const wdf::Packed &p = ens->pk;
    const bool overlap = m > kCodeRows;
    wdf_status s = ensure_codes(ens, m, overlap ? 2 : 1);
    if (s == WDF_OK && overlap) s = ensure_streams(ens);
    if (s != WDF_OK) return s;
    wdf::BgOverlap ov{ens->d_codes[1], ens->ist[0], {ens->ev_enc[0], ens->ev_enc[1]}, {ens->ev_cnt[0], ens->ev_cnt[1]}};
    WDF_CUDA(wdf::launch_bg_hist(p.D, B, m, ldb, ens->arrays(), p.T, ens->d_codes[0], ens->code_rows, hist,
                                 ens->ctx->dev, st, overlap ? &ov : nullptr));
    return WDF_OK;
}

// Split operand stages, 128-row tiles and the error flag for the tensor-core
// contraction in split mode `mode`: the tiles, the flag and the A stages (room for any
// mode) once, the B stages (the tables split for this mode) whenever the mode changes.
wdf_status ensure_tensor_core_state(wdf_ensemble *e, int mode) {
    const wdf::Packed &p = e->pk;
    if (!e->d_tiles128) {
        std::vector<int4> tiles;
        for (int gi = 0; gi < e->G; ++gi)
            for (int r0 = p.group_off[(size_t)gi]; r0 < p.group_off[(size_t)gi + 1]; r0 += 128)
                tiles.push_back(make_int4(gi, r0, std::min(r0 + 128, p.group_off[(size_t)gi + 1]), 0));
        WDF_CUDA(dalloc(&e->d_tiles128, std::max<size_t>(tiles.size(), 1), &e->bytes));
        WDF_CUDA(dalloc(&e->d_err, 1, &e->bytes));
        WDF_CUDA(cudaMemset(e->d_err, 0, sizeof(int)));
        if (!tiles.empty())
            WDF_CUDA(cudaMemcpy(e->d_tiles128, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice));
        e->n_tiles128 = (int)tiles.size();
        WDF_CUDA(dalloc(&e->d_apk, std::max<size_t>(wdf::contract_tc_a_bytes(p.D, e->n_tiles128), 16), &e->bytes));
    }
    if (e->bpk_mode != mode) {
        if (e->d_bpk) {
            WDF_CUDA(cudaDeviceSynchronize());  // an earlier contraction may still read it
            e->bytes -= (int64_t)wdf::contract_tc_b_bytes(p.D, e->bpk_mode, e->G);
            dfree(e->d_bpk);
        }
        e->bpk_mode = -1;
        WDF_CUDA(dalloc(&e->d_bpk, std::max<size_t>(wdf::contract_tc_b_bytes(p.D, mode, e->G), 16), &e->bytes));
        WDF_CUDA(wdf::launch_pack_b(p.D, mode, e->d_t32, e->G, e->d_bpk, 0));
        WDF_CUDA(cudaStreamSynchronize(0));
        e->bpk_mode = mode;
    }
    return WDF_OK;
}

// Copy `rows` rows of F floats between a strided host matrix and a packed device one.
cudaError_t copy_rows(float *dst, int64_t ldd, const float *src, int64_t lds, int64_t rows, int F,
                      cudaMemcpyKind kind, cudaStream_t st) {
    if (ldd == F && lds == F) return cudaMemcpyAsync(dst, src, (size_t)rows * F * 4, kind, st);
    return cudaMemcpy2DAsync(dst, (size_t)ldd * 4, src, (size_t)lds * 4, (size_t)F * 4, (size_t)rows, kind, st);
}

bool valid_precision(wdf_precision p) {
    return p == WDF_FP32 || p == WDF_TF32X3 || p == WDF_BF16X3 || p == WDF_BF16X6;
}

// The tensor-core kernel's operand split: 0 = TF32 two parts, 1 = BF16 two, 2 = BF16 three.
int tc_mode(wdf_precision p) { return p == WDF_TF32X3 ? 0 : (p == WDF_BF16X3 ? 1 : 2); }

// Buffers of the consumer-independent half (counts, frequencies, S, folded vectors) and,
// for the tensor-core precisions, the K-major tables.
wdf_status ensure_frequency_state(wdf_ensemble *ens, wdf_precision precision) {
    const wdf::Packed &p = ens->pk;
    const int K = 1 << p.D, N = p.D << p.D;
    const size_t hist_n = (size_t)p.T * p.NS * (2 * K);
    if (!ens->d_hist) {
        WDF_CUDA(dalloc(&ens->d_hist, hist_n, &ens->bytes));
        WDF_CUDA(dalloc(&ens->d_vc, (size_t)ens->n_live * K, &ens->bytes));
        WDF_CUDA(dalloc(&ens->d_A, (size_t)ens->n_live * K, &ens->bytes));
        WDF_CUDA(dalloc(&ens->d_scale, (size_t)ens->n_live, &ens->bytes));
        WDF_CUDA(dalloc(&ens->d_S, (size_t)ens->n_live * N, &ens->bytes));
        WDF_CUDA(dalloc(&ens->d_sfold, hist_n * wdf::slots_per_entry(p.D), &ens->bytes));
        WDF_CUDA(dalloc(&ens->d_lines, (size_t)p.T * wdf::lines_words(p.D), &ens->bytes));
        WDF_CUDA(dalloc(&ens->d_base, 1, &ens->bytes));
    }
    ens->has_bg = 0;
    if (precision != WDF_FP32) return ensure_tensor_core_state(ens, tc_mode(precision));
    return WDF_OK;
}

// Step 3 of Algorithm 3 (S = w * M * f for every live leaf, from the frequencies in d_A
// and the per-leaf scale) in the requested precision, then the fold of every bottom
// subtree into the vectors the consumer kernel gathers.
wdf_status contract_and_fold(wdf_ensemble *ens, wdf_precision precision, cudaStream_t st) {
    const wdf::Packed &p = ens->pk;
    if (precision == WDF_FP32) {
        WDF_CUDA(wdf::launch_contract_fp32(p.D, ens->d_A, ens->d_scale, ens->d_tiles, ens->n_tiles, ens->d_t32,
                                           ens->d_S, st));
    } else {
        // the flag may hold an expiry of an earlier call: clear it first
        WDF_CUDA(cudaMemsetAsync(ens->d_err, 0, sizeof(int), st));
        WDF_CUDA(wdf::launch_contract_tc(p.D, tc_mode(precision), ens->d_A, ens->d_scale, ens->d_tiles128,
                                         ens->n_tiles128, ens->d_apk, ens->d_bpk, ens->d_S, ens->d_err, st));
        // a bounded wait inside the kernel that expired is reported here
        int flag = 0;
        WDF_CUDA(cudaMemcpyAsync(&flag, ens->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
        WDF_CUDA(cudaStreamSynchronize(st));
        if (flag) return fail(WDF_ETIMEOUT, "tensor-core contraction: an mbarrier wait expired");
    }
    WDF_CUDA(wdf::launch_fold(p.D, ens->d_S, ens->d_leaf_row, p.T, ens->d_lines, ens->d_sfold, st));
    return WDF_OK;
}

// Steps 2-3 of Algorithm 3 after the joint counts are in d_hist: per-leaf counts (and
// the FP32 frequency operand), scales w_l / m, E_b f(b), contraction and fold.
wdf_status finish_background(wdf_ensemble *ens, int64_t m, wdf_precision precision, cudaStream_t st) {
    const wdf::Packed &p = ens->pk;
    WDF_CUDA(wdf::launch_leaf_counts(p.D, ens->d_hist, ens->d_group_leaf, ens->n_live, ens->d_vc, ens->d_A, st));
    WDF_CUDA(wdf::launch_scale(ens->d_w_rows, ens->n_live, m, ens->d_scale, st));
    WDF_CUDA(wdf::launch_base_value(p.D, ens->d_vc, nullptr, ens->d_w_rows, ens->n_live, m, ens->d_base, st));
    WDF_CUDA(wdf::launch_line_maps(p.D, ens->d_hist, p.T, ens->d_lines, st));
    wdf_status s1 = contract_and_fold(ens, precision, st);
    if (s1 != WDF_OK) return s1;
    ens->m = m;
    ens->pd = 0;
    ens->has_bg = 1;
    return WDF_OK;
}

}  // namespace

extern "C" {

const char *wdf_last_error(void) { return g_err.c_str(); }

const char *wdf_version(void) { return "woodelf-gb300 0.2 (sm_103a)"; }

void wdf_debug_contract_wait_limit(int32_t polls) { wdf::set_contract_first_wait_limit(polls > 0 ? (uint32_t)polls : 0u); }

int64_t wdf_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

wdf_status wdf_explain_timing(int32_t enable) {
    wdf::explain_timing(enable != 0);
    return WDF_OK;
}

wdf_status wdf_explain_timing_read(double *ms, int64_t *launches) {
    if (!ms || !launches) return fail(WDF_EINVAL, "null output");
    const cudaError_t e = wdf::explain_timing_read(ms, launches);
    if (e != cudaSuccess) return cuda_fail(e, "wdf_explain_timing_read");
    return WDF_OK;
}

wdf_status wdf_ctx_create(int32_t device, wdf_ctx **out) {
    if (!out) return fail(WDF_EINVAL, "out is null");
    *out = nullptr;
    int count = 0;
    WDF_CUDA(cudaGetDeviceCount(&count));
    if (device < 0 || device >= count) return fail(WDF_EINVAL, "device index out of range");
    DeviceGuard g(device);
    if (!g.ok) return fail(WDF_ECUDA, "cudaSetDevice failed");
    wdf_ctx *c = new wdf_ctx();
    c->device = device;
    int sms = 0, smem = 0;
    cudaError_t e1 = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaError_t e2 = cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
        delete c;
        return cuda_fail(e1 != cudaSuccess ? e1 : e2, "cudaDeviceGetAttribute");
    }
    c->dev.sms = sms;
    c->dev.smem_optin = (size_t)smem;
    *out = c;
    return WDF_OK;
}

void wdf_ctx_destroy(wdf_ctx *ctx) { ctx_release(ctx); }

wdf_status wdf_load_ensemble(wdf_ctx *ctx, int32_t n_features, int32_t n_trees, const int64_t *tree_offset,
                             const int32_t *feature, const float *threshold, const int32_t *left,
                             const int32_t *right, const float *value, wdf_ensemble **out) {
    wdf::TraceRange trace_("wdf_load_ensemble");
    if (!ctx || !out) return fail(WDF_EINVAL, "ctx and out must be non-null");
    *out = nullptr;
    wdf_ensemble *e = new wdf_ensemble();
    e->ctx = ctx_retain(ctx);
    std::string err;
    const int rc = wdf::pack_ensemble(n_features, n_trees, tree_offset, feature, threshold, left, right, value,
                                      &e->pk, &err);
    if (rc != 0) {
        delete e;
        ctx_release(ctx);
        return fail((wdf_status)rc, err);
    }
    DeviceGuard g(ctx->device);
    const wdf::Packed &p = e->pk;
    e->G = (int)p.sig_key.size();
    e->n_live = (int)p.group_leaf.size();
    std::vector<int2> nodes((size_t)p.T * p.NI);
    for (size_t i = 0; i < nodes.size(); ++i) {
        int32_t bits;
        std::memcpy(&bits, &p.node_thr[i], 4);
        nodes[i] = make_int2(p.node_feat[i], bits);
    }
    std::vector<double> w_rows((size_t)e->n_live);
    for (int r = 0; r < e->n_live; ++r) w_rows[(size_t)r] = (double)p.leaf_w[(size_t)p.group_leaf[(size_t)r]];
    std::vector<int4> tiles;
    for (int gi = 0; gi < e->G; ++gi)
        for (int r0 = p.group_off[(size_t)gi]; r0 < p.group_off[(size_t)gi + 1]; r0 += 64)
            tiles.push_back(make_int4(gi, r0, std::min(r0 + 64, p.group_off[(size_t)gi + 1]), 0));
    e->n_tiles = (int)tiles.size();
    const int K = 1 << p.D, N = p.D << p.D;
    cudaError_t ce = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (ce == cudaSuccess) ce = x; };
    chk(dalloc(&e->d_nodes, nodes.size(), &e->bytes));
    chk(dalloc(&e->d_keys, p.sig_key.size(), &e->bytes));
    chk(dalloc(&e->d_group_leaf, p.group_leaf.size(), &e->bytes));
    chk(dalloc(&e->d_leaf_row, p.leaf_row.size(), &e->bytes));
    chk(dalloc(&e->d_w_rows, w_rows.size(), &e->bytes));
    chk(dalloc(&e->d_tiles, tiles.size(), &e->bytes));
    chk(dalloc(&e->d_t32, (size_t)e->G * K * N, &e->bytes));
    chk(dalloc(&e->d_rec, p.rec.size(), &e->bytes));
    chk(dalloc(&e->d_meta, p.meta.size(), &e->bytes));
    chk(dalloc(&e->d_flfeat, p.flush_feat.size(), &e->bytes));
    if (!p.xmask.empty()) chk(dalloc(&e->d_xmask, p.xmask.size(), &e->bytes));
    chk(dalloc(&e->d_cols, p.cols.size(), &e->bytes));
    chk(dalloc(&e->d_col_thr, std::max<size_t>(p.col_thr.size(), 1), &e->bytes));
    if (ce == cudaSuccess) {
        chk(cudaMemcpy(e->d_nodes, nodes.data(), nodes.size() * sizeof(int2), cudaMemcpyHostToDevice));
        if (e->G) chk(cudaMemcpy(e->d_keys, p.sig_key.data(), p.sig_key.size() * 4, cudaMemcpyHostToDevice));
        if (e->n_live) {
            chk(cudaMemcpy(e->d_group_leaf, p.group_leaf.data(), p.group_leaf.size() * 4, cudaMemcpyHostToDevice));
            chk(cudaMemcpy(e->d_w_rows, w_rows.data(), w_rows.size() * 8, cudaMemcpyHostToDevice));
        }
        chk(cudaMemcpy(e->d_leaf_row, p.leaf_row.data(), p.leaf_row.size() * 4, cudaMemcpyHostToDevice));
        chk(cudaMemcpy(e->d_rec, p.rec.data(), p.rec.size() * sizeof(wdf::NodeRec), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(e->d_meta, p.meta.data(), p.meta.size() * sizeof(wdf::TreeMeta), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(e->d_flfeat, p.flush_feat.data(), p.flush_feat.size() * 4, cudaMemcpyHostToDevice));
        if (!p.xmask.empty())
            chk(cudaMemcpy(e->d_xmask, p.xmask.data(), p.xmask.size() * 8, cudaMemcpyHostToDevice));
        chk(cudaMemcpy(e->d_cols, p.cols.data(), p.cols.size() * sizeof(wdf::CodeCol), cudaMemcpyHostToDevice));
        if (!p.col_thr.empty())
            chk(cudaMemcpy(e->d_col_thr, p.col_thr.data(), p.col_thr.size() * 4, cudaMemcpyHostToDevice));
        if (e->n_tiles) chk(cudaMemcpy(e->d_tiles, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice));
        // step 2 of Algorithm 3 depends only on the path signatures: build the tables now
        chk(wdf::launch_tables(p.D, e->metric, e->d_keys, e->G, e->d_t32, nullptr, 0));
        chk(cudaStreamSynchronize(0));
    }
    if (ce != cudaSuccess) {
        free_ensemble(e);
        delete e;
        ctx_release(ctx);
        return cuda_fail(ce, "wdf_load_ensemble");
    }
    *out = e;
    return WDF_OK;
}

void wdf_ensemble_destroy(wdf_ensemble *ens) {
    if (!ens) return;
    wdf_ctx *ctx = ens->ctx;
    {
        DeviceGuard g(ctx->device);
        cudaDeviceSynchronize();
        free_ensemble(ens);
        delete ens;
    }
    ctx_release(ctx);
}

wdf_status wdf_ensemble_info(const wdf_ensemble *ens, wdf_info *out) {
    if (!ens || !out) return fail(WDF_EINVAL, "null argument");
    out->n_features = ens->pk.F;
    out->n_trees = ens->pk.T;
    out->depth = ens->pk.D;
    out->n_live_leaves = ens->n_live;
    out->n_signatures = ens->G;
    out->has_background = ens->has_bg;
    out->device_bytes = ens->bytes;
    return WDF_OK;
}

wdf_status wdf_set_metric(wdf_ensemble *ens, wdf_metric metric) {
    if (!ens) return fail(WDF_EINVAL, "ens is null");
    if (metric != WDF_SHAPLEY && metric != WDF_BANZHAF) return fail(WDF_EINVAL, "unknown metric");
    if ((int)metric == ens->metric) return WDF_OK;
    DeviceGuard g(ens->ctx->device);
    WDF_CUDA(cudaDeviceSynchronize());
    const wdf::Packed &p = ens->pk;
    ens->metric = (int)metric;
    ens->has_bg = 0;  // the folded vectors were built from the other tables
    WDF_CUDA(wdf::launch_tables(p.D, ens->metric, ens->d_keys, ens->G, ens->d_t32, nullptr, 0));
    if (ens->d_bpk) {  // split the new tables again on the next tensor-core contraction
        ens->bytes -= (int64_t)wdf::contract_tc_b_bytes(p.D, ens->bpk_mode, ens->G);
        dfree(ens->d_bpk);
        ens->bpk_mode = -1;
    }
    WDF_CUDA(cudaStreamSynchronize(0));
    return WDF_OK;
}

wdf_status wdf_set_background(wdf_ensemble *ens, const float *B, int64_t m, int64_t ldb, wdf_memkind kind,
                              wdf_precision precision, void *stream) {
    wdf::TraceRange trace_("wdf_set_background");
    if (!ens) return fail(WDF_EINVAL, "ens is null");
    if (m == 0) return fail(WDF_EUNSUPPORTED, "empty background (m == 0)");
    if (m < 0 || !B) return fail(WDF_EINVAL, "m must be positive and B non-null");
    if (ldb < ens->pk.F) return fail(WDF_EINVAL, "ldb < n_features");
    if (m > (int64_t)0xFFFFFFFF) return fail(WDF_EUNSUPPORTED, "more than 2^32-1 background rows");
    if (kind != WDF_MEM_HOST && kind != WDF_MEM_DEVICE) return fail(WDF_EINVAL, "bad memory kind");
    if (!valid_precision(precision))
        return fail(WDF_EINVAL, "unknown precision");
    DeviceGuard g(ens->ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const wdf::Packed &p = ens->pk;
    const int K = 1 << p.D;
    const size_t hist_n = (size_t)p.T * p.NS * (2 * K);
    wdf_status s0 = ensure_frequency_state(ens, precision);
    if (s0 != WDF_OK) return s0;
    WDF_CUDA(cudaMemsetAsync(ens->d_hist, 0, hist_n * 4, st));
    if (kind == WDF_MEM_DEVICE) {
        wdf_status s = count_device_rows(ens, B, m, ldb, ens->d_hist, st);
        if (s != WDF_OK) return s;
    } else {
        wdf_status s = ensure_staging(ens, m, false);
        if (s == WDF_OK) s = ensure_codes(ens, ens->stage_rows, 2);
        if (s != WDF_OK) return s;
        WDF_CUDA(cudaEventRecord(ens->ev_fork, st));
        for (int i = 0; i < 2; ++i) WDF_CUDA(cudaStreamWaitEvent(ens->ist[i], ens->ev_fork, 0));
        int64_t chunk = 0;
        for (int64_t r0 = 0; r0 < m; r0 += ens->stage_rows, ++chunk) {
            const int64_t rows = std::min(ens->stage_rows, m - r0);
            const int b = (int)(chunk & 1);
            WDF_CUDA(copy_rows(ens->d_stage_in[b], p.F, B + r0 * ldb, ldb, rows, p.F, cudaMemcpyHostToDevice,
                               ens->ist[b]));
            WDF_CUDA(wdf::launch_bg_hist(p.D, ens->d_stage_in[b], rows, p.F, ens->arrays(), p.T, ens->d_codes[b],
                                         ens->code_rows, ens->d_hist, ens->ctx->dev, ens->ist[b]));
        }
        for (int i = 0; i < 2; ++i) {
            WDF_CUDA(cudaEventRecord(ens->ev_join[i], ens->ist[i]));
            WDF_CUDA(cudaStreamWaitEvent(st, ens->ev_join[i], 0));
        }
    }
    wdf_status s1 = finish_background(ens, m, precision, st);
    if (s1 != WDF_OK) return s1;
    if (kind == WDF_MEM_HOST) WDF_CUDA(cudaStreamSynchronize(st));
    return WDF_OK;
}

int64_t wdf_background_counts_size(const wdf_ensemble *ens) {
    if (!ens) return -1;
    const wdf::Packed &p = ens->pk;
    return (int64_t)p.T * p.NS * (2 << p.D);
}

wdf_status wdf_background_counts(wdf_ensemble *ens, const float *B, int64_t m, int64_t ldb, uint32_t *counts,
                                 void *stream) {
    wdf::TraceRange trace_("wdf_background_counts");
    if (!ens) return fail(WDF_EINVAL, "ens is null");
    if (m < 0) return fail(WDF_EINVAL, "m < 0");
    if (m == 0) return WDF_OK;
    if (!B || !counts) return fail(WDF_EINVAL, "B and counts must be non-null");
    if (ldb < ens->pk.F) return fail(WDF_EINVAL, "ldb < n_features");
    if (m > (int64_t)0xFFFFFFFF) return fail(WDF_EUNSUPPORTED, "more than 2^32-1 background rows");
    DeviceGuard g(ens->ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const wdf::Packed &p = ens->pk;
    (void)p;
    return count_device_rows(ens, B, m, ldb, counts, st);
}

wdf_status wdf_set_background_counts(wdf_ensemble *ens, const uint32_t *counts, int64_t m_total,
                                     wdf_precision precision, void *stream) {
    wdf::TraceRange trace_("wdf_set_background_counts");
    if (!ens) return fail(WDF_EINVAL, "ens is null");
    if (!counts) return fail(WDF_EINVAL, "counts is null");
    if (m_total < 1) return fail(WDF_EUNSUPPORTED, "empty background (m_total < 1)");
    if (m_total > (int64_t)0xFFFFFFFF) return fail(WDF_EUNSUPPORTED, "more than 2^32-1 background rows");
    if (!valid_precision(precision))
        return fail(WDF_EINVAL, "unknown precision");
    DeviceGuard g(ens->ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    wdf_status s0 = ensure_frequency_state(ens, precision);
    if (s0 != WDF_OK) return s0;
    WDF_CUDA(cudaMemcpyAsync(ens->d_hist, counts, (size_t)wdf_background_counts_size(ens) * 4,
                             cudaMemcpyDeviceToDevice, st));
    return finish_background(ens, m_total, precision, st);
}

wdf_status wdf_set_covers(wdf_ensemble *ens, const double *cover) {
    if (!ens) return fail(WDF_EINVAL, "ens is null");
    std::vector<double> ratio;
    std::string err;
    const int rc = wdf::pd_ratios(ens->pk, cover, &ratio, &err);
    if (rc) return fail((wdf_status)rc, err);
    DeviceGuard g(ens->ctx->device);
    if (!ens->d_ratio) WDF_CUDA(dalloc(&ens->d_ratio, std::max<size_t>(ratio.size(), 1), &ens->bytes));
    if (!ratio.empty())
        WDF_CUDA(cudaMemcpy(ens->d_ratio, ratio.data(), ratio.size() * sizeof(double), cudaMemcpyHostToDevice));
    ens->has_covers = 1;
    return WDF_OK;
}

wdf_status wdf_set_path_dependent(wdf_ensemble *ens, wdf_precision precision, void *stream) {
    wdf::TraceRange trace_("wdf_set_path_dependent");
    if (!ens) return fail(WDF_EINVAL, "ens is null");
    if (!ens->has_covers) return fail(WDF_EINVAL, "wdf_set_covers must succeed before wdf_set_path_dependent");
    if (!valid_precision(precision))
        return fail(WDF_EINVAL, "unknown precision");
    DeviceGuard g(ens->ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const wdf::Packed &p = ens->pk;
    wdf_status s0 = ensure_frequency_state(ens, precision);
    if (s0 != WDF_OK) return s0;
    WDF_CUDA(wdf::launch_pd_freq(p.D, ens->d_ratio, ens->n_live, ens->d_A, st));
    WDF_CUDA(wdf::launch_scale(ens->d_w_rows, ens->n_live, 1, ens->d_scale, st));
    WDF_CUDA(wdf::launch_base_value(p.D, nullptr, ens->d_ratio, ens->d_w_rows, ens->n_live, 1, ens->d_base, st));
    WDF_CUDA(wdf::launch_line_maps(p.D, nullptr, p.T, ens->d_lines, st));
    wdf_status s1 = contract_and_fold(ens, precision, st);
    if (s1 != WDF_OK) return s1;
    ens->m = 0;
    ens->pd = 1;
    ens->has_bg = 1;
    return WDF_OK;
}

wdf_status wdf_explain(wdf_ensemble *ens, const float *C, int64_t n, int64_t ldc, wdf_memkind kind, float *phi,
                       int64_t ldphi, void *stream) {
    wdf::TraceRange trace_("wdf_explain");
    if (!ens) return fail(WDF_EINVAL, "ens is null");
    if (!ens->has_bg) return fail(WDF_EINVAL, "wdf_set_background must succeed before wdf_explain");
    if (n < 0) return fail(WDF_EINVAL, "n < 0");
    if (n == 0) return WDF_OK;
    if (!C || !phi) return fail(WDF_EINVAL, "C and phi must be non-null");
    const wdf::Packed &p = ens->pk;
    if (ldc < p.F || ldphi < p.F) return fail(WDF_EINVAL, "leading dimension < n_features");
    if (kind != WDF_MEM_HOST && kind != WDF_MEM_DEVICE) return fail(WDF_EINVAL, "bad memory kind");
    DeviceGuard g(ens->ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (kind == WDF_MEM_DEVICE) {
        WDF_CUDA(wdf::launch_explain(p.D, C, n, ldc, ens->job(), phi, ldphi, 0, ens->ctx->dev, st));
        return WDF_OK;
    }
    wdf_status s = ensure_staging(ens, n, true);
    if (s != WDF_OK) return s;
    WDF_CUDA(cudaEventRecord(ens->ev_fork, st));
    for (int i = 0; i < 2; ++i) WDF_CUDA(cudaStreamWaitEvent(ens->ist[i], ens->ev_fork, 0));
    int64_t chunk = 0;
    for (int64_t r0 = 0; r0 < n; r0 += ens->stage_rows, ++chunk) {
        const int64_t rows = std::min(ens->stage_rows, n - r0);
        const int b = (int)(chunk & 1);
        cudaStream_t sb = ens->ist[b];
        WDF_CUDA(copy_rows(ens->d_stage_in[b], p.F, C + r0 * ldc, ldc, rows, p.F, cudaMemcpyHostToDevice, sb));
        WDF_CUDA(wdf::launch_explain(p.D, ens->d_stage_in[b], rows, p.F, ens->job(), ens->d_stage_out[b], p.F, 0,
                                     ens->ctx->dev, sb));
        WDF_CUDA(copy_rows(phi + r0 * ldphi, ldphi, ens->d_stage_out[b], p.F, rows, p.F, cudaMemcpyDeviceToHost, sb));
    }
    for (int i = 0; i < 2; ++i) {
        WDF_CUDA(cudaEventRecord(ens->ev_join[i], ens->ist[i]));
        WDF_CUDA(cudaStreamWaitEvent(st, ens->ev_join[i], 0));
    }
    WDF_CUDA(cudaStreamSynchronize(st));
    return WDF_OK;
}

wdf_status wdf_explain_interactions(wdf_ensemble *ens, const float *C, int64_t n, int64_t ldc, float *out,
                                    int64_t ldo, void *stream) {
    wdf::TraceRange trace_("wdf_explain_interactions");
    if (!ens) return fail(WDF_EINVAL, "ens is null");
    if (!ens->has_bg)
        return fail(WDF_EINVAL, "wdf_set_background or wdf_set_path_dependent must succeed before interactions");
    if (n < 0) return fail(WDF_EINVAL, "n < 0");
    if (n == 0) return WDF_OK;
    if (!C || !out) return fail(WDF_EINVAL, "C and out must be non-null");
    const wdf::Packed &p = ens->pk;
    if (ldc < p.F) return fail(WDF_EINVAL, "ldc < n_features");
    if (ldo < (int64_t)p.F * p.F) return fail(WDF_EINVAL, "ldo < n_features^2");
    DeviceGuard g(ens->ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int D = p.D, K = 1 << D, P = D * (D - 1) / 2, PP = (P + 3) & ~3;
    // pair tables, the contraction and its repacking live in one stream-ordered block
    // depth <= 6: pair values folded per bottom-subtree entry; deeper: per leaf
    const bool folded = D <= 6;
    const size_t n_t2 = (size_t)ens->G * K * P * K, n_s2 = (size_t)ens->n_live * P * K;
    const size_t n_s2t = folded ? wdf::iv_fold_floats(D, p.T) : (size_t)ens->n_live * K * PP;
    float *buf = nullptr;
    WDF_CUDA(cudaMallocAsync(reinterpret_cast<void **>(&buf), std::max<size_t>(n_t2 + n_s2 + n_s2t, 4) * 4, st));
    float *t2 = buf, *s2 = buf + n_t2, *s2t = buf + n_t2 + n_s2;
    cudaError_t e = wdf::launch_tables_iv(D, ens->metric, ens->d_keys, ens->G, t2, st);
    if (e == cudaSuccess)
        e = wdf::launch_contract_fp32(D, ens->d_A, ens->d_scale, ens->d_tiles, ens->n_tiles, t2, s2, st, P);
    if (e == cudaSuccess)
        e = folded ? wdf::launch_iv_fold(D, s2, ens->d_leaf_row, p.T, s2t, st)
                   : wdf::launch_iv_pack(D, PP, s2, ens->n_live, s2t, st);
    if (e == cudaSuccess)
        e = wdf::launch_explain_iv(D, C, n, ldc, p.F, ens->arrays(), p.T, ens->d_group_leaf, ens->n_live,
                                   folded ? nullptr : s2t, folded ? s2t : nullptr, out, ldo, ens->ctx->dev, st);
    const cudaError_t fe = cudaFreeAsync(buf, st);
    WDF_CUDA(e);
    WDF_CUDA(fe);
    return WDF_OK;
}

wdf_status wdf_expected_value(const wdf_ensemble *ens, double *out, void *stream) {
    if (!ens || !out) return fail(WDF_EINVAL, "null argument");
    if (!ens->has_bg) return fail(WDF_EINVAL, "no background set");
    DeviceGuard g(ens->ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    WDF_CUDA(cudaMemcpyAsync(out, ens->d_base, sizeof(double), cudaMemcpyDeviceToHost, st));
    WDF_CUDA(cudaStreamSynchronize(st));
    return WDF_OK;
}

wdf_status wdf_global_attribution(wdf_ctx *ctx, const float *phi, int64_t n, int64_t ldphi, int32_t n_features,
                                  double *mean_abs, double *mean, void *stream) {
    wdf::TraceRange trace_("wdf_global_attribution");
    if (!ctx || !mean_abs || !mean) return fail(WDF_EINVAL, "null argument");
    if (n < 0 || n_features < 1 || ldphi < n_features) return fail(WDF_EINVAL, "bad sizes");
    if (n > 0 && !phi) return fail(WDF_EINVAL, "phi is null");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t pn = (size_t)wdf::global_attr_partial_doubles(n, n_features);
    double *partial = nullptr;
    WDF_CUDA(cudaMallocAsync((void **)&partial, pn * sizeof(double), st));
    cudaError_t e = wdf::launch_global_attr(phi, n, ldphi, n_features, partial, mean_abs, mean, st);
    cudaFreeAsync(partial, st);
    if (e != cudaSuccess) return cuda_fail(e, "wdf_global_attribution");
    return WDF_OK;
}

wdf_status wdf_debug_leaf_hist(const wdf_ensemble *ens, uint32_t *out, int64_t out_elems) {
    if (!ens || !out) return fail(WDF_EINVAL, "null argument");
    if (!ens->has_bg || ens->pd) return fail(WDF_EINVAL, "no background set");
    const wdf::Packed &p = ens->pk;
    const int64_t total = (int64_t)p.T * p.NL * p.NL;
    if (out_elems < total) return fail(WDF_EINVAL, "output too small");
    DeviceGuard g(ens->ctx->device);
    std::vector<int32_t> all((size_t)p.T * p.NL);
    for (size_t i = 0; i < all.size(); ++i) all[i] = (int32_t)i;
    int32_t *d_all = nullptr;
    uint32_t *d_out = nullptr;
    int64_t dummy = 0;
    cudaError_t ce = dalloc(&d_all, all.size(), &dummy);
    if (ce == cudaSuccess) ce = dalloc(&d_out, (size_t)total, &dummy);
    if (ce == cudaSuccess) ce = cudaDeviceSynchronize();
    if (ce == cudaSuccess) ce = cudaMemcpy(d_all, all.data(), all.size() * 4, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = wdf::launch_leaf_counts(p.D, ens->d_hist, d_all, (int)all.size(), d_out, nullptr, 0);
    if (ce == cudaSuccess) ce = cudaMemcpy(out, d_out, (size_t)total * 4, cudaMemcpyDeviceToHost);
    dfree(d_all);
    dfree(d_out);
    if (ce != cudaSuccess) return cuda_fail(ce, "wdf_debug_leaf_hist");
    return WDF_OK;
}

wdf_status wdf_debug_pair_table(wdf_ctx *ctx, int32_t depth, const int32_t *first, wdf_metric metric, double *out) {
    if (!ctx || !first || !out) return fail(WDF_EINVAL, "null argument");
    if (depth < 1 || depth > wdf::kMaxDepth) return fail(WDF_EINVAL, "depth must be in [1, 8]");
    if (metric != WDF_SHAPLEY && metric != WDF_BANZHAF) return fail(WDF_EINVAL, "unknown metric");
    uint32_t key = 0;
    for (int k = 0; k < depth; ++k) {
        if (first[k] < 0 || first[k] > k || first[first[k]] != first[k])
            return fail(WDF_EINVAL, "first[k] must be the first position of position k's feature");
        key |= (uint32_t)first[k] << (3 * k);
    }
    DeviceGuard g(ctx->device);
    const size_t K = (size_t)1 << depth, N = (size_t)depth << depth;
    uint32_t *d_key = nullptr;
    float *d_t32 = nullptr;
    double *d_t64 = nullptr;
    int64_t dummy = 0;
    cudaError_t ce = dalloc(&d_key, 1, &dummy);
    if (ce == cudaSuccess) ce = dalloc(&d_t32, K * N, &dummy);
    if (ce == cudaSuccess) ce = dalloc(&d_t64, K * N, &dummy);
    if (ce == cudaSuccess) ce = cudaMemcpy(d_key, &key, 4, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = wdf::launch_tables(depth, (int)metric, d_key, 1, d_t32, d_t64, 0);
    if (ce == cudaSuccess) ce = cudaMemcpy(out, d_t64, K * N * sizeof(double), cudaMemcpyDeviceToHost);
    dfree(d_key);
    dfree(d_t32);
    dfree(d_t64);
    if (ce != cudaSuccess) return cuda_fail(ce, "wdf_debug_shapley_table");
    return WDF_OK;
}

}  // extern "C"
