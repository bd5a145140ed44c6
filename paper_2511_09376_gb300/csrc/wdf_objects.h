// Library object definitions shared by the C-ABI translation units (internal).
#pragma once
#include <atomic>
#include <cstdint>

#include "launch.h"
#include "wdf_internal.h"

struct wdf_ctx {
    int device = 0;
    wdf::DevInfo dev;
    // the caller's handle plus one reference per ensemble, batch and server made from the
    // context, so wdf_ctx_destroy may come before theirs: the last reference frees it
    std::atomic<int> refs{1};
};
inline wdf_ctx *ctx_retain(wdf_ctx *c) {
    c->refs.fetch_add(1, std::memory_order_relaxed);
    return c;
}
inline void ctx_release(wdf_ctx *c) {
    if (c && c->refs.fetch_sub(1, std::memory_order_acq_rel) == 1) delete c;
}

struct wdf_ensemble {
    wdf_ctx *ctx = nullptr;
    wdf::Packed pk;
    int G = 0, n_live = 0, n_tiles = 0;
    int metric = 0;  // 0 Shapley, 1 Banzhaf (the pattern-pair table formula)
    int pd = 0;          // 1 when the frequencies are the path-dependent ones
    int has_covers = 0;  // wdf_set_covers succeeded
    float *d_A = nullptr;       // frequencies of every live leaf's baseline patterns (FP32)
    double *d_ratio = nullptr;  // path-dependent cover ratios [live leaves][D]
    int64_t bytes = 0;
    // ensemble (load time)
    int2 *d_nodes = nullptr;
    uint32_t *d_keys = nullptr;
    int32_t *d_group_leaf = nullptr;
    int32_t *d_leaf_row = nullptr;
    double *d_w_rows = nullptr;
    int4 *d_tiles = nullptr;
    float *d_t32 = nullptr;
    wdf::NodeRec *d_rec = nullptr;
    wdf::TreeMeta *d_meta = nullptr;
    int32_t *d_flfeat = nullptr;  // features in consumer flush order (Packed::flush_feat)
    unsigned long long *d_xmask = nullptr;  // per tree expand masks of the real nodes (depth <= 6)
    wdf::CodeCol *d_cols = nullptr;
    float *d_col_thr = nullptr;
    // tensor-core contraction: split operand stages (A for any mode, B for bpk_mode),
    // 128-row tiles, wait-expiry flag
    unsigned char *d_apk = nullptr;
    unsigned char *d_bpk = nullptr;
    int bpk_mode = -1;
    int4 *d_tiles128 = nullptr;
    int n_tiles128 = 0;
    int *d_err = nullptr;
    wdf::TreeArrays arrays() const {
        return wdf::TreeArrays{d_nodes, d_rec, d_meta, d_cols, d_col_thr, (int)pk.cols.size(), pk.code_bytes,
                              d_xmask};
    }
    wdf::ExplainJob job() const { return wdf::ExplainJob{arrays(), d_sfold, d_lines, d_flfeat, pk.T, pk.F}; }
    // background state (set_background)
    int has_bg = 0;
    int64_t m = 0;
    uint32_t *d_hist = nullptr;
    uint32_t *d_vc = nullptr;
    float *d_scale = nullptr;
    float *d_S = nullptr;
    float *d_sfold = nullptr;
    uint32_t *d_lines = nullptr;  // line maps of the folded vectors (launch.h)
    double *d_base = nullptr;
    // staging for host-memory calls: two buffers per direction, one per internal stream
    float *d_stage_in[2] = {nullptr, nullptr};
    float *d_stage_out[2] = {nullptr, nullptr};
    int64_t stage_rows = 0;
    // decision codes of background rows (one buffer per staging stream)
    unsigned char *d_codes[2] = {nullptr, nullptr};
    int64_t code_rows = 0;
    cudaStream_t ist[2] = {nullptr, nullptr};
    cudaEvent_t ev_fork = nullptr, ev_join[2] = {nullptr, nullptr};
    cudaEvent_t ev_enc[2] = {nullptr, nullptr}, ev_cnt[2] = {nullptr, nullptr};  // encode / count overlap
};

