// Ragged batches: one graph launch explains requests against many ensembles of
// different depths and feature counts.
//
// Ensembles are grouped into depth classes (one kernel instantiation per depth).  A
// call writes every class's work description -- the ensembles' device arrays (jobs),
// the requests, the encode items (request, 32-row block) and the work items (job,
// request, first row) of tile_rows consumer rows each -- into one pinned host blob; the
// captured graph copies that blob to the device with a single memcpy and then runs, per
// class on parallel branches, k_encode_batch (the rows' decision codes into the batch's
// code arena) and one persistent k_explain_batch.  The item count is read on the device, so the same graph serves
// every call until a capacity grows.  Results per consumer row are exactly those of
// wdf_explain: the per-row arithmetic and its order do not depend on the batch.
//
// The autotuner times every tile size that fits the class's shared-memory budget on the
// caller's own requests and keeps the fastest per class; results can be cached in a text
// file keyed by (depth, feature count rounded up to 32).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "wdf_objects.h"
#include "woodelf.h"

namespace {

size_t up16(size_t v) { return (v + 15) & ~(size_t)15; }

wdf_status fail(wdf_status s, const std::string &msg) {
    wdf::set_last_error(msg);
    return s;
}

#define WDF_CUDA(call)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return fail(WDF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

struct Cls {
    int D = 0, F_max = 0, xb_max = 0, tile_rows = 0;
    std::vector<int> members;  // batch ensemble indices, in job-slot order
    int cap_reqs = 0, cap_items = 0, cap_eitems = 0;
    size_t off_jobs = 0, off_reqs = 0, off_items = 0, off_count = 0, off_eitems = 0, off_ecount = 0;
};

// Rows of a request's code region: a multiple of every tile size (and of 32).
constexpr int64_t kCodePad = 128;
int64_t padded_rows(int64_t n) { return (n + kCodePad - 1) / kCodePad * kCodePad; }

}  // namespace

struct wdf_batch {
    wdf_ctx *ctx = nullptr;
    std::vector<wdf_ensemble *> ens;
    std::vector<int> cls_of, slot_of;
    std::vector<Cls> cls;
    unsigned char *h_blob = nullptr, *d_blob = nullptr;
    size_t blob_bytes = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
    std::vector<cudaStream_t> branch;
    cudaEvent_t ev_fork = nullptr, ev_copied = nullptr;
    std::vector<cudaEvent_t> ev_join;
    bool copied_pending = false;
    unsigned char *d_codes = nullptr;  // decision codes of the requests' rows
    size_t codes_cap = 0;
};

namespace {

struct Req {
    int e;  // batch ensemble index
    const float *C;
    float *phi;
    int64_t n, ldc, ldp;
    size_t codes_off = 0;  // the request's region of the code arena
};

void drop_graph(wdf_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

wdf_status wait_copied(wdf_batch *b) {
    if (b->copied_pending) WDF_CUDA(cudaEventSynchronize(b->ev_copied));
    b->copied_pending = false;
    return WDF_OK;
}

// Code arena regions of the requests (one per request, padded rows x the ensemble's code
// bytes per row), growing the arena if needed.  The regions' addresses travel in the
// blob, so the captured graph stays valid when the arena moves.
wdf_status place_codes(wdf_batch *b, std::vector<Req> *reqs) {
    size_t total = 0;
    for (Req &r : *reqs) {
        const wdf::Packed &p = b->ens[(size_t)r.e]->pk;
        r.codes_off = total;
        total += (size_t)padded_rows(r.n) * p.cols.size() * (size_t)p.code_bytes;
    }
    if (total > b->codes_cap) {
        wdf_status s = wait_copied(b);
        if (s != WDF_OK) return s;
        WDF_CUDA(cudaDeviceSynchronize());  // earlier launches may still read the old arena
        if (b->d_codes) cudaFree(b->d_codes);
        b->d_codes = nullptr;
        b->codes_cap = 0;
        const size_t cap = std::max<size_t>(total + total / 2, 1 << 20);
        WDF_CUDA(cudaMalloc((void **)&b->d_codes, cap));
        b->codes_cap = cap;
    }
    return WDF_OK;
}

// Blob layout for the current capacities; reallocates (and drops the graph) if it grew.
wdf_status ensure_blob(wdf_batch *b, const std::vector<int> &need_reqs, const std::vector<int> &need_items,
                       const std::vector<int> &need_eitems) {
    bool grow = b->h_blob == nullptr;
    for (size_t c = 0; c < b->cls.size(); ++c)
        if (need_reqs[c] > b->cls[c].cap_reqs || need_items[c] > b->cls[c].cap_items ||
            need_eitems[c] > b->cls[c].cap_eitems)
            grow = true;
    if (!grow) return WDF_OK;
    wdf_status s = wait_copied(b);
    if (s != WDF_OK) return s;
    WDF_CUDA(cudaDeviceSynchronize());
    drop_graph(b);
    size_t off = 0;
    for (size_t c = 0; c < b->cls.size(); ++c) {
        Cls &k = b->cls[c];
        k.cap_reqs = std::max(k.cap_reqs, std::max(need_reqs[c], 4) * 3 / 2);
        k.cap_items = std::max(k.cap_items, std::max(need_items[c], 64) * 3 / 2);
        k.cap_eitems = std::max(k.cap_eitems, std::max(need_eitems[c], 64) * 3 / 2);
        k.off_jobs = off;
        off = up16(off + k.members.size() * sizeof(wdf::ExplainJob));
        k.off_reqs = off;
        off = up16(off + (size_t)k.cap_reqs * sizeof(wdf::BatchRequest));
        k.off_items = off;
        off = up16(off + (size_t)k.cap_items * sizeof(int4));
        k.off_count = off;
        off = up16(off + 2 * sizeof(int));
        k.off_eitems = off;
        off = up16(off + (size_t)k.cap_eitems * sizeof(int2));
        k.off_ecount = off;
        off = up16(off + sizeof(int));
    }
    if (b->h_blob) cudaFreeHost(b->h_blob);
    if (b->d_blob) cudaFree(b->d_blob);
    b->h_blob = nullptr;
    b->d_blob = nullptr;
    WDF_CUDA(cudaMallocHost((void **)&b->h_blob, off));
    WDF_CUDA(cudaMalloc((void **)&b->d_blob, off));
    std::memset(b->h_blob, 0, off);
    b->blob_bytes = off;
    return WDF_OK;
}

// Writes one class's jobs, requests and items into the host blob.
int fill_class(wdf_batch *b, int c, const std::vector<Req> &reqs, int tile_rows) {
    Cls &k = b->cls[(size_t)c];
    auto *jobs = reinterpret_cast<wdf::ExplainJob *>(b->h_blob + k.off_jobs);
    for (size_t j = 0; j < k.members.size(); ++j) jobs[j] = b->ens[(size_t)k.members[j]]->job();
    auto *rq = reinterpret_cast<wdf::BatchRequest *>(b->h_blob + k.off_reqs);
    auto *items = reinterpret_cast<int4 *>(b->h_blob + k.off_items);
    auto *eitems = reinterpret_cast<int2 *>(b->h_blob + k.off_eitems);
    int nr = 0, ni = 0, ne = 0;
    for (const Req &r : reqs) {
        if (b->cls_of[(size_t)r.e] != c) continue;
        rq[nr] = wdf::BatchRequest{r.C, r.phi, b->d_codes + r.codes_off, r.n, r.ldc, r.ldp, b->slot_of[(size_t)r.e]};
        for (int64_t c0 = 0; c0 < r.n; c0 += tile_rows)
            items[ni++] = make_int4(b->slot_of[(size_t)r.e], nr, (int)(c0 >> 31), (int)(c0 & 0x7FFFFFFF));
        for (int64_t blk = 0; blk < padded_rows(r.n) / 32; ++blk) eitems[ne++] = make_int2(nr, (int)blk);
        ++nr;
    }
    // longest first: tiles of ensembles with more trees cost more; blocks claim items in
    // this order, so the cheap ones fill the tail of the launch
    std::stable_sort(items, items + ni, [&](const int4 &a, const int4 &c) {
        return b->ens[(size_t)k.members[(size_t)a.x]]->pk.T > b->ens[(size_t)k.members[(size_t)c.x]]->pk.T;
    });
    int *hdr = reinterpret_cast<int *>(b->h_blob + k.off_count);
    hdr[0] = ni;  // item count
    hdr[1] = 0;   // claim counter, zero at every launch
    *reinterpret_cast<int *>(b->h_blob + k.off_ecount) = ne;
    return ni;
}

// Blocks of the batched encode: eight per SM walk the (request, 32-row block) items.
int kEncodeGrid(const wdf_batch *b) { return 8 * std::max(1, b->ctx->dev.sms); }

wdf_status capture(wdf_batch *b) {
    drop_graph(b);
    WDF_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed));
    cudaError_t e = cudaMemcpyAsync(b->d_blob, b->h_blob, b->blob_bytes, cudaMemcpyHostToDevice, b->cap);
    // an event-record node the host can wait on before rewriting the pinned blob
    if (e == cudaSuccess) e = cudaEventRecordWithFlags(b->ev_copied, b->cap, cudaEventRecordExternal);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_fork, b->cap);
    for (size_t c = 0; c < b->cls.size() && e == cudaSuccess; ++c) {
        const Cls &k = b->cls[c];
        e = cudaStreamWaitEvent(b->branch[c], b->ev_fork, 0);
        if (e == cudaSuccess)
            e = wdf::launch_encode_batch(reinterpret_cast<const wdf::ExplainJob *>(b->d_blob + k.off_jobs),
                                         reinterpret_cast<const wdf::BatchRequest *>(b->d_blob + k.off_reqs),
                                         reinterpret_cast<const int2 *>(b->d_blob + k.off_eitems),
                                         reinterpret_cast<const int *>(b->d_blob + k.off_ecount), kEncodeGrid(b),
                                         b->branch[c]);
        if (e == cudaSuccess)
            e = wdf::launch_explain_batch(
                k.D, reinterpret_cast<const wdf::ExplainJob *>(b->d_blob + k.off_jobs),
                reinterpret_cast<const wdf::BatchRequest *>(b->d_blob + k.off_reqs),
                reinterpret_cast<const int4 *>(b->d_blob + k.off_items),
                reinterpret_cast<int *>(b->d_blob + k.off_count), k.F_max, k.xb_max, k.tile_rows, 0, b->ctx->dev,
                b->branch[c]);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_join[c], b->branch[c]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, b->ev_join[c], 0);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
    wdf::count_launches(-2 * (int)b->cls.size());  // counted per graph launch instead
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(WDF_ECUDA, std::string("batch graph capture: ") + cudaGetErrorString(e));
    }
    if (e2 != cudaSuccess) return fail(WDF_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e2));
    b->graph = g;
    WDF_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
    return WDF_OK;
}

wdf_status gather_requests(wdf_batch *b, int32_t nreq, const int32_t *idx, const float *const *C, const int64_t *n,
                           const int64_t *ldc, float *const *phi, const int64_t *ldphi, std::vector<Req> *out) {
    if (nreq < 0 || (nreq > 0 && (!idx || !C || !n || !ldc || !phi || !ldphi)))
        return fail(WDF_EINVAL, "bad request arrays");
    out->clear();
    for (int i = 0; i < nreq; ++i) {
        if (idx[i] < 0 || idx[i] >= (int)b->ens.size()) return fail(WDF_EINVAL, "ensemble index out of range");
        const wdf_ensemble *e = b->ens[(size_t)idx[i]];
        if (!e->has_bg) return fail(WDF_EINVAL, "an ensemble of the batch has no background");
        if (n[i] < 0 || (n[i] > 0 && (!C[i] || !phi[i])) || ldc[i] < e->pk.F || ldphi[i] < e->pk.F)
            return fail(WDF_EINVAL, "bad request " + std::to_string(i));
        if (n[i] > 0) out->push_back(Req{idx[i], C[i], phi[i], n[i], ldc[i], ldphi[i]});
    }
    return WDF_OK;
}

void count_needs(const wdf_batch *b, const std::vector<Req> &reqs, const std::vector<int> &tile_rows,
                 std::vector<int> *need_reqs, std::vector<int> *need_items, std::vector<int> *need_eitems) {
    need_reqs->assign(b->cls.size(), 0);
    need_items->assign(b->cls.size(), 0);
    need_eitems->assign(b->cls.size(), 0);
    for (const Req &r : reqs) {
        const int c = b->cls_of[(size_t)r.e];
        (*need_reqs)[(size_t)c] += 1;
        (*need_items)[(size_t)c] += (int)((r.n + tile_rows[(size_t)c] - 1) / tile_rows[(size_t)c]);
        (*need_eitems)[(size_t)c] += (int)(padded_rows(r.n) / 32);
    }
}

}  // namespace

extern "C" {

wdf_status wdf_batch_create(wdf_ctx *ctx, int32_t n_ensembles, wdf_ensemble *const *ensembles, wdf_batch **out) {
    if (!ctx || !out || n_ensembles < 1 || !ensembles) return fail(WDF_EINVAL, "bad arguments");
    *out = nullptr;
    for (int i = 0; i < n_ensembles; ++i)
        if (!ensembles[i] || ensembles[i]->ctx != ctx) return fail(WDF_EINVAL, "ensemble missing or of another context");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    wdf_batch *b = new wdf_batch();
    b->ctx = ctx_retain(ctx);
    b->ens.assign(ensembles, ensembles + n_ensembles);
    b->cls_of.assign((size_t)n_ensembles, -1);
    b->slot_of.assign((size_t)n_ensembles, -1);
    for (int i = 0; i < n_ensembles; ++i) {
        const int D = b->ens[(size_t)i]->pk.D;
        int c = -1;
        for (size_t k = 0; k < b->cls.size(); ++k)
            if (b->cls[k].D == D) c = (int)k;
        if (c < 0) {
            b->cls.push_back(Cls());
            c = (int)b->cls.size() - 1;
            b->cls.back().D = D;
        }
        Cls &k = b->cls[(size_t)c];
        k.F_max = std::max(k.F_max, b->ens[(size_t)i]->pk.F);
        k.xb_max = std::max(k.xb_max, (int)b->ens[(size_t)i]->pk.cols.size() * b->ens[(size_t)i]->pk.code_bytes);
        b->cls_of[(size_t)i] = c;
        b->slot_of[(size_t)i] = (int)k.members.size();
        k.members.push_back(i);
    }
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_copied, cudaEventDisableTiming);
    b->branch.assign(b->cls.size(), nullptr);
    b->ev_join.assign(b->cls.size(), nullptr);
    for (size_t c = 0; c < b->cls.size() && e == cudaSuccess; ++c) {
        Cls &k = b->cls[c];
        k.tile_rows = wdf::default_tile_rows(k.D, k.F_max, k.xb_max, ctx->dev);
        if (wdf::explain_smem_bytes(k.D, k.F_max, k.xb_max, k.tile_rows) > ctx->dev.smem_optin) {
            e = cudaErrorInvalidConfiguration;
            break;
        }
        e = cudaStreamCreateWithFlags(&b->branch[c], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[c], cudaEventDisableTiming);
    }
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        wdf_batch_destroy(b);
        return fail(WDF_ECUDA, std::string("wdf_batch_create: ") + cudaGetErrorString(e));
    }
    *out = b;
    return WDF_OK;
}

void wdf_batch_destroy(wdf_batch *b) {
    if (!b) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (b->ctx && prev != b->ctx->device) cudaSetDevice(b->ctx->device);
    cudaDeviceSynchronize();
    drop_graph(b);
    if (b->h_blob) cudaFreeHost(b->h_blob);
    if (b->d_blob) cudaFree(b->d_blob);
    if (b->d_codes) cudaFree(b->d_codes);
    for (cudaStream_t s : b->branch)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t ev : b->ev_join)
        if (ev) cudaEventDestroy(ev);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_copied) cudaEventDestroy(b->ev_copied);
    if (b->ctx && prev >= 0 && prev != b->ctx->device) cudaSetDevice(prev);
    ctx_release(b->ctx);
    delete b;
}

wdf_status wdf_batch_explain(wdf_batch *b, int32_t n_requests, const int32_t *ensemble_index, const float *const *C,
                             const int64_t *n, const int64_t *ldc, float *const *phi, const int64_t *ldphi,
                             void *stream) {
    wdf::TraceRange trace_("wdf_batch_explain");
    if (!b) return fail(WDF_EINVAL, "batch is null");
    std::vector<Req> reqs;
    wdf_status s = gather_requests(b, n_requests, ensemble_index, C, n, ldc, phi, ldphi, &reqs);
    if (s != WDF_OK) return s;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->ctx->device) cudaSetDevice(b->ctx->device);
    std::vector<int> tiles, need_reqs, need_items, need_eitems;
    for (const Cls &k : b->cls) tiles.push_back(k.tile_rows);
    count_needs(b, reqs, tiles, &need_reqs, &need_items, &need_eitems);
    s = ensure_blob(b, need_reqs, need_items, need_eitems);
    if (s == WDF_OK) s = place_codes(b, &reqs);
    if (s == WDF_OK) s = wait_copied(b);
    if (s == WDF_OK) {
        for (size_t c = 0; c < b->cls.size(); ++c) fill_class(b, (int)c, reqs, b->cls[c].tile_rows);
        if (!b->exec) s = capture(b);
    }
    if (s == WDF_OK) {
        const cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
        if (e != cudaSuccess) s = fail(WDF_ECUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
        else {
            b->copied_pending = true;
            wdf::count_launches(2 * (int)b->cls.size());
        }
    }
    if (prev >= 0 && prev != b->ctx->device) cudaSetDevice(prev);
    return s;
}

wdf_status wdf_batch_autotune(wdf_batch *b, int32_t n_requests, const int32_t *ensemble_index, const float *const *C,
                              const int64_t *n, const int64_t *ldc, float *const *phi, const int64_t *ldphi,
                              int32_t reps, const char *cache_path, void *stream) {
    wdf::TraceRange trace_("wdf_batch_autotune");
    if (!b) return fail(WDF_EINVAL, "batch is null");
    std::vector<Req> reqs;
    wdf_status s = gather_requests(b, n_requests, ensemble_index, C, n, ldc, phi, ldphi, &reqs);
    if (s != WDF_OK) return s;
    reps = std::max(1, reps);
    // cached choices: "depth features_rounded code_bytes_rounded tile_rows ms" per line
    std::vector<std::vector<int>> cached;
    if (cache_path) {
        std::ifstream in(cache_path);
        std::string line;
        while (std::getline(in, line)) {
            std::istringstream ls(line);
            int d, f, x, t;
            if (ls >> d >> f >> x >> t) cached.push_back({d, f, x, t});
        }
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->ctx->device) cudaSetDevice(b->ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int cand[3] = {32, 64, 128};
    std::vector<int> t32(b->cls.size(), 32), need_reqs, need_items, need_eitems;
    count_needs(b, reqs, t32, &need_reqs, &need_items, &need_eitems);  // tile_rows 32 needs the most items
    s = ensure_blob(b, need_reqs, need_items, need_eitems);
    if (s == WDF_OK) s = place_codes(b, &reqs);
    if (s == WDF_OK) s = wait_copied(b);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (s == WDF_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        s = fail(WDF_ECUDA, "cudaEventCreate");
    std::ofstream log;
    if (s == WDF_OK && cache_path) log.open(cache_path, std::ios::app);
    for (size_t c = 0; c < b->cls.size() && s == WDF_OK; ++c) {
        Cls &k = b->cls[c];
        if (need_reqs[c] == 0) continue;
        const int fkey = (k.F_max + 31) / 32 * 32, xkey = (k.xb_max + 31) / 32 * 32;
        int hit = 0;
        for (const auto &row : cached)
            if (row[0] == k.D && row[1] == fkey && row[2] == xkey) hit = row[3];
        if (hit) {
            k.tile_rows = hit;
            continue;
        }
        float best_ms = 1e30f;
        int best = k.tile_rows;
        // the rows' codes do not depend on the tile size: encode them once
        fill_class(b, (int)c, reqs, k.tile_rows);
        {
            cudaError_t e = cudaMemcpyAsync(b->d_blob, b->h_blob, b->blob_bytes, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess)
                e = wdf::launch_encode_batch(reinterpret_cast<const wdf::ExplainJob *>(b->d_blob + k.off_jobs),
                                             reinterpret_cast<const wdf::BatchRequest *>(b->d_blob + k.off_reqs),
                                             reinterpret_cast<const int2 *>(b->d_blob + k.off_eitems),
                                             reinterpret_cast<const int *>(b->d_blob + k.off_ecount), kEncodeGrid(b),
                                             st);
            if (e != cudaSuccess) {
                s = fail(WDF_ECUDA, std::string("autotune: ") + cudaGetErrorString(e));
                break;
            }
        }
        for (int tc : cand) {
            if (wdf::explain_smem_bytes(k.D, k.F_max, k.xb_max, tc) > b->ctx->dev.smem_optin) continue;
            fill_class(b, (int)c, reqs, tc);
            cudaError_t e = cudaMemcpyAsync(b->d_blob, b->h_blob, b->blob_bytes, cudaMemcpyHostToDevice, st);
            float ms = 0.0f;
            for (int r = -1; r < reps && e == cudaSuccess; ++r) {  // r = -1 warms up
                if (r == 0) e = cudaEventRecord(e0, st);
                if (e == cudaSuccess)  // reset the claim counter of this class
                    e = cudaMemsetAsync(b->d_blob + k.off_count + sizeof(int), 0, sizeof(int), st);
                if (e == cudaSuccess)
                    e = wdf::launch_explain_batch(k.D, reinterpret_cast<const wdf::ExplainJob *>(b->d_blob + k.off_jobs),
                                                  reinterpret_cast<const wdf::BatchRequest *>(b->d_blob + k.off_reqs),
                                                  reinterpret_cast<const int4 *>(b->d_blob + k.off_items),
                                                  reinterpret_cast<int *>(b->d_blob + k.off_count), k.F_max, k.xb_max, tc,
                                                  0, b->ctx->dev, st);
            }
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                s = fail(WDF_ECUDA, std::string("autotune: ") + cudaGetErrorString(e));
                break;
            }
            ms /= (float)reps;
            if (ms < best_ms) {
                best_ms = ms;
                best = tc;
            }
        }
        if (s != WDF_OK) break;
        k.tile_rows = best;
        if (log.is_open()) log << k.D << " " << fkey << " " << xkey << " " << best << " " << best_ms << "\n";
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    drop_graph(b);  // recaptured with the chosen tile sizes on the next explain
    if (prev >= 0 && prev != b->ctx->device) cudaSetDevice(prev);
    return s;
}

wdf_status wdf_batch_tile_rows(const wdf_batch *b, int32_t depth, int32_t *tile_rows) {
    if (!b || !tile_rows) return fail(WDF_EINVAL, "null argument");
    *tile_rows = -1;
    for (const Cls &k : b->cls)
        if (k.D == depth) *tile_rows = k.tile_rows;
    return WDF_OK;
}

}  // extern "C"
