// Depth and tile dispatch of the consumer kernels (k_explain.cuh); the kernels are
// compiled in the k_explain_d*.cu translation units.
#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

#include "k_explain.cuh"

namespace wdf {

namespace {
std::mutex g_tmu;
bool g_timing = false;
std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_tev;

void drop_events() {
    for (auto &p : g_tev) {
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
    }
    g_tev.clear();
}
}  // namespace

void explain_timing(bool on) {
    std::lock_guard<std::mutex> lk(g_tmu);
    drop_events();
    g_timing = on;
}

cudaError_t explain_timing_read(double *ms, int64_t *launches) {
    std::lock_guard<std::mutex> lk(g_tmu);
    double total = 0.0;
    cudaError_t err = cudaSuccess;
    for (auto &p : g_tev) {
        float t = 0.0f;
        if (err == cudaSuccess) err = cudaEventSynchronize(p.second);
        if (err == cudaSuccess) err = cudaEventElapsedTime(&t, p.first, p.second);
        total += t;
    }
    *ms = total;
    *launches = (int64_t)g_tev.size();
    drop_events();
    return err;
}

WDF_EXPLAIN_DEPTH(2, extern)
WDF_EXPLAIN_DEPTH(3, extern)
WDF_EXPLAIN_DEPTH(4, extern)
WDF_EXPLAIN_DEPTH(5, extern)
WDF_EXPLAIN_DEPTH(6, extern)
WDF_EXPLAIN_DEPTH(7, extern)
WDF_EXPLAIN_DEPTH(8, extern)

template <int D>
static cudaError_t explain_depth(const unsigned char *codes, int64_t n, const ExplainJob &job, float *phi,
                                 int64_t ldp, int tile_rows, const DevInfo &dev, cudaStream_t st) {
    switch (tile_rows) {
        case 32: return explain_t<D, 32>(codes, n, job, phi, ldp, dev, st);
        case 128: return explain_t<D, 128>(codes, n, job, phi, ldp, dev, st);
        default: return explain_t<D, 64>(codes, n, job, phi, ldp, dev, st);
    }
}

template <int D>
static cudaError_t batch_depth(const ExplainJob *jobs, const BatchRequest *reqs, const int4 *items, int *n_items,
                               int F_max, int xb_max, int tile_rows, int grid, const DevInfo &dev, cudaStream_t st) {
    switch (tile_rows) {
        case 32: return batch_t<D, 32>(jobs, reqs, items, n_items, F_max, xb_max, grid, dev, st);
        case 128: return batch_t<D, 128>(jobs, reqs, items, n_items, F_max, xb_max, grid, dev, st);
        default: return batch_t<D, 64>(jobs, reqs, items, n_items, F_max, xb_max, grid, dev, st);
    }
}

int default_tile_rows(int D, int F, int xb, const DevInfo &dev) {
    const size_t s64 = explain_smem_bytes(D, F, xb, 64);
    return s64 <= dev.smem_optin / 2 ? 64 : 32;
}

// Rows per encoded chunk: the decision codes of a chunk live in a stream-ordered
// scratch allocation (so concurrent calls on other streams never share it).
constexpr int64_t kExplainChunkRows = 1 << 20;

cudaError_t launch_explain(int D, const float *C, int64_t n, int64_t ldc, const ExplainJob &job, float *phi,
                           int64_t ldp, int tile_rows, const DevInfo &dev, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    if (D < 2 || D > 8) return cudaErrorInvalidValue;
    const int xb = job.ta.n_cols * job.ta.code_bytes;
    if (tile_rows <= 0) tile_rows = default_tile_rows(D, job.F, xb, dev);
    const int64_t chunk = std::min(n, kExplainChunkRows);
    const int64_t pad = 128;  // every tile size divides it
    unsigned char *codes = nullptr;
    cudaError_t err = cudaMallocAsync(reinterpret_cast<void **>(&codes), (size_t)((chunk + pad - 1) / pad * pad) * xb,
                                      st);
    if (err != cudaSuccess) return err;
    for (int64_t r0 = 0; r0 < n && err == cudaSuccess; r0 += chunk) {
        const int64_t rows = std::min(chunk, n - r0);
        err = launch_encode_codes(C + r0 * ldc, rows, ldc, job.ta, (rows + pad - 1) / pad * pad, codes, st);
        if (err != cudaSuccess) break;
        float *out = phi + r0 * ldp;
        cudaEvent_t ev0 = nullptr, ev1 = nullptr;
        {
            std::lock_guard<std::mutex> lk(g_tmu);
            if (g_timing && cudaEventCreate(&ev0) == cudaSuccess) {
                if (cudaEventCreate(&ev1) == cudaSuccess) {
                    cudaEventRecord(ev0, st);
                } else {
                    cudaEventDestroy(ev0);
                    ev0 = ev1 = nullptr;
                }
            }
        }
        switch (D) {
            case 2: err = explain_depth<2>(codes, rows, job, out, ldp, tile_rows, dev, st); break;
            case 3: err = explain_depth<3>(codes, rows, job, out, ldp, tile_rows, dev, st); break;
            case 4: err = explain_depth<4>(codes, rows, job, out, ldp, tile_rows, dev, st); break;
            case 5: err = explain_depth<5>(codes, rows, job, out, ldp, tile_rows, dev, st); break;
            case 6: err = explain_depth<6>(codes, rows, job, out, ldp, tile_rows, dev, st); break;
            case 7: err = explain_depth<7>(codes, rows, job, out, ldp, tile_rows, dev, st); break;
            default: err = explain_depth<8>(codes, rows, job, out, ldp, tile_rows, dev, st); break;
        }
        if (ev1) {  // the pair is kept only once both ends are recorded
            std::lock_guard<std::mutex> lk(g_tmu);
            cudaEventRecord(ev1, st);
            g_tev.emplace_back(ev0, ev1);
        }
    }
    const cudaError_t ferr = cudaFreeAsync(codes, st);
    return err != cudaSuccess ? err : ferr;
}

cudaError_t launch_explain_batch(int D, const ExplainJob *jobs, const BatchRequest *reqs, const int4 *items,
                                 int *n_items, int F_max, int xb_max, int tile_rows, int grid, const DevInfo &dev,
                                 cudaStream_t st) {
    switch (D) {
        case 2: return batch_depth<2>(jobs, reqs, items, n_items, F_max, xb_max, tile_rows, grid, dev, st);
        case 3: return batch_depth<3>(jobs, reqs, items, n_items, F_max, xb_max, tile_rows, grid, dev, st);
        case 4: return batch_depth<4>(jobs, reqs, items, n_items, F_max, xb_max, tile_rows, grid, dev, st);
        case 5: return batch_depth<5>(jobs, reqs, items, n_items, F_max, xb_max, tile_rows, grid, dev, st);
        case 6: return batch_depth<6>(jobs, reqs, items, n_items, F_max, xb_max, tile_rows, grid, dev, st);
        case 7: return batch_depth<7>(jobs, reqs, items, n_items, F_max, xb_max, tile_rows, grid, dev, st);
        case 8: return batch_depth<8>(jobs, reqs, items, n_items, F_max, xb_max, tile_rows, grid, dev, st);
        default: return cudaErrorInvalidValue;
    }
}

size_t explain_smem_bytes(int D, int F, int xb, int tile_rows) {
    switch (D * 1000 + tile_rows) {
#define WDF_SMEM_CASE(d, tc) \
    case d * 1000 + tc: return ExLayout<d>(F, xb, tc).total;
        WDF_SMEM_CASE(2, 32) WDF_SMEM_CASE(2, 64) WDF_SMEM_CASE(2, 128)
        WDF_SMEM_CASE(3, 32) WDF_SMEM_CASE(3, 64) WDF_SMEM_CASE(3, 128)
        WDF_SMEM_CASE(4, 32) WDF_SMEM_CASE(4, 64) WDF_SMEM_CASE(4, 128)
        WDF_SMEM_CASE(5, 32) WDF_SMEM_CASE(5, 64) WDF_SMEM_CASE(5, 128)
        WDF_SMEM_CASE(6, 32) WDF_SMEM_CASE(6, 64) WDF_SMEM_CASE(6, 128)
        WDF_SMEM_CASE(7, 32) WDF_SMEM_CASE(7, 64) WDF_SMEM_CASE(7, 128)
        WDF_SMEM_CASE(8, 32) WDF_SMEM_CASE(8, 64) WDF_SMEM_CASE(8, 128)
#undef WDF_SMEM_CASE
        default: return (size_t)-1;
    }
}

}  // namespace wdf
