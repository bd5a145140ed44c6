// Decision codes (tree_layout.h) of a block of rows, in the 32-row code-block layout the
// decision kernels stage (wdf_device.cuh).
#include "launch.h"
#include "wdf_device.cuh"

namespace wdf {

// Decision codes of rows [0, rows) of X into code blocks (wdf_device.cuh): element
// (block, column c, row r of block) at ((block * n_cols + c) * 32 + r) * code bytes.
// One thread block per 32-row code block: for every run of kEncodeCols columns the
// rows' values of the columns' features are read into shared memory (a warp reads
// along a row), then each warp encodes whole columns (lane = row).  Rows from rows to
// the end of the last block get code 0 (never counted).
constexpr int kEncodeThreads = 256;
constexpr int kEncodeCols = 128;  // 16.5 KB of staging: fits beside a counting block

// Code block `block` (rows 32 block .. 32 block + 31) of rows [0, rows) of X, written at
// codes + block * n_cols * 32 * code bytes.  xs: 32 x (kEncodeCols + 1) floats of shared
// memory.  All threads of the block call it.
__device__ __forceinline__ void encode_block(const float *__restrict__ X, int64_t rows, int64_t ldx,
                                             const TreeArrays &ta, int64_t block, unsigned char *__restrict__ codes,
                                             float *xs) {
    const int ncol = ta.n_cols, cb = ta.code_bytes;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t row0 = block * 32;
    const bool valid = row0 + lane < rows;
    unsigned char *dst = codes + (size_t)block * ncol * 32 * cb;
    for (int c0 = 0; c0 < ncol; c0 += kEncodeCols) {
        const int cn = min(kEncodeCols, ncol - c0);
        __syncthreads();
        for (int r = warp; r < 32; r += kEncodeThreads / 32) {
            const int64_t row = row0 + r;
            for (int c = lane; c < cn; c += 32) {
                const int f = __ldg(&ta.cols[c0 + c].feature);
                xs[r * (kEncodeCols + 1) + c] = row < rows ? __ldg(X + row * ldx + f) : 0.0f;
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int c = warp; c < cn; c += kEncodeThreads / 32) {
            const int4 cv = __ldg(reinterpret_cast<const int4 *>(ta.cols) + c0 + c);
            const CodeCol col{cv.x, cv.y, cv.z, cv.w};
            const float x = xs[lane * (kEncodeCols + 1) + c];
            if (cb == 1) {
                // binary search from the column's top power of two (the same for the whole
                // warp) over its 255 padded entries: NaN padding is never <= x, so no bound
                // checks; a NaN x gets the count, as in decision_code
                const float *u = ta.col_thr + col.first;
                int pos = 0;
                for (int step = col.top; step > 0; step >>= 1) pos += __ldg(u + pos + step - 1) <= x ? step : 0;
                const int code = !valid ? 0 : (x != x ? col.count : pos);
                dst[(size_t)(c0 + c) * 32 + lane] = (unsigned char)code;
            } else {
                const int code = valid ? decision_code(x, ta.col_thr + col.first, col) : 0;
                reinterpret_cast<uint16_t *>(dst)[(size_t)(c0 + c) * 32 + lane] = (uint16_t)code;
            }
        }
    }
}

__global__ void __launch_bounds__(kEncodeThreads) k_encode_codes(const float *__restrict__ X, int64_t rows,
                                                                int64_t ldx, TreeArrays ta,
                                                                unsigned char *__restrict__ codes) {
    __shared__ float xs[32 * (kEncodeCols + 1)];
    encode_block(X, rows, ldx, ta, blockIdx.x, codes, xs);
}

// The rows of a ragged batch: item i = (request, 32-row block); blocks walk the items.
__global__ void __launch_bounds__(kEncodeThreads) k_encode_batch(const ExplainJob *__restrict__ jobs,
                                                                const BatchRequest *__restrict__ reqs,
                                                                const int2 *__restrict__ items,
                                                                const int *__restrict__ n_items) {
    __shared__ float xs[32 * (kEncodeCols + 1)];
    const int count = n_items[0];
    for (int i = blockIdx.x; i < count; i += gridDim.x) {
        const int2 it = items[i];
        const BatchRequest rq = reqs[it.x];
        const TreeArrays ta = jobs[rq.job].ta;
        encode_block(rq.C, rq.n, rq.ldc, ta, it.y, rq.codes, xs);
    }
}

cudaError_t launch_encode_batch(const ExplainJob *jobs, const BatchRequest *reqs, const int2 *items,
                                const int *n_items, int grid, cudaStream_t st) {
    k_encode_batch<<<grid, kEncodeThreads, 0, st>>>(jobs, reqs, items, n_items);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_encode_codes(const float *X, int64_t rows, int64_t ldx, const TreeArrays &ta, int64_t rows_pad,
                                unsigned char *codes, cudaStream_t st) {
    const int64_t blocks = rows_pad / 32;
    if (blocks == 0) return cudaSuccess;
    k_encode_codes<<<(unsigned)blocks, kEncodeThreads, 0, st>>>(X, rows, ldx, ta, codes);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace wdf
