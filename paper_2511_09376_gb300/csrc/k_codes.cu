// Decision codes (tree_layout.h) of a block of rows, in the 32-row code-block layout the
// decision kernels stage (wdf_device.cuh).
#include <algorithm>

#include "launch.h"
#include "wdf_device.cuh"

namespace wdf {

// Decision codes of rows [0, rows) of X into code blocks (wdf_device.cuh):
// element (block, column c, row r of block) at ((block * n_cols + c) * 32 + r) * code
// bytes.  Rows from rows to rows_pad (a multiple of 32) get code 0 (never counted).
__global__ void k_encode_codes(const float *__restrict__ X, int64_t rows, int64_t ldx, TreeArrays ta,
                               int64_t rows_pad, unsigned char *__restrict__ codes) {
    const int ncol = ta.n_cols, cb = ta.code_bytes;
    const int64_t total = rows_pad * ncol;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx & 31);
        const int64_t rest = idx >> 5;
        const int c = (int)(rest % ncol);
        const int64_t row = (rest / ncol) * 32 + r;
        const int4 cv = __ldg(reinterpret_cast<const int4 *>(ta.cols) + c);
        const CodeCol col{cv.x, cv.y, cv.z, cv.w};
        const int code = row < rows ? decision_code(__ldg(X + row * ldx + col.feature), ta.col_thr + col.first, col) : 0;
        if (cb == 1)
            codes[idx] = (unsigned char)code;
        else
            reinterpret_cast<uint16_t *>(codes)[idx] = (uint16_t)code;
    }
}

cudaError_t launch_encode_codes(const float *X, int64_t rows, int64_t ldx, const TreeArrays &ta, int64_t rows_pad,
                                unsigned char *codes, const DevInfo &dev, cudaStream_t st) {
    const int64_t total = rows_pad * ta.n_cols;
    if (total == 0) return cudaSuccess;
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((total + threads - 1) / threads, (int64_t)dev.sms * 16);
    k_encode_codes<<<(unsigned)blocks, threads, 0, st>>>(X, rows, ldx, ta, rows_pad, codes);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace wdf
