// Global attribution: per-feature means of |phi| and phi over many explained rows,
// accumulated in FP64 (the paper's global attribution combines many local
// attributions, section "Introduction").  Two passes with a fixed summation order, so
// the result does not depend on scheduling: row blocks write FP64 partial sums, then
// one thread per feature adds the partials in block order.
#include <algorithm>

#include "launch.h"

namespace wdf {

constexpr int kRowsPerBlock = 4096;

int global_attr_blocks(int64_t n) { return (int)std::max<int64_t>(1, (n + kRowsPerBlock - 1) / kRowsPerBlock); }

// block (32, 8): column f = 32 * blockIdx.y + threadIdx.x, row sub-lane threadIdx.y.
__global__ void __launch_bounds__(256) k_colsum_partial(const float *__restrict__ phi, int64_t n, int64_t ldp, int F,
                                                        double *__restrict__ partial) {
    __shared__ double sa[8][32], ss[8][32];
    const int f = blockIdx.y * 32 + threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * kRowsPerBlock;
    const int64_t r1 = (n < r0 + kRowsPerBlock) ? n : r0 + kRowsPerBlock;
    double a = 0.0, s = 0.0;
    if (f < F) {
        for (int64_t r = r0 + threadIdx.y; r < r1; r += 8) {
            const double v = (double)__ldg(phi + r * ldp + f);
            a += fabs(v);
            s += v;
        }
    }
    sa[threadIdx.y][threadIdx.x] = a;
    ss[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && f < F) {
        double ta = 0.0, ts = 0.0;
        for (int k = 0; k < 8; ++k) {
            ta += sa[k][threadIdx.x];
            ts += ss[k][threadIdx.x];
        }
        partial[((size_t)blockIdx.x * F + f) * 2 + 0] = ta;
        partial[((size_t)blockIdx.x * F + f) * 2 + 1] = ts;
    }
}

__global__ void k_colsum_final(const double *__restrict__ partial, int nb, int F, int64_t n,
                               double *__restrict__ mean_abs, double *__restrict__ mean) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    double ta = 0.0, ts = 0.0;
    for (int b = 0; b < nb; ++b) {
        ta += partial[((size_t)b * F + f) * 2 + 0];
        ts += partial[((size_t)b * F + f) * 2 + 1];
    }
    const double inv = n > 0 ? 1.0 / (double)n : 0.0;
    mean_abs[f] = ta * inv;
    mean[f] = ts * inv;
}

cudaError_t launch_global_attr(const float *phi, int64_t n, int64_t ldp, int F, double *partial, double *mean_abs,
                               double *mean, cudaStream_t st) {
    const int nb = global_attr_blocks(n);
    if (n > 0) {
        dim3 grid(nb, (F + 31) / 32);
        k_colsum_partial<<<grid, dim3(32, 8), 0, st>>>(phi, n, ldp, F, partial);
        count_launches(1);
        cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    }
    k_colsum_final<<<(F + 127) / 128, 128, 0, st>>>(partial, n > 0 ? nb : 0, F, n, mean_abs, mean);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace wdf
