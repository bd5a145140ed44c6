// Global attribution: per-feature means of |phi| and phi over many explained rows,
// accumulated in FP64 (the paper's global attribution combines many local
// attributions, section "Introduction").  Two passes with a fixed summation order, so
// the result does not depend on scheduling: row blocks write FP64 partial sums, then
// one thread per feature adds the partials in block order.
#include <algorithm>
#include <cstdint>

#include "launch.h"

namespace wdf {

constexpr int kRowsPerBlock = 4096;

int64_t global_attr_blocks(int64_t n) { return std::max<int64_t>(1, (n + kRowsPerBlock - 1) / kRowsPerBlock); }

int64_t global_attr_partial_doubles(int64_t n, int F) { return global_attr_blocks(n) * (int64_t)F * 2; }

// block (32, 8): column f = 32 * blockIdx.y + threadIdx.x, row sub-lane threadIdx.y.
// The general form (any row stride and alignment).
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

// Packed rows (row stride F, 16-byte aligned) with F <= kVecMaxF: the block's rows are
// one flat run of floats read as float4.  Threads = F * c, so 4 * threads is a multiple
// of F and thread t always meets features (4t + j) mod F, j = 0..3.  Each thread sums
// runs of kRun of its float4s as unevaluated FP32 pairs (hi + lo, hi updated by an
// error-free TwoSum, lo collecting the errors: the pair's sum is within 2^-42 of the
// run's exact sum, relative to its largest partial sum), then adds hi and lo to its FP64
// sums; a feature's partial is the sum of its 4c thread slots in a fixed order.  FP64 adds
// run at a small fraction of the FP32 rate on this GPU, so this takes one FP64 add per
// element where the general form takes two plus a conversion.
constexpr int kVecMaxF = 512;
constexpr int kRun = 8;

__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float x) {
    const float s = hi + x;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (x - bp);
    hi = s;
}

__global__ void __launch_bounds__(kVecMaxF) k_colsum_vec(const float *__restrict__ phi, int64_t n, int F,
                                                          double *__restrict__ partial) {
    __shared__ double sa[4 * kVecMaxF], ss[4 * kVecMaxF];
    const int NT = blockDim.x, t = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * kRowsPerBlock;
    const int64_t r1 = (n < r0 + kRowsPerBlock) ? n : r0 + kRowsPerBlock;
    const float *base = phi + r0 * F;  // 16-byte aligned: r0 is a multiple of 4
    const int64_t nel = (r1 - r0) * F, nq = nel / 4;
    const float4 *b4 = reinterpret_cast<const float4 *>(base);
    double A[4] = {0.0, 0.0, 0.0, 0.0}, S[4] = {0.0, 0.0, 0.0, 0.0};
    int64_t q = t;
    for (; q + (int64_t)(kRun - 1) * NT < nq; q += (int64_t)kRun * NT) {
        float4 v[kRun];
#pragma unroll
        for (int k = 0; k < kRun; ++k) v[k] = __ldg(b4 + q + (int64_t)k * NT);
        float ah[4] = {0.f, 0.f, 0.f, 0.f}, al[4] = {0.f, 0.f, 0.f, 0.f};
        float sh[4] = {0.f, 0.f, 0.f, 0.f}, sl[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < kRun; ++k) {
            const float x[4] = {v[k].x, v[k].y, v[k].z, v[k].w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                two_sum_acc(ah[j], al[j], fabsf(x[j]));
                two_sum_acc(sh[j], sl[j], x[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            A[j] += (double)ah[j];
            A[j] += (double)al[j];
            S[j] += (double)sh[j];
            S[j] += (double)sl[j];
        }
    }
    for (; q < nq; q += NT) {
        const float4 v = __ldg(b4 + q);
        const float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            A[j] += fabs((double)x[j]);
            S[j] += (double)x[j];
        }
    }
    // the last (nel mod 4) elements belong to the slots of the thread that owns float4 nq
    if (t == (int)(nq % NT)) {
        const int tail = (int)(nel - 4 * nq);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            if (j < tail) {
                const double x = (double)__ldg(base + 4 * nq + j);
                A[j] += fabs(x);
                S[j] += x;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        sa[4 * t + j] = A[j];
        ss[4 * t + j] = S[j];
    }
    __syncthreads();
    const int c4 = 4 * NT / F;
    for (int f = t; f < F; f += NT) {
        double ta = 0.0, ts = 0.0;
        for (int i = 0; i < c4; ++i) {
            ta += sa[f + F * i];
            ts += ss[f + F * i];
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
    const int64_t nb64 = global_attr_blocks(n);
    if (nb64 > 0x7FFFFFFF) return cudaErrorInvalidValue;
    const int nb = (int)nb64;
    if (n > 0) {
        if (ldp == F && F <= kVecMaxF && (reinterpret_cast<uintptr_t>(phi) & 15) == 0) {
            const int threads = F * std::max(1, 256 / F);
            k_colsum_vec<<<nb, threads, 0, st>>>(phi, n, F, partial);
        } else {
            dim3 grid(nb, (F + 31) / 32);
            k_colsum_partial<<<grid, dim3(32, 8), 0, st>>>(phi, n, ldp, F, partial);
        }
        count_launches(1);
        cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    }
    k_colsum_final<<<(F + 127) / 128, 128, 0, st>>>(partial, n > 0 ? nb : 0, F, n, mean_abs, mean);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace wdf
