// Consumer side of Algorithm 3, step 4 (Eq. "bg_shap_derivation" step (g)):
// phi[c, i] = sum over trees and leaves of s_{l,i}[P[l][c]].
//
// One thread per consumer row.  The block stages its rows feature-major in shared
// memory together with a per-row phi accumulator of the same shape.  Per tree the
// thread evaluates the inner nodes (decision bitmask in registers), forms its entry at
// every live bottom subtree, and gathers one slot vector per subtree from the folded
// table: the slots of the subtree's three inner nodes go straight into phi[feature of
// the node]; the slots of the nodes above accumulate in registers (one per node, the
// node-level form of the NumPy indexing of section "Algorithmic Improvements" item 6)
// and are added into phi once per tree.  The order of every floating-point addition
// into a row's phi depends only on the ensemble, never on which rows share a block.
#include <algorithm>

#include "launch.h"
#include "wdf_device.cuh"

namespace wdf {

template <int D, int TC>
__global__ void __launch_bounds__(TC) k_explain(const float *__restrict__ C, int64_t n, int64_t ldc, int F,
                                                const int2 *__restrict__ nodes, const uint64_t *__restrict__ live,
                                                const float *__restrict__ sfold, int T, float *__restrict__ phi,
                                                int64_t ldp) {
    using S = Shape<D>;
    constexpr int XS = TC + 1;
    constexpr int NA = S::NS > 1 ? S::NS - 1 : 1;
    extern __shared__ __align__(16) float smem[];
    float *sx = smem;
    float *sp = smem + (size_t)(F + 1) * XS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t c0 = (int64_t)blockIdx.x * TC;
    for (int r = warp; r < TC; r += TC / 32) {
        const int64_t row = c0 + r;
        const float *src = C + row * ldc;
        for (int f = lane; f < F; f += 32) sx[f * XS + r] = (row < n) ? __ldg(src + f) : 0.0f;
    }
    for (int i = tid; i < (F + 1) * XS; i += TC) sp[i] = 0.0f;
    sx[F * XS + tid] = 0.0f;
    __syncthreads();
    float *myphi = sp + tid;
    for (int t = 0; t < T; ++t) {
        const int2 *tn = nodes + (size_t)t * S::NI;
        uint32_t dm[S::NW];
        tree_decisions<D>(tn, sx, XS, tid, dm);
        uint32_t ent[S::NS];
        subtree_entries<D>(dm, ent);
        const uint64_t lv = __ldg(live + t);
        const float *tf = sfold + (size_t)t * S::NS * S::E * S::SP;
        float acc[NA];
#pragma unroll
        for (int a = 0; a < NA; ++a) acc[a] = 0.0f;
#pragma unroll
        for (int s = 0; s < S::NS; ++s) {
            if ((lv >> s) & 1ull) {
                const float4 *src = reinterpret_cast<const float4 *>(tf + ((size_t)s * S::E + ent[s]) * S::SP);
                float v[S::SP];
#pragma unroll
                for (int k = 0; k < S::SP / 4; ++k) {
                    const float4 q = __ldg(src + k);
                    v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
                }
                const int r = S::NS - 1 + s;
#pragma unroll
                for (int k = 0; k < D - 2; ++k) acc[((r + 1) >> (D - 2 - k)) - 1] += v[k];
                myphi[__ldg(&tn[r].x) * XS] += v[D - 2];
                myphi[__ldg(&tn[2 * r + 1].x) * XS] += v[D - 1];
                myphi[__ldg(&tn[2 * r + 2].x) * XS] += v[D];
            }
        }
        if (S::NS > 1) {
#pragma unroll
            for (int a = 0; a < S::NS - 1; ++a) myphi[__ldg(&tn[a].x) * XS] += acc[a];
        }
    }
    __syncthreads();
    for (int r = warp; r < TC; r += TC / 32) {
        const int64_t row = c0 + r;
        if (row >= n) break;
        float *dst = phi + row * ldp;
        for (int f = lane; f < F; f += 32) dst[f] = sp[f * XS + r];
    }
}

template <int D, int TC>
static cudaError_t explain_t(const float *C, int64_t n, int64_t ldc, int F, const int2 *nodes, const uint64_t *live,
                             const float *sfold, int T, float *phi, int64_t ldp, const DevInfo &dev, cudaStream_t st) {
    const size_t smem = 2 * (size_t)(F + 1) * (TC + 1) * sizeof(float);
    if (smem > dev.smem_optin) return cudaErrorInvalidConfiguration;
    auto kern = k_explain<D, TC>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    const int64_t blocks = (n + TC - 1) / TC;
    kern<<<(unsigned)blocks, TC, smem, st>>>(C, n, ldc, F, nodes, live, sfold, T, phi, ldp);
    count_launches(1);
    return cudaGetLastError();
}

template <int D>
static cudaError_t explain_d(const float *C, int64_t n, int64_t ldc, int F, const int2 *nodes, const uint64_t *live,
                             const float *sfold, int T, float *phi, int64_t ldp, const DevInfo &dev, cudaStream_t st) {
    if (2 * (size_t)(F + 1) * 65 * 4 <= dev.smem_optin / 2)
        return explain_t<D, 64>(C, n, ldc, F, nodes, live, sfold, T, phi, ldp, dev, st);
    return explain_t<D, 32>(C, n, ldc, F, nodes, live, sfold, T, phi, ldp, dev, st);
}

cudaError_t launch_explain(int D, const float *C, int64_t n, int64_t ldc, int F, const int2 *nodes,
                           const uint64_t *live, const float *sfold, int T, float *phi, int64_t ldp,
                           const DevInfo &dev, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    switch (D) {
        case 2: return explain_d<2>(C, n, ldc, F, nodes, live, sfold, T, phi, ldp, dev, st);
        case 3: return explain_d<3>(C, n, ldc, F, nodes, live, sfold, T, phi, ldp, dev, st);
        case 4: return explain_d<4>(C, n, ldc, F, nodes, live, sfold, T, phi, ldp, dev, st);
        case 5: return explain_d<5>(C, n, ldc, F, nodes, live, sfold, T, phi, ldp, dev, st);
        case 6: return explain_d<6>(C, n, ldc, F, nodes, live, sfold, T, phi, ldp, dev, st);
        case 7: return explain_d<7>(C, n, ldc, F, nodes, live, sfold, T, phi, ldp, dev, st);
        case 8: return explain_d<8>(C, n, ldc, F, nodes, live, sfold, T, phi, ldp, dev, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace wdf
