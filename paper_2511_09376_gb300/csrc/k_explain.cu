// Consumer side of Algorithm 3, step 4 (Eq. "bg_shap_derivation" step (g)):
// phi[c, i] = sum over trees and leaves of s_{l,i}[P[l][c]].
//
// One thread per consumer row.  The block stages its rows feature-major in shared
// memory together with a per-row phi accumulator of the same shape, and the real
// inner nodes of a chunk of trees.  Per tree the thread evaluates those nodes
// (decision bitmask in registers), forms its entry at every bottom subtree, and
// gathers one slot vector per subtree from the folded table -- all gathers of a tree
// are issued before any is used, so their L2 latency overlaps; a dead subtree reads a
// zero row instead.  The slots of the subtree's three inner nodes go straight into
// phi[feature of the node]; the slots of the nodes above accumulate in registers (one
// per node, the node-level form of the NumPy indexing of section "Algorithmic
// Improvements" item 6) and are added into phi once per tree.  Pass-through nodes
// carry nothing and are skipped.  The order of every floating-point addition into a
// row's phi depends only on the ensemble, never on which rows share a block.
#include <algorithm>
#include <cstdlib>

#include "launch.h"
#include "wdf_device.cuh"

namespace wdf {

template <int D>
struct ExplainCfg {
    static constexpr int TCH = 8;  // trees per shared-memory chunk
    // bottom subtrees gathered together: the largest power of two (a divisor of NS) whose
    // slot vectors fit in 128 registers
    static constexpr int gs(int g) { return (g > 1 && g * Shape<D>::SP > 128) ? gs(g / 2) : g; }
    static constexpr int GS = gs(Shape<D>::NS);
    static_assert(Shape<D>::NS % GS == 0, "gather groups must tile the bottom subtrees");
};

template <int D>
struct ExLayout {
    size_t x, meta, rn, fo, f3, total;
    static __host__ __device__ size_t up(size_t v) { return (v + 15) & ~(size_t)15; }
    __host__ __device__ ExLayout(int F, int TC) {
        x = up((size_t)(F + 1) * (TC + 1) * 4);  // one of x and phi
        meta = up((size_t)ExplainCfg<D>::TCH * sizeof(TreeMeta));
        rn = up((size_t)ExplainCfg<D>::TCH * Shape<D>::NI * sizeof(int2));
        fo = up((size_t)ExplainCfg<D>::TCH * Shape<D>::NI * sizeof(int));
        f3 = up((size_t)ExplainCfg<D>::TCH * Shape<D>::NS * sizeof(int4));
        total = 2 * x + meta + rn + fo + f3;
    }
};

__device__ __forceinline__ float4 ldg_f4(const float4 *p) {
    float4 r;
    asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                 : "l"(p));
    return r;
}

// One 32-byte entry in a single 256-bit load (the address is 32-byte aligned).
__device__ __forceinline__ void ldg_f8(const float4 *p, float4 &a, float4 &b) {
    asm volatile("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
                 : "l"(p));
}

// One tile of TC consumer rows starting at row c0 of C (n rows), for one ensemble.
template <int D, int TC>
__device__ __forceinline__ void explain_tile(const ExplainJob &job, const float *__restrict__ C, int64_t n,
                                             int64_t ldc, float *__restrict__ phi, int64_t ldp, int64_t c0,
                                             unsigned char *smem_raw) {
    using S = Shape<D>;
    using X = ExplainCfg<D>;
    constexpr int XS = TC + 1;
    constexpr int NA = S::NS > 1 ? S::NS - 1 : 1;
    constexpr int GS = X::GS;
    constexpr int Q = S::SP / 4;
    const int F = job.F, T = job.T;
    const TreeArrays &ta = job.ta;
    const float *__restrict__ sfold = job.sfold;
    const ExLayout<D> L(F, TC);
    float *sx = reinterpret_cast<float *>(smem_raw);
    float *sp = reinterpret_cast<float *>(smem_raw + L.x);
    TreeMeta *smeta = reinterpret_cast<TreeMeta *>(smem_raw + 2 * L.x);
    int2 *srn = reinterpret_cast<int2 *>(smem_raw + 2 * L.x + L.meta);
    int *sfo = reinterpret_cast<int *>(smem_raw + 2 * L.x + L.meta + L.rn);
    int *sf3 = reinterpret_cast<int *>(smem_raw + 2 * L.x + L.meta + L.rn + L.fo);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int r = warp; r < TC; r += TC / 32) {
        const int64_t row = c0 + r;
        const float *src = C + row * ldc;
        for (int f = lane; f < F; f += 32) sx[f * XS + r] = (row < n) ? __ldg(src + f) : 0.0f;
    }
    for (int i = tid; i < (F + 1) * XS; i += TC) sp[i] = 0.0f;
    sx[F * XS + tid] = 0.0f;
    float *myphi = sp + tid;
    const float4 *z4 = reinterpret_cast<const float4 *>(job.zero);
    for (int tc0 = 0; tc0 < T; tc0 += X::TCH) {
        const int tcn = min(X::TCH, T - tc0);
        __syncthreads();
        stage_trees<D>(tc0, tcn, XS, ta.nodes, ta.rn_key, ta.rn_thr, ta.rn_count, ta.pt_mask, ta.live, srn, sfo,
                       smeta, tid, TC);
        __syncthreads();
        // phi offsets of the three inner nodes of every bottom subtree, one 128-bit word each
        for (int i = tid; i < tcn * S::NS; i += TC) {
            const int g = i / S::NS, r = S::NS - 1 + (i % S::NS);
            const int *fo = sfo + g * S::NI;
            reinterpret_cast<int4 *>(sf3)[i] = make_int4(fo[r], fo[2 * r + 1], fo[2 * r + 2], 0);
        }
        __syncthreads();
        for (int g = 0; g < tcn; ++g) {
            const int t = tc0 + g;
            const TreeMeta &mt = smeta[g];
            const int *fo = sfo + g * S::NI;
            const int4 *fs3 = reinterpret_cast<const int4 *>(sf3 + (size_t)g * S::NS * 4);
            uint64_t dm[S::NW];
            tree_decisions<D>(srn + g * S::NI, mt, sx, tid, dm);
            uint32_t ent[S::NS];
            subtree_entries<D>(dm, ent);
            const uint64_t lv = mt.live;
            const float4 *tf = reinterpret_cast<const float4 *>(sfold + (size_t)t * S::NS * S::E * S::SP);
            float acc[NA];
#pragma unroll
            for (int a = 0; a < NA; ++a) acc[a] = 0.0f;
#pragma unroll
            for (int s0 = 0; s0 < S::NS; s0 += GS) {
                const uint64_t gmask = (GS >= 64) ? ~0ull : (((1ull << GS) - 1ull) << s0);
                if (!(lv & gmask)) continue;  // every subtree of the group is dead (warp-uniform)
                float4 v[GS][Q];
#pragma unroll
                for (int j = 0; j < GS; ++j) {
                    const bool lj = (lv >> (s0 + j)) & 1ull;
                    const float4 *src = lj ? tf + ((size_t)(s0 + j) * S::E + ent[s0 + j]) * Q : z4;
                    if (Q == 2) {
                        ldg_f8(src, v[j][0], v[j][Q > 1 ? 1 : 0]);
                    } else {
#pragma unroll
                        for (int k = 0; k < Q; ++k) v[j][k] = ldg_f4(src + k);
                    }
                }
#pragma unroll
                for (int j = 0; j < GS; ++j) {
                    const int r = S::NS - 1 + s0 + j;
                    const float *vj = reinterpret_cast<const float *>(&v[j][0]);
#pragma unroll
                    for (int k = 0; k < D - 2; ++k) acc[((r + 1) >> (D - 2 - k)) - 1] += vj[k];
                    // pass-through nodes add into the scratch row, dead subtrees add zeros
                    const int4 f3 = fs3[s0 + j];
                    myphi[f3.x] += vj[D - 2];
                    myphi[f3.y] += vj[D - 1];
                    myphi[f3.z] += vj[D];
                }
            }
            if (S::NS > 1) {
#pragma unroll
                for (int a = 0; a < S::NS - 1; ++a) myphi[fo[a]] += acc[a];
            }
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
__global__ void __launch_bounds__(TC) k_explain(const float *__restrict__ C, int64_t n, int64_t ldc, ExplainJob job,
                                                float *__restrict__ phi, int64_t ldp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    explain_tile<D, TC>(job, C, n, ldc, phi, ldp, (int64_t)blockIdx.x * TC, smem_raw);
}

// Persistent form over a ragged batch: work item i is (job, request, first row).  Blocks
// claim items in order from a counter (n_items[1], zero at launch), so expensive items,
// which the host puts first, spread over the whole grid and cheap ones fill the tail.
// The item count n_items[0] is read from device memory, so one captured graph serves
// batches of any size up to its capacity.  Which block computes a tile does not change
// any row's arithmetic.
template <int D, int TC>
__global__ void __launch_bounds__(TC) k_explain_batch(const ExplainJob *__restrict__ jobs,
                                                      const BatchRequest *__restrict__ reqs,
                                                      const int4 *__restrict__ items, int *__restrict__ n_items) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int claimed;
    const int count = n_items[0];
    for (;;) {
        if (threadIdx.x == 0) claimed = atomicAdd(n_items + 1, 1);
        __syncthreads();
        const int i = claimed;
        if (i >= count) break;
        const int4 it = items[i];
        const ExplainJob job = jobs[it.x];
        const BatchRequest rq = reqs[it.y];
        const int64_t c0 = ((int64_t)it.z << 31) | (uint32_t)it.w;
        explain_tile<D, TC>(job, rq.C, rq.n, rq.ldc, rq.phi, rq.ldp, c0, smem_raw);
        __syncthreads();
    }
}

template <int D, int TC>
static cudaError_t explain_t(const float *C, int64_t n, int64_t ldc, const ExplainJob &job, float *phi, int64_t ldp,
                             const DevInfo &dev, cudaStream_t st) {
    const size_t smem = ExLayout<D>(job.F, TC).total;
    if (smem > dev.smem_optin) return cudaErrorInvalidConfiguration;
    auto kern = k_explain<D, TC>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    const int64_t blocks = (n + TC - 1) / TC;
    kern<<<(unsigned)blocks, TC, smem, st>>>(C, n, ldc, job, phi, ldp);
    count_launches(1);
    return cudaGetLastError();
}

int default_tile_rows(int D, int F, const DevInfo &dev) {
    size_t s64 = 0;
    switch (D) {
        case 2: s64 = ExLayout<2>(F, 64).total; break;
        case 3: s64 = ExLayout<3>(F, 64).total; break;
        case 4: s64 = ExLayout<4>(F, 64).total; break;
        case 5: s64 = ExLayout<5>(F, 64).total; break;
        case 6: s64 = ExLayout<6>(F, 64).total; break;
        case 7: s64 = ExLayout<7>(F, 64).total; break;
        default: s64 = ExLayout<8>(F, 64).total; break;
    }
    return s64 <= dev.smem_optin / 2 ? 64 : 32;
}

template <int D>
static cudaError_t explain_d(const float *C, int64_t n, int64_t ldc, const ExplainJob &job, float *phi, int64_t ldp,
                             int tile_rows, const DevInfo &dev, cudaStream_t st) {
    switch (tile_rows) {
        case 32: return explain_t<D, 32>(C, n, ldc, job, phi, ldp, dev, st);
        case 128: return explain_t<D, 128>(C, n, ldc, job, phi, ldp, dev, st);
        default: return explain_t<D, 64>(C, n, ldc, job, phi, ldp, dev, st);
    }
}

cudaError_t launch_explain(int D, const float *C, int64_t n, int64_t ldc, const ExplainJob &job, float *phi,
                           int64_t ldp, int tile_rows, const DevInfo &dev, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    if (tile_rows <= 0) tile_rows = default_tile_rows(D, job.F, dev);
    switch (D) {
        case 2: return explain_d<2>(C, n, ldc, job, phi, ldp, tile_rows, dev, st);
        case 3: return explain_d<3>(C, n, ldc, job, phi, ldp, tile_rows, dev, st);
        case 4: return explain_d<4>(C, n, ldc, job, phi, ldp, tile_rows, dev, st);
        case 5: return explain_d<5>(C, n, ldc, job, phi, ldp, tile_rows, dev, st);
        case 6: return explain_d<6>(C, n, ldc, job, phi, ldp, tile_rows, dev, st);
        case 7: return explain_d<7>(C, n, ldc, job, phi, ldp, tile_rows, dev, st);
        case 8: return explain_d<8>(C, n, ldc, job, phi, ldp, tile_rows, dev, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int D, int TC>
static cudaError_t batch_t(const ExplainJob *jobs, const BatchRequest *reqs, const int4 *items, int *n_items,
                           int F_max, int grid, const DevInfo &dev, cudaStream_t st) {
    const size_t smem = ExLayout<D>(F_max, TC).total;
    if (smem > dev.smem_optin) return cudaErrorInvalidConfiguration;
    auto kern = k_explain_batch<D, TC>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    if (grid <= 0) {
        int per_sm = 0;
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TC, smem);
        if (err != cudaSuccess) return err;
        grid = dev.sms * (per_sm > 0 ? per_sm : 1);
    }
    kern<<<grid, TC, smem, st>>>(jobs, reqs, items, n_items);
    count_launches(1);
    return cudaGetLastError();
}

template <int D>
static cudaError_t batch_d(const ExplainJob *jobs, const BatchRequest *reqs, const int4 *items, int *n_items,
                           int F_max, int tile_rows, int grid, const DevInfo &dev, cudaStream_t st) {
    switch (tile_rows) {
        case 32: return batch_t<D, 32>(jobs, reqs, items, n_items, F_max, grid, dev, st);
        case 128: return batch_t<D, 128>(jobs, reqs, items, n_items, F_max, grid, dev, st);
        default: return batch_t<D, 64>(jobs, reqs, items, n_items, F_max, grid, dev, st);
    }
}

cudaError_t launch_explain_batch(int D, const ExplainJob *jobs, const BatchRequest *reqs, const int4 *items,
                                 int *n_items, int F_max, int tile_rows, int grid, const DevInfo &dev,
                                 cudaStream_t st) {
    switch (D) {
        case 2: return batch_d<2>(jobs, reqs, items, n_items, F_max, tile_rows, grid, dev, st);
        case 3: return batch_d<3>(jobs, reqs, items, n_items, F_max, tile_rows, grid, dev, st);
        case 4: return batch_d<4>(jobs, reqs, items, n_items, F_max, tile_rows, grid, dev, st);
        case 5: return batch_d<5>(jobs, reqs, items, n_items, F_max, tile_rows, grid, dev, st);
        case 6: return batch_d<6>(jobs, reqs, items, n_items, F_max, tile_rows, grid, dev, st);
        case 7: return batch_d<7>(jobs, reqs, items, n_items, F_max, tile_rows, grid, dev, st);
        case 8: return batch_d<8>(jobs, reqs, items, n_items, F_max, tile_rows, grid, dev, st);
        default: return cudaErrorInvalidValue;
    }
}

size_t explain_smem_bytes(int D, int F, int tile_rows) {
    switch (D * 1000 + tile_rows) {
#define WDF_SMEM_CASE(d, tc) \
    case d * 1000 + tc: return ExLayout<d>(F, tc).total;
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
