// Background side of Algorithm 3, step 1: decision patterns of every background row
// (Algorithm 1, kept in registers) and their counts vc[l][p_b] (Eq.
// "bg_shap_derivation" step (d)); plus the per-leaf marginals and E_b f(b).
//
// K1 counts, per tree and bottom subtree, the joint entry e = (pattern at the subtree
// root, the three decisions inside the subtree) of every background row: one shared
// memory increment per (row, tree, live bottom subtree) instead of one per leaf.  The
// four leaf patterns of the subtree are functions of e, so per-leaf counts are exact
// marginals of these joint counts (the sibling-leaf observation of section
// "Algorithmic Improvements" item 3, applied two levels up).
//
// Work split: the trees are cut into chunks whose counters fit in shared memory as
// 16-bit halves of 32-bit words; blocks are numbered chunk-fastest, so the blocks that
// stage the same row tile run at the same time and share it through L2.  A block
// flushes its 16-bit counters into the global 32-bit counts before any can overflow.
#include <algorithm>
#include <cstdlib>

#include "launch.h"
#include "wdf_device.cuh"

namespace wdf {

// Shared memory layout (bytes, 16-aligned pieces): x tile | tree metadata | real-node
// lists | 16-bit counters.
template <int D>
struct BgLayout {
    size_t x, meta, rn, hist, total;
    static __host__ __device__ size_t up(size_t v) { return (v + 15) & ~(size_t)15; }
    __host__ __device__ BgLayout(int F, int RT, int G, bool smem_hist) {
        x = up((size_t)(F + 1) * (RT + 1) * 4);
        meta = up((size_t)G * sizeof(TreeMeta));
        rn = up((size_t)G * Shape<D>::NI * sizeof(int2));
        hist = smem_hist ? up((size_t)G * Shape<D>::NS * Shape<D>::E * 2) : 0;
        total = x + meta + rn + hist;
    }
};

template <int D, int RT, bool SMEM, bool AGG>
__global__ void __launch_bounds__(RT) k_bg_hist(const float *__restrict__ B, int64_t m, int64_t ldb, int F,
                                                TreeArrays ta, int T, int G, int chunks,
                                                uint32_t *__restrict__ hist) {
    using S = Shape<D>;
    constexpr int XS = RT + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const BgLayout<D> L(F, RT, G, SMEM);
    float *sx = reinterpret_cast<float *>(smem_raw);
    TreeMeta *smeta = reinterpret_cast<TreeMeta *>(smem_raw + L.x);
    int2 *srn = reinterpret_cast<int2 *>(smem_raw + L.x + L.meta);
    uint32_t *sh = reinterpret_cast<uint32_t *>(smem_raw + L.x + L.meta + L.rn);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int chunk = blockIdx.x % chunks;
    const int slice = blockIdx.x / chunks, nslices = gridDim.x / chunks;
    const int t0 = chunk * G;
    const int g_cnt = min(G, T - t0);
    const int bins = g_cnt * S::NS * S::E;  // 16-bit counters, two per word
    uint32_t *gdst = hist + (size_t)t0 * S::NS * S::E;
    stage_trees<D>(t0, g_cnt, XS, ta.nodes, ta.rn_key, ta.rn_thr, ta.rn_count, ta.pt_mask, ta.live, nullptr, srn,
                   nullptr, smeta, tid, RT);
    if (SMEM)
        for (int i = tid; i < bins / 2; i += RT) sh[i] = 0u;
    int64_t since_flush = 0;
    for (int64_t row0 = (int64_t)slice * RT; row0 < m; row0 += (int64_t)nslices * RT) {
        __syncthreads();
        if (SMEM && since_flush + RT > 65535) {  // a 16-bit counter could overflow: flush
            for (int i = tid; i < bins / 2; i += RT) {
                const uint32_t v = sh[i];
                if (v & 0xFFFFu) atomicAdd(gdst + 2 * i, v & 0xFFFFu);
                if (v >> 16) atomicAdd(gdst + 2 * i + 1, v >> 16);
                sh[i] = 0u;
            }
            since_flush = 0;
        }
        for (int r = warp; r < RT; r += RT / 32) {
            const int64_t row = row0 + r;
            const float *src = B + row * ldb;
            for (int f = lane; f < F; f += 32) sx[f * XS + r] = (row < m) ? __ldg(src + f) : 0.0f;
        }
        sx[F * XS + tid] = 0.0f;
        __syncthreads();
        since_flush += RT;
        const bool valid = row0 + tid < m;
        for (int g = 0; g < g_cnt; ++g) {
            const TreeMeta &mt = smeta[g];
            uint64_t dm[S::NW];
            tree_decisions<D>(srn + (size_t)g * S::NI, mt, sx, tid, dm);
            uint32_t ent[S::NS];
            subtree_entries<D>(dm, ent);
            const uint64_t lv = mt.live;
#pragma unroll
            for (int s = 0; s < S::NS; ++s) {
                if ((lv >> s) & 1ull) {  // warp-uniform
                    const uint32_t idx = (uint32_t)(g * S::NS + s) * S::E + ent[s];
                    if (AGG) {
                        // lanes with the same counter add once, by the lowest such lane
                        const uint32_t key = valid ? idx : 0xFFFFFFFFu;
                        const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
                        if (valid && lane == __ffs(peers) - 1) {
                            const uint32_t k = (uint32_t)__popc(peers);
                            if (SMEM)
                                atomicAdd(sh + (idx >> 1), k << ((idx & 1u) << 4));
                            else
                                atomicAdd(gdst + idx, k);
                        }
                    } else if (valid) {
                        if (SMEM)
                            atomicAdd(sh + (idx >> 1), 1u << ((idx & 1u) << 4));
                        else
                            atomicAdd(gdst + idx, 1u);
                    }
                }
            }
        }
    }
    if (SMEM) {
        __syncthreads();
        for (int i = tid; i < bins / 2; i += RT) {
            const uint32_t v = sh[i];
            if (v & 0xFFFFu) atomicAdd(gdst + 2 * i, v & 0xFFFFu);
            if (v >> 16) atomicAdd(gdst + 2 * i + 1, v >> 16);
        }
    }
}

template <int D, int RT, bool SMEM, bool AGG>
static cudaError_t bg_hist_launch(const float *B, int64_t m, int64_t ldb, int F, const TreeArrays &ta, int T, int G,
                                  size_t smem, const DevInfo &dev, uint32_t *hist, cudaStream_t st) {
    auto kern = k_bg_hist<D, RT, SMEM, AGG>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, RT, smem);
    if (err != cudaSuccess) return err;
    per_sm = std::max(per_sm, 1);
    const int chunks = (T + G - 1) / G;
    const int64_t tiles = (m + RT - 1) / RT;
    const int64_t slices = std::max<int64_t>(1, std::min<int64_t>(tiles, ((int64_t)dev.sms * per_sm) / chunks));
    kern<<<(unsigned)(slices * chunks), RT, smem, st>>>(B, m, ldb, F, ta, T, G, chunks, hist);
    count_launches(1);
    return cudaGetLastError();
}

template <int D, int RT>
static cudaError_t bg_hist_t(const float *B, int64_t m, int64_t ldb, int F, const TreeArrays &ta, int T,
                             uint32_t *hist, const DevInfo &dev, cudaStream_t st) {
    // One block per SM (measured faster than two, and than match-aggregated increments).
    // Shared 16-bit counters while the trees fit in at most 8 chunks; beyond that (deep
    // trees: 64 KB of counters per depth-8 tree) every row tile would be staged once per
    // chunk, so the counts go straight to global memory and only the node lists are
    // chunked.
    const size_t budget = dev.smem_optin;
    int G = std::min(T, 256);
    while (G > 1 && BgLayout<D>(F, RT, G, true).total > budget) --G;
    bool smem_hist = BgLayout<D>(F, RT, G, true).total <= budget && (T + G - 1) / G <= 8;
    if (!smem_hist) {
        G = std::min(T, 256);
        while (G > 1 && BgLayout<D>(F, RT, G, false).total > budget) --G;
    }
    const size_t smem = BgLayout<D>(F, RT, G, smem_hist).total;
    if (smem > dev.smem_optin) return cudaErrorInvalidConfiguration;
    if (smem_hist) return bg_hist_launch<D, RT, true, false>(B, m, ldb, F, ta, T, G, smem, dev, hist, st);
    return bg_hist_launch<D, RT, false, false>(B, m, ldb, F, ta, T, G, smem, dev, hist, st);
}

template <int D>
static cudaError_t bg_hist_d(const float *B, int64_t m, int64_t ldb, int F, const TreeArrays &ta, int T,
                             uint32_t *hist, const DevInfo &dev, cudaStream_t st) {
    // 128 rows per block while a row tile fits comfortably, else smaller tiles
    if ((size_t)(F + 1) * 129 * 4 <= dev.smem_optin / 3) return bg_hist_t<D, 128>(B, m, ldb, F, ta, T, hist, dev, st);
    if ((size_t)(F + 1) * 65 * 4 <= dev.smem_optin / 3) return bg_hist_t<D, 64>(B, m, ldb, F, ta, T, hist, dev, st);
    return bg_hist_t<D, 32>(B, m, ldb, F, ta, T, hist, dev, st);
}

cudaError_t launch_bg_hist(int D, const float *B, int64_t m, int64_t ldb, int F, const TreeArrays &ta, int T,
                           uint32_t *hist, const DevInfo &dev, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    switch (D) {
        case 2: return bg_hist_d<2>(B, m, ldb, F, ta, T, hist, dev, st);
        case 3: return bg_hist_d<3>(B, m, ldb, F, ta, T, hist, dev, st);
        case 4: return bg_hist_d<4>(B, m, ldb, F, ta, T, hist, dev, st);
        case 5: return bg_hist_d<5>(B, m, ldb, F, ta, T, hist, dev, st);
        case 6: return bg_hist_d<6>(B, m, ldb, F, ta, T, hist, dev, st);
        case 7: return bg_hist_d<7>(B, m, ldb, F, ta, T, hist, dev, st);
        case 8: return bg_hist_d<8>(B, m, ldb, F, ta, T, hist, dev, st);
        default: return cudaErrorInvalidValue;
    }
}

// vc[row][p] for live leaf row (tree t, leaf q = 4s + j): the leaf pattern p has the
// subtree-root pattern in its high D-2 bits, then the bit for node r and the bit for
// the child of r on the path; the decision at the other child of r is summed out.
// A (when non-null) receives the counts as FP32, the A operand of the contraction
// (exact below 2^24 background rows).
__global__ void k_leaf_counts(int D, const uint32_t *__restrict__ hist, const int32_t *__restrict__ group_leaf,
                              int n_live, uint32_t *__restrict__ vc, float *__restrict__ A) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)n_live << D;
    if (idx >= total) return;
    const int row = (int)(idx >> D);
    const uint32_t p = (uint32_t)(idx & ((1 << D) - 1));
    const int leaf = __ldg(group_leaf + row);
    const int t = leaf >> D, q = leaf & ((1 << D) - 1);
    const int s = q >> 2, j = q & 3;
    const int NS = 1 << (D - 2), E = 1 << (D + 1);
    const uint32_t pp = p >> 2, fn = (p >> 1) & 1u, fc = p & 1u;
    const uint32_t dn = (j < 2) ? fn : (fn ^ 1u);         // path goes left at r for j < 2
    const uint32_t dch = ((j & 1) == 0) ? fc : (fc ^ 1u);  // and left at the child for even j
    const uint32_t *h = hist + ((size_t)t * NS + s) * E;
    uint32_t e0, e1;
    if (j < 2) {
        e0 = (pp << 3) | (dn << 2) | (dch << 1) | 0u;
        e1 = e0 | 1u;
    } else {
        e0 = (pp << 3) | (dn << 2) | 0u | dch;
        e1 = e0 | 2u;
    }
    const uint32_t v = __ldg(h + e0) + __ldg(h + e1);
    vc[idx] = v;
    if (A) A[idx] = (float)v;
}

cudaError_t launch_leaf_counts(int D, const uint32_t *hist, const int32_t *group_leaf, int n_live, uint32_t *vc,
                               float *A, cudaStream_t st) {
    const int64_t total = (int64_t)n_live << D;
    if (total == 0) return cudaSuccess;
    const int threads = 256;
    k_leaf_counts<<<(unsigned)((total + threads - 1) / threads), threads, 0, st>>>(D, hist, group_leaf, n_live, vc,
                                                                                  A);
    count_launches(1);
    return cudaGetLastError();
}

// Path-dependent frequencies (Eq. "path_dependent_estimation"): for live leaf row `row`
// with cover ratios r_k = cover(path node k+1) / cover(path node k), the frequency of
// baseline pattern p is the product over the path of r_k where bit D-1-k of p is 1 and
// of 1 - r_k where it is 0, in FP64, stored as the FP32 A operand.
__global__ void k_pd_freq(int D, const double *__restrict__ ratio, int n_live, float *__restrict__ A) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ((int64_t)n_live << D)) return;
    const int row = (int)(idx >> D);
    const uint32_t p = (uint32_t)(idx & ((1 << D) - 1));
    double f = 1.0;
    for (int k = 0; k < D; ++k) {
        const double r = __ldg(ratio + (size_t)row * D + k);
        f *= ((p >> (D - 1 - k)) & 1u) ? r : 1.0 - r;
    }
    A[idx] = (float)f;
}

cudaError_t launch_pd_freq(int D, const double *ratio, int n_live, float *A, cudaStream_t st) {
    const int64_t total = (int64_t)n_live << D;
    if (total == 0) return cudaSuccess;
    k_pd_freq<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(D, ratio, n_live, A);
    count_launches(1);
    return cudaGetLastError();
}

// v({}) = sum_l w_l * freq_l(all ones): for the background game freq = vc / m (a row
// reaches leaf l exactly when its pattern there is all ones, so this is E_b f(b)); for
// the path-dependent game (ratio non-null) freq = the product of the leaf's cover ratios.
// One block, fixed reduction order.
__global__ void k_base_value(int D, const uint32_t *__restrict__ vc, const double *__restrict__ ratio,
                             const double *__restrict__ w, int n_live, int64_t m, double *__restrict__ out) {
    __shared__ double red[256];
    const int full = (1 << D) - 1;
    double acc = 0.0;
    for (int r = threadIdx.x; r < n_live; r += blockDim.x) {
        double f;
        if (ratio) {
            f = 1.0;
            for (int k = 0; k < D; ++k) f *= ratio[(size_t)r * D + k];
        } else {
            f = (double)vc[((size_t)r << D) + full] / (double)m;
        }
        acc += w[r] * f;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

cudaError_t launch_base_value(int D, const uint32_t *vc, const double *ratio, const double *leaf_w_rows, int n_live,
                              int64_t m, double *out, cudaStream_t st) {
    k_base_value<<<1, 256, 0, st>>>(D, vc, ratio, leaf_w_rows, n_live, m, out);
    count_launches(1);
    return cudaGetLastError();
}

// scale[row] = w_row / m, the leaf weight and the 1/|B| of Eq. "bg_shap_derivation"
// step (e) folded into one FP32 factor per leaf.
__global__ void k_scale(const double *__restrict__ w, int n_live, int64_t m, float *__restrict__ scale) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_live) scale[i] = (float)(w[i] / (double)m);
}

cudaError_t launch_scale(const double *w, int n_live, int64_t m, float *scale, cudaStream_t st) {
    if (n_live == 0) return cudaSuccess;
    k_scale<<<(n_live + 255) / 256, 256, 0, st>>>(w, n_live, m, scale);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace wdf
