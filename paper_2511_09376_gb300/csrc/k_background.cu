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
#include <algorithm>

#include "launch.h"
#include "wdf_device.cuh"

namespace wdf {

template <int D, int RT>
__global__ void __launch_bounds__(RT) k_bg_hist(const float *__restrict__ B, int64_t m, int64_t ldb, int F,
                                                const int2 *__restrict__ nodes, const uint64_t *__restrict__ live,
                                                int T, int G, int use_smem, uint32_t *__restrict__ hist) {
    using S = Shape<D>;
    constexpr int XS = RT + 1;
    extern __shared__ __align__(16) uint32_t smem[];
    float *sx = reinterpret_cast<float *>(smem);
    uint32_t *sh = smem + (size_t)(F + 1) * XS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int t0 = blockIdx.y * G;
    const int g_cnt = min(G, T - t0);
    const int chunk_bins = g_cnt * S::NS * S::E;
    uint32_t *hdst = use_smem ? sh : hist + (size_t)t0 * S::NS * S::E;
    if (use_smem)
        for (int i = tid; i < chunk_bins; i += RT) sh[i] = 0u;
    for (int64_t row0 = (int64_t)blockIdx.x * RT; row0 < m; row0 += (int64_t)gridDim.x * RT) {
        __syncthreads();
        for (int r = warp; r < RT; r += RT / 32) {
            const int64_t row = row0 + r;
            const float *src = B + row * ldb;
            for (int f = lane; f < F; f += 32) sx[f * XS + r] = (row < m) ? __ldg(src + f) : 0.0f;
        }
        if (tid < RT) sx[F * XS + tid] = 0.0f;
        __syncthreads();
        const bool valid = row0 + tid < m;
        for (int g = 0; g < g_cnt; ++g) {
            const int t = t0 + g;
            uint32_t dm[S::NW];
            tree_decisions<D>(nodes + (size_t)t * S::NI, sx, XS, tid, dm);
            uint32_t ent[S::NS];
            subtree_entries<D>(dm, ent);
            const uint64_t lv = __ldg(live + t);
#pragma unroll
            for (int s = 0; s < S::NS; ++s) {
                if ((lv >> s) & 1ull) {
                    if (valid) atomicAdd(hdst + ((size_t)g * S::NS + s) * S::E + ent[s], 1u);
                }
            }
        }
    }
    if (use_smem) {
        __syncthreads();
        uint32_t *dst = hist + (size_t)t0 * S::NS * S::E;
        for (int i = tid; i < chunk_bins; i += RT) {
            const uint32_t v = sh[i];
            if (v) atomicAdd(dst + i, v);
        }
    }
}

template <int D, int RT>
static cudaError_t bg_hist_t(const float *B, int64_t m, int64_t ldb, int F, const int2 *nodes, const uint64_t *live,
                             int T, uint32_t *hist, const DevInfo &dev, cudaStream_t st) {
    using S = Shape<D>;
    const size_t xbytes = (size_t)(F + 1) * (RT + 1) * sizeof(float);
    const size_t tbytes = (size_t)S::NS * S::E * sizeof(uint32_t);
    const size_t budget = dev.smem_optin;
    int G = 0;
    if (xbytes < budget) G = (int)std::min<size_t>((size_t)T, (budget - xbytes) / tbytes);
    const int use_smem = G >= 1;
    if (!use_smem) G = T;  // counts go straight to global memory
    const size_t smem = xbytes + (use_smem ? (size_t)G * tbytes : 0);
    if (smem > budget) return cudaErrorInvalidConfiguration;
    auto kern = k_bg_hist<D, RT>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    const int chunks = (T + G - 1) / G;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, RT, smem);
    if (err != cudaSuccess) return err;
    per_sm = std::max(per_sm, 1);
    const int64_t tiles = (m + RT - 1) / RT;
    const int64_t want = std::max<int64_t>(1, ((int64_t)dev.sms * per_sm * 2 + chunks - 1) / chunks);
    dim3 grid((unsigned)std::min<int64_t>(tiles, want), (unsigned)chunks);
    kern<<<grid, RT, smem, st>>>(B, m, ldb, F, nodes, live, T, G, use_smem, hist);
    count_launches(1);
    return cudaGetLastError();
}

template <int D>
static cudaError_t bg_hist_d(const float *B, int64_t m, int64_t ldb, int F, const int2 *nodes, const uint64_t *live,
                             int T, uint32_t *hist, const DevInfo &dev, cudaStream_t st) {
    // 128 rows per block while a row tile and one tree's counts fit, else smaller tiles
    const size_t tbytes = (size_t)Shape<D>::NS * Shape<D>::E * sizeof(uint32_t);
    if ((size_t)(F + 1) * 129 * 4 + tbytes <= dev.smem_optin)
        return bg_hist_t<D, 128>(B, m, ldb, F, nodes, live, T, hist, dev, st);
    if ((size_t)(F + 1) * 65 * 4 + tbytes <= dev.smem_optin)
        return bg_hist_t<D, 64>(B, m, ldb, F, nodes, live, T, hist, dev, st);
    return bg_hist_t<D, 32>(B, m, ldb, F, nodes, live, T, hist, dev, st);
}

cudaError_t launch_bg_hist(int D, const float *B, int64_t m, int64_t ldb, int F, const int2 *nodes,
                           const uint64_t *live, int T, uint32_t *hist, const DevInfo &dev, cudaStream_t st) {
    switch (D) {
        case 2: return bg_hist_d<2>(B, m, ldb, F, nodes, live, T, hist, dev, st);
        case 3: return bg_hist_d<3>(B, m, ldb, F, nodes, live, T, hist, dev, st);
        case 4: return bg_hist_d<4>(B, m, ldb, F, nodes, live, T, hist, dev, st);
        case 5: return bg_hist_d<5>(B, m, ldb, F, nodes, live, T, hist, dev, st);
        case 6: return bg_hist_d<6>(B, m, ldb, F, nodes, live, T, hist, dev, st);
        case 7: return bg_hist_d<7>(B, m, ldb, F, nodes, live, T, hist, dev, st);
        case 8: return bg_hist_d<8>(B, m, ldb, F, nodes, live, T, hist, dev, st);
        default: return cudaErrorInvalidValue;
    }
}

// vc[row][p] for live leaf row (tree t, leaf q = 4s + j): the leaf pattern p has the
// subtree-root pattern in its high D-2 bits, then the bit for node r and the bit for
// the child of r on the path; the decision at the other child of r is summed out.
__global__ void k_leaf_counts(int D, const uint32_t *__restrict__ hist, const int32_t *__restrict__ group_leaf,
                              int n_live, uint32_t *__restrict__ vc) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int NLb = D;  // log2 leaves per tree
    const int64_t total = (int64_t)n_live << D;
    if (idx >= total) return;
    const int row = (int)(idx >> D);
    const uint32_t p = (uint32_t)(idx & ((1 << D) - 1));
    const int leaf = __ldg(group_leaf + row);
    const int t = leaf >> NLb, q = leaf & ((1 << D) - 1);
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
    vc[idx] = __ldg(h + e0) + __ldg(h + e1);
}

cudaError_t launch_leaf_counts(int D, const uint32_t *hist, const int32_t *group_leaf, int n_live, uint32_t *vc,
                               cudaStream_t st) {
    const int64_t total = (int64_t)n_live << D;
    if (total == 0) return cudaSuccess;
    const int threads = 256;
    k_leaf_counts<<<(unsigned)((total + threads - 1) / threads), threads, 0, st>>>(D, hist, group_leaf, n_live, vc);
    count_launches(1);
    return cudaGetLastError();
}

// E_b f(b): a background row reaches leaf l exactly when its pattern there is all
// ones, so sum_l w_l * vc[l][all ones] / m.  One block, fixed reduction order.
__global__ void k_base_value(int D, const uint32_t *__restrict__ vc, const double *__restrict__ w, int n_live,
                             int64_t m, double *__restrict__ out) {
    __shared__ double red[256];
    const int full = (1 << D) - 1;
    double acc = 0.0;
    for (int r = threadIdx.x; r < n_live; r += blockDim.x) acc += w[r] * (double)vc[((size_t)r << D) + full];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0] / (double)m;
}

cudaError_t launch_base_value(int D, const uint32_t *vc, const double *leaf_w_rows, int n_live, int64_t m,
                              double *out, cudaStream_t st) {
    k_base_value<<<1, 256, 0, st>>>(D, vc, leaf_w_rows, n_live, m, out);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace wdf

namespace wdf {

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
