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
// Work split: the rows are first encoded to decision codes (tree_layout.h, one pass
// over B); the trees are cut into chunks whose counters fit in shared memory as 16-bit
// halves of 32-bit words; blocks are numbered chunk-fastest, so the blocks that stage
// the same code tile run at the same time and share it through L2.  A block flushes
// its 16-bit counters into the global 32-bit counts before any can overflow.
#include <algorithm>
#include <cstdlib>

#include "launch.h"
#include "wdf_device.cuh"

namespace wdf {

// 16-bit counter slots in shared memory.  The rows of one warp increment the entries of
// one (tree, subtree) together, and background entries are far from uniform (a warp's
// most frequent entry is hit by about a quarter of its lanes), so lanes that land in
// one bank serialise.  Two rules spread them: the two halves of a 32-bit word hold the
// same entry of two sibling subtrees (so one instruction touches one entry per word),
// and the word of entry e within its subtree pair is fold(e), which XORs the higher
// entry bits into the five bank bits.  fold is its own inverse (bits 5 and up pass
// through unchanged).
__host__ __device__ __forceinline__ uint32_t bg_fold(uint32_t e) {
    return e ^ ((e >> 5) & 31u) ^ ((e >> 10) & 31u);
}

template <int D>
__device__ __forceinline__ uint32_t bg_slot(int g, int s, uint32_t e) {
    using S = Shape<D>;
    if constexpr (S::NS == 1)
        return (uint32_t)g * S::E + e;
    else
        return (((uint32_t)g * (S::NS / 2) + (uint32_t)(s >> 1)) * S::E + bg_fold(e)) * 2u + (uint32_t)(s & 1);
}

// Adds the shared counters of a block's trees into the global 32-bit counts ([tree]
// [subtree][entry], gdst at the block's first tree) and zeroes them.
template <int D>
__device__ void bg_flush(uint32_t *sh, uint32_t *gdst, int bins, int tid, int nthreads) {
    using S = Shape<D>;
    for (int i = tid; i < bins / 2; i += nthreads) {
        const uint32_t v = sh[i];
        sh[i] = 0u;
        if (!v) continue;
        size_t i0, i1;
        if constexpr (S::NS == 1) {
            i0 = 2 * (size_t)i;
            i1 = i0 + 1;
        } else {
            const uint32_t pair = (uint32_t)i / S::E, e = bg_fold((uint32_t)i % S::E);
            i0 = (size_t)(2 * pair) * S::E + e;  // subtree 2k of the pair; 2k + 1 is E further
            i1 = i0 + S::E;
        }
        if (v & 0xFFFFu) atomicAdd(gdst + i0, v & 0xFFFFu);
        if (v >> 16) atomicAdd(gdst + i1, v >> 16);
    }
}

// Shared memory layout (bytes, 16-aligned pieces): code tile | tree metadata | node
// records | 16-bit counters.
template <int D>
struct BgLayout {
    size_t x, meta, rec, hist, total;
    static __host__ __device__ size_t up(size_t v) { return (v + 15) & ~(size_t)15; }
    __host__ __device__ BgLayout(int xb, int RT, int G, bool smem_hist) {
        x = up((size_t)RT * xb);
        meta = up((size_t)G * sizeof(TreeMeta));
        rec = up((size_t)G * Shape<D>::NI * sizeof(NodeRec));
        hist = smem_hist ? up((size_t)G * Shape<D>::NS * Shape<D>::E * 2) : 0;
        total = x + meta + rec + hist;
    }
};

// 16-byte code words per thread of the next tile held in registers (512-row tiles of up to
// 128 one-byte codes per row fit entirely): 1.8 % off the large workload's background
// step.  None at depth 5, where the registers made the compiler spill, nor for deep
// trees, whose decision loop needs them.
template <int D>
__host__ __device__ constexpr int bg_prefetch() { return D <= 6 && D != 5 ? 8 : 0; }

// codes: rows [0, m) of one encoded chunk, padded to a multiple of RT rows.
template <int D, int RT, bool SMEM>
__global__ void __launch_bounds__(RT) k_bg_hist(const unsigned char *__restrict__ codes, int64_t m, TreeArrays ta,
                                                int T, int G, int chunks, uint32_t *__restrict__ hist) {
    using S = Shape<D>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int cb = ta.code_bytes, xb = ta.n_cols * cb;
    const BgLayout<D> L(xb, RT, G, SMEM);
    unsigned char *sx = smem_raw;
    TreeMeta *smeta = reinterpret_cast<TreeMeta *>(smem_raw + L.x);
    int4 *srec = reinterpret_cast<int4 *>(smem_raw + L.x + L.meta);
    uint32_t *sh = reinterpret_cast<uint32_t *>(smem_raw + L.x + L.meta + L.rec);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int chunk = blockIdx.x % chunks;
    const int slice = blockIdx.x / chunks, nslices = gridDim.x / chunks;
    const int t0 = chunk * G;
    const int g_cnt = min(G, T - t0);
    const int bins = g_cnt * S::NS * S::E;  // 16-bit counters, two per word
    uint32_t *gdst = hist + (size_t)t0 * S::NS * S::E;
    stage_trees<D>(t0, g_cnt, ta.rec, ta.meta, srec, smeta, tid, RT);
    if (SMEM)
        for (int i = tid; i < bins / 2; i += RT) sh[i] = 0u;
    const CodeReader xr(sx + (size_t)warp * 32 * xb, lane, cb);
    const int tile16 = RT * xb / 16;
    // The first bg_prefetch 16-byte words per thread of the next tile are loaded into
    // registers while the current tile is counted (the rest, for wide rows, at staging).
    constexpr int PF = bg_prefetch<D>();
    uint4 pf[PF > 0 ? PF : 1];
    auto fetch = [&](int64_t r0) {
        const uint4 *src = reinterpret_cast<const uint4 *>(codes + r0 * xb);
#pragma unroll
        for (int k = 0; k < PF; ++k) {
            const int i = tid + k * RT;
            if (i < tile16) pf[k] = __ldg(src + i);
        }
    };
    const int64_t step = (int64_t)nslices * RT;
    if (PF > 0 && (int64_t)slice * RT < m) fetch((int64_t)slice * RT);
    int64_t since_flush = 0;
    for (int64_t row0 = (int64_t)slice * RT; row0 < m; row0 += step) {
        __syncthreads();
        if (SMEM && since_flush + RT > 65535) {  // a 16-bit counter could overflow: flush
            bg_flush<D>(sh, gdst, bins, tid, RT);
            since_flush = 0;
        }
        // the tile's RT rows are RT / 32 consecutive code blocks
#pragma unroll
        for (int k = 0; k < PF; ++k) {
            const int i = tid + k * RT;
            if (i < tile16) reinterpret_cast<uint4 *>(sx)[i] = pf[k];
        }
        const uint4 *src = reinterpret_cast<const uint4 *>(codes + row0 * xb);
        for (int i = tid + PF * RT; i < tile16; i += RT) reinterpret_cast<uint4 *>(sx)[i] = __ldg(src + i);
        __syncthreads();
        if (PF > 0 && row0 + step < m) fetch(row0 + step);
        since_flush += RT;
        const bool valid = row0 + tid < m;
        for (int g = 0; g < g_cnt; ++g) {
            const TreeMeta &mt = smeta[g];
            uint32_t dw[S::NW];
            if (cb == 1)
                tree_decisions<D, true>(srec + (size_t)g * S::NI, mt, xr, dw);
            else
                tree_decisions<D, false>(srec + (size_t)g * S::NI, mt, xr, dw);
            uint32_t ent[S::NS];
            subtree_entries<D>(dw, ent);
            const uint64_t lv = mt.live;
#pragma unroll
            for (int s = 0; s < S::NS; ++s) {
                if (((lv >> s) & 1ull) && valid) {
                    if (SMEM) {
                        const uint32_t sl = bg_slot<D>(g, s, ent[s]);
                        atomicAdd(sh + (sl >> 1), 1u << ((sl & 1u) << 4));
                    } else {
                        atomicAdd(gdst + (uint32_t)(g * S::NS + s) * S::E + ent[s], 1u);
                    }
                }
            }
        }
    }
    if (SMEM) {
        __syncthreads();
        bg_flush<D>(sh, gdst, bins, tid, RT);
    }
}

// Tree chunking of one launch: G trees per block with counters in shared memory whenever
// one tree's counters fit beside the code tile; otherwise the counts go straight to
// global memory and only the node records are chunked.  Deep trees (64 KB of counters
// per depth-8 tree) then take one to a few trees per block and hundreds of chunks, each
// block streaming every code tile through shared memory (from L2, where the blocks
// walking the same tiles meet): 47.5 instead of 62.8 ms per 1M rows for 500 trees of
// depth 7, 203 instead of 254 ms for 1000 of depth 8, against global-memory atomics.
// With counters in shared memory G is chosen by a cost model rather than as
// the most that fits: the blocks of a launch (chunks x row slices) are all resident, a
// block's work is its tiles times (G trees + about one tree's worth for staging the
// tile), and the busiest SM runs ceil(blocks / SMs) of them.  So 200 trees go in 8
// chunks of 25 (152 blocks) rather than 7 of 32 (147 blocks, the last chunk nearly
// empty): 6.1 ms against 6.9 ms per 1M rows.
template <int D, int RT>
static cudaError_t bg_hist_t(const unsigned char *codes, int64_t m, const TreeArrays &ta, int T, uint32_t *hist,
                             const DevInfo &dev, cudaStream_t st) {
    const int xb = ta.n_cols * ta.code_bytes;
    const size_t budget = dev.smem_optin;
    const int64_t tiles = (m + RT - 1) / RT;
    int G = std::min(T, 256);
    while (G > 1 && BgLayout<D>(xb, RT, G, true).total > budget) --G;
    const bool smem_hist = BgLayout<D>(xb, RT, G, true).total <= budget;
    cudaError_t err;
    if (smem_hist) {
        auto kern = k_bg_hist<D, RT, true>;
        err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)BgLayout<D>(xb, RT, G, true).total);
        if (err != cudaSuccess) return err;
        int64_t best = -1;
        int best_g = G;
        for (int g = G; g >= 1; --g) {
            const int chunks = (T + g - 1) / g;
            int per_sm = 0;
            err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, RT, BgLayout<D>(xb, RT, g, true).total);
            if (err != cudaSuccess) return err;
            per_sm = std::max(per_sm, 1);
            if (chunks > dev.sms * per_sm) break;
            const int64_t slices = std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)dev.sms * per_sm / chunks));
            const int64_t blocks = slices * chunks;
            const int64_t cost = (int64_t)(g + 1) * ((tiles + slices - 1) / slices) * ((blocks + dev.sms - 1) / dev.sms);
            if (best < 0 || cost < best) {
                best = cost;
                best_g = g;
            }
        }
        G = best_g;
    } else {
        G = std::min(T, 256);
        while (G > 1 && BgLayout<D>(xb, RT, G, false).total > budget) --G;
    }
    const size_t smem = BgLayout<D>(xb, RT, G, smem_hist).total;
    if (smem > dev.smem_optin) return cudaErrorInvalidConfiguration;
    auto kern = smem_hist ? k_bg_hist<D, RT, true> : k_bg_hist<D, RT, false>;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, RT, smem);
    if (err != cudaSuccess) return err;
    per_sm = std::max(per_sm, 1);
    const int chunks = (T + G - 1) / G;
    const int64_t slices = std::max<int64_t>(1, std::min<int64_t>(tiles, ((int64_t)dev.sms * per_sm) / chunks));
    kern<<<(unsigned)(slices * chunks), RT, smem, st>>>(codes, m, ta, T, G, chunks, hist);
    count_launches(1);
    return cudaGetLastError();
}

// Rows per block: the largest tile whose codes take at most 30 % of shared memory.
static int bg_tile_rows(int xb, const DevInfo &dev) {
    for (int rt = kBgMaxTileRows; rt > 32; rt /= 2)
        if ((size_t)rt * xb <= dev.smem_optin * 3 / 10) return rt;
    return 32;
}

// Deep trees (depth 7, 8): the most rows per block (one warp per 32 rows) that fit beside
// one tree's counters, since a block holds only one or two trees anyway: 32.5 instead of
// 47.5 ms per 1M rows for 500 trees of depth 7 (512 instead of 256-row tiles), 150 instead
// of 203 ms for 1000 of depth 8 (512 instead of 128).
template <int D>
static int bg_tile_rows_d(int xb, const DevInfo &dev) {
    if (D >= 7) {
        for (int rt = kBgMaxTileRows; rt > 32; rt /= 2)
            if (BgLayout<D>(xb, rt, 1, true).total <= dev.smem_optin) return rt;
        return 32;
    }
    return bg_tile_rows(xb, dev);
}

template <int D>
static cudaError_t bg_hist_d(const unsigned char *codes, int64_t m, const TreeArrays &ta, int T, uint32_t *hist,
                             const DevInfo &dev, cudaStream_t st) {
    switch (bg_tile_rows_d<D>(ta.n_cols * ta.code_bytes, dev)) {
        case 512: return bg_hist_t<D, 512>(codes, m, ta, T, hist, dev, st);
        case 256: return bg_hist_t<D, 256>(codes, m, ta, T, hist, dev, st);
        case 128: return bg_hist_t<D, 128>(codes, m, ta, T, hist, dev, st);
        case 64: return bg_hist_t<D, 64>(codes, m, ta, T, hist, dev, st);
        default: return bg_hist_t<D, 32>(codes, m, ta, T, hist, dev, st);
    }
}

template <int D>
static cudaError_t bg_count_chunk(const unsigned char *codes, int64_t rows, const TreeArrays &ta, int T,
                                  uint32_t *hist, const DevInfo &dev, cudaStream_t st) {
    return bg_hist_d<D>(codes, rows, ta, T, hist, dev, st);
}

cudaError_t launch_bg_hist(int D, const float *B, int64_t m, int64_t ldb, const TreeArrays &ta, int T,
                           unsigned char *codes, int64_t code_rows, uint32_t *hist, const DevInfo &dev,
                           cudaStream_t st, const BgOverlap *ov) {
    if (m == 0) return cudaSuccess;
    if (code_rows < kBgMaxTileRows || code_rows % kBgMaxTileRows) return cudaErrorInvalidValue;
    cudaError_t err = cudaSuccess;
    if (ov) {
        // the side stream starts after everything already queued on st (B, the zeroed counts)
        err = cudaEventRecord(ov->cnt[0], st);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(ov->side, ov->cnt[0], 0);
        if (err != cudaSuccess) return err;
    }
    int64_t k = 0;
    for (int64_t r0 = 0; r0 < m; r0 += code_rows, ++k) {
        const int64_t rows = std::min(code_rows, m - r0);
        const int64_t rows_pad = (rows + kBgMaxTileRows - 1) / kBgMaxTileRows * kBgMaxTileRows;
        const int b = ov ? (int)(k & 1) : 0;
        unsigned char *buf = b ? ov->codes1 : codes;
        if (ov) {
            // encode chunk k on the side stream once the count of chunk k - 2 (the last
            // reader of this buffer) is done; the count of chunk k waits for the encode
            if (k >= 2) err = cudaStreamWaitEvent(ov->side, ov->cnt[b], 0);
            if (err == cudaSuccess) err = launch_encode_codes(B + r0 * ldb, rows, ldb, ta, rows_pad, buf, ov->side);
            if (err == cudaSuccess) err = cudaEventRecord(ov->enc[b], ov->side);
            if (err == cudaSuccess) err = cudaStreamWaitEvent(st, ov->enc[b], 0);
        } else {
            err = launch_encode_codes(B + r0 * ldb, rows, ldb, ta, rows_pad, buf, st);
        }
        if (err != cudaSuccess) return err;
        switch (D) {
            case 2: err = bg_count_chunk<2>(buf, rows, ta, T, hist, dev, st); break;
            case 3: err = bg_count_chunk<3>(buf, rows, ta, T, hist, dev, st); break;
            case 4: err = bg_count_chunk<4>(buf, rows, ta, T, hist, dev, st); break;
            case 5: err = bg_count_chunk<5>(buf, rows, ta, T, hist, dev, st); break;
            case 6: err = bg_count_chunk<6>(buf, rows, ta, T, hist, dev, st); break;
            case 7: err = bg_count_chunk<7>(buf, rows, ta, T, hist, dev, st); break;
            case 8: err = bg_count_chunk<8>(buf, rows, ta, T, hist, dev, st); break;
            default: return cudaErrorInvalidValue;
        }
        if (err == cudaSuccess && ov) err = cudaEventRecord(ov->cnt[b], st);
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
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
    const uint32_t R = pp ^ (uint32_t)s;  // ancestors' raw decisions (wdf_internal.h)
    uint32_t e0, e1;
    if (j < 2) {  // the path takes 2r+1 (entry bit 0); sum over the decision at 2r+2
        e0 = (R << 3) | (dn << 2) | dch;
        e1 = e0 | 2u;
    } else {  // the path takes 2r+2 (entry bit 1); sum over the decision at 2r+1
        e0 = (R << 3) | (dn << 2) | (dch << 1);
        e1 = e0 | 1u;
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
