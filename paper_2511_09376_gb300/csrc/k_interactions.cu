// Pairwise interaction values (section "Beyond SHAP": Def. "shap_iv_def" with Table
// "table_shap_iv", Def. "banzhaf_iv_def" with Formula
// "banzhaf_simplified_formula_interactions") of the game the ensemble holds.  By
// linearity (the derivation of Eq. "bg_shap_derivation" uses only linearity) the
// pipeline is the one of the values with a pair table in place of the value table:
//   k_tables_iv   per path signature, for every (p_b, p_c) cube and every pair of path
//                 positions, the pair's cell (FP64 built, stored FP32);
//   contraction   s2_{l,q}[p_c] = w_l sum_{p_b} M2[p_c][p_b][q] f_l[p_b] (the FP32 GEMM of
//                 the values with P = D(D-1)/2 pair slots per pattern);
//   k_iv_fold     (depth <= 6) the four leaves of every bottom subtree folded per entry
//                 into one vector of slot-pair values, as the values' k_fold does;
//   k_iv_pack     (deeper trees) s2 per (leaf row, p_c) as PP contiguous floats;
//   k_explain_iv_fold / k_explain_iv  one block per consumer row: the row's decision
//                 codes, every tree's decision words, then per tree (folded: one gather
//                 per live bottom subtree, the pairs of nodes above the bottom subtrees
//                 summed in registers) or per live leaf the pair values added
//                 (shared-memory atomics) into the upper triangle of the row's F x F
//                 matrix, written out symmetric with a zero diagonal.
// Unlike the values, the additions into one matrix element come from many threads,
// so their order (and the last bits of the FP32 result) can change from run to run.
#include <algorithm>

#include "launch.h"
#include "wdf_device.cuh"

namespace wdf {

__device__ __forceinline__ double iv_binom(int n, int k) {
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
    return r;
}

// One thread per (p_b, p_c) of one signature.  Position pair q runs over (k1, k2), k1 <
// k2, in the order (0,1), (0,2), ..., (D-2, D-1).  A feature met at several positions
// is one variable: only pairs of first occurrences carry a value.
__global__ void k_tables_iv(int D, int metric, const uint32_t *__restrict__ keys, float *__restrict__ t2) {
    const int g = blockIdx.y;
    const int K = 1 << D, P = D * (D - 1) / 2, N2 = P << D;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= K * K) return;
    const int pb = idx >> D, pc = idx & (K - 1);
    const uint32_t key = keys[g];
    uint32_t posm = 0, negm = 0;
    const bool bottom = (pc | pb) != K - 1;  // rule 4
    for (int k = 0; k < D; ++k) {
        const int bc = (pc >> (D - 1 - k)) & 1, bb = (pb >> (D - 1 - k)) & 1;
        const int f = (key >> (3 * k)) & 7;
        if (bc && !bb) posm |= 1u << f;  // rule 1
        if (!bc && bb) negm |= 1u << f;  // rule 2
    }
    const bool unsat = bottom || (posm & negm);
    const int a = __popc(posm), b = __popc(negm), s = a + b;
    double pp = 0.0, nn = 0.0, pn = 0.0, np = 0.0;  // (i in S+, j in S+), (-,-), (+,-), (-,+)
    if (!unsat && s >= 2) {
        if (metric == 1) {
            const double v = 1.0 / (double)(1u << (s - 2));
            pp = nn = v;
            pn = np = -v;
        } else {
            if (a >= 2) pp = 1.0 / ((double)(a - 1) * iv_binom(s - 1, a - 1));
            if (b >= 2) nn = 1.0 / ((double)(b - 1) * iv_binom(s - 1, b - 1));
            if (b >= 1) pn = -1.0 / ((double)b * iv_binom(s - 1, b));
            if (a >= 1) np = -1.0 / ((double)a * iv_binom(s - 1, a));
        }
    }
    float *row = t2 + ((size_t)g * K + pb) * N2;
    int q = 0;
    for (int k1 = 0; k1 < D; ++k1)
        for (int k2 = k1 + 1; k2 < D; ++k2, ++q) {
            double v = 0.0;
            const int f1 = (key >> (3 * k1)) & 7, f2 = (key >> (3 * k2)) & 7;
            if (!unsat && f1 == k1 && f2 == k2) {
                const bool p1 = (posm >> k1) & 1u, n1 = (negm >> k1) & 1u;
                const bool p2 = (posm >> k2) & 1u, n2 = (negm >> k2) & 1u;
                if (p1 && p2) v = pp;
                else if (n1 && n2) v = nn;
                else if (p1 && n2) v = pn;
                else if (n1 && p2) v = np;
            }
            row[((size_t)q << D) + pc] = (float)v;
        }
}

cudaError_t launch_tables_iv(int D, int metric, const uint32_t *sig_keys, int G, float *t2, cudaStream_t st) {
    if (G == 0) return cudaSuccess;
    const int total = 1 << (2 * D);
    dim3 grid((total + 255) / 256, G);
    k_tables_iv<<<grid, 256, 0, st>>>(D, metric, sig_keys, t2);
    count_launches(1);
    return cudaGetLastError();
}

// S2T[row][p_c][0..PP) = S2[row][q * 2^D + p_c] (zeros past P).
__global__ void k_iv_pack(int D, int PP, const float *__restrict__ S2, int n_live, float *__restrict__ S2T) {
    const int K = 1 << D, P = D * (D - 1) / 2;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n_live * K) return;
    const int64_t row = idx >> D;
    const int pc = (int)(idx & (K - 1));
    const float *src = S2 + (size_t)row * ((size_t)P << D);
    float *dst = S2T + (size_t)idx * PP;
    for (int q = 0; q < PP; ++q) dst[q] = q < P ? __ldg(src + ((size_t)q << D) + pc) : 0.0f;
}

cudaError_t launch_iv_pack(int D, int PP, const float *S2, int n_live, float *S2T, cudaStream_t st) {
    const int64_t total = (int64_t)n_live << D;
    if (total == 0) return cudaSuccess;
    k_iv_pack<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(D, PP, S2, n_live, S2T);
    count_launches(1);
    return cudaGetLastError();
}

// ---- folded form for trees of depth <= 6 ----
// The four leaves of a bottom subtree share their path above the subtree root r.  Slots
// of a subtree: 0..D-3 the ancestors of r (root first), D-2 = r, D-1 = its left child,
// D = its right child.  A folded vector holds, per entry, the pair values of every slot
// pair (u, v), u < v, except (left child, right child) (never on one path), summed
// over the four leaves: IV_FP(D) = C(D+1, 2) - 1 values, padded to a multiple of 4.
__host__ __device__ constexpr int iv_fp(int D) { return (D + 1) * D / 2 - 1; }
__host__ __device__ constexpr int iv_fpp(int D) { return (iv_fp(D) + 3) & ~3; }
// index of slot pair (u, v), u < v, in a folded vector (pairs ordered by u, then v)
__host__ __device__ constexpr int iv_pidx(int D, int u, int v) {
    return u * D - u * (u - 1) / 2 + (v - u - 1);
}

// One thread per (tree, bottom subtree, entry): fold the per-leaf pair values S2 [leaf
// row][q * 2^D + p] of the subtree's four leaves (q over the leaf's position pairs).
__global__ void k_iv_fold(int D, const float *__restrict__ S2, const int32_t *__restrict__ leaf_row, int T,
                          float *__restrict__ fold) {
    const int NS = 1 << (D - 2), E = 1 << (D + 1), NL = 1 << D, K = 1 << D, P = D * (D - 1) / 2;
    const int FPP = iv_fpp(D);
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)T * NS * E) return;
    const int e = (int)(idx % E);
    const int s = (int)((idx / E) % NS);
    const int t = (int)(idx / ((int64_t)E * NS));
    const uint32_t pp = ((uint32_t)e >> 3) ^ (uint32_t)s, dn = (e >> 2) & 1, dnl = e & 1, dnr = (e >> 1) & 1;
    float out[20];
#pragma unroll
    for (int k = 0; k < 20; ++k) out[k] = 0.0f;
    for (int j = 0; j < 4; ++j) {
        const int row = __ldg(leaf_row + (size_t)t * NL + 4 * s + j);
        if (row < 0) continue;
        const uint32_t fn = (j < 2) ? dn : (dn ^ 1u);
        const uint32_t dch = (j < 2) ? dnl : dnr;
        const uint32_t fc = ((j & 1) == 0) ? dch : (dch ^ 1u);
        const uint32_t p = (pp << 2) | (fn << 1) | fc;
        const float *Sr = S2 + (size_t)row * ((size_t)P << D);
        int q = 0;
        for (int k1 = 0; k1 < D; ++k1)
            for (int k2 = k1 + 1; k2 < D; ++k2, ++q) {
                // path position D-1 is the child of r on this leaf's path
                const int u = k1, v = (k2 == D - 1 && j >= 2) ? D : k2;
                out[iv_pidx(D, u, v)] += __ldg(Sr + ((size_t)q << D) + p);
            }
    }
    (void)K;
    float *dst = fold + idx * FPP;
    for (int k = 0; k < FPP; ++k) dst[k] = out[k];
}

// Words of the depth <= 6 interaction scratch: the folded vectors, then a byte per
// complete-layout node of every tree (its feature; 16 words per tree), then every tree's
// decision records packed into words (kIvPackWords per tree); the last two are used when
// F <= 255 and the codes take one byte.
constexpr int kIvPackWords = 68;
static size_t iv_fold_only(int D, int T) { return ((size_t)T << (D - 2 + D + 1)) * iv_fpp(D); }
size_t iv_fold_floats(int D, int T) { return D <= 6 ? iv_fold_only(D, T) + (size_t)T * (16 + kIvPackWords) : 0; }

// prec[t]: words 0-2 = the tree's pass-through decision words and its real inner-node
// count, then one word per real node: column << 16 | (rank + 1) << 7 | decision bit (the
// row goes left at the node when its code < rank + 1).  One-byte codes only.
__global__ void k_iv_pack_records(int NW, int NI, const int4 *__restrict__ rec, const TreeMeta *__restrict__ meta,
                                  int T, uint32_t *__restrict__ prec) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)T * kIvPackWords) return;
    const int t = (int)(i / kIvPackWords), k = (int)(i % kIvPackWords);
    const int cnt = meta[t].wend[NW - 1];
    uint32_t w = 0u;
    if (k == 0) {
        w = meta[t].pt[0];
    } else if (k == 1) {
        w = NW == 2 ? meta[t].pt[1] : 0u;
    } else if (k == 2) {
        w = (uint32_t)cnt;
    } else if (k >= 4 && k - 4 < cnt) {
        const int4 r = rec[(size_t)t * NI + (k - 4)];
        const int bit = r.z ? __ffs(r.z) - 1 : 32 + __ffs(r.w) - 1;
        w = ((uint32_t)(r.x >> 5) << 16) | ((uint32_t)(r.y + 1) << 7) | (uint32_t)bit;
    }
    prec[i] = w;
}

// ftab[t][h] = the feature of node h of tree t (h < 2^D - 1; 255 past the last node).
__global__ void k_iv_feature_bytes(int NI, const int2 *__restrict__ nodes, int T, unsigned char *__restrict__ ftab) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)T * 64) return;
    const int t = (int)(i >> 6), h = (int)(i & 63);
    ftab[i] = h < NI ? (unsigned char)__ldg(&nodes[(size_t)t * NI + h].x) : (unsigned char)255;
}

cudaError_t launch_iv_fold(int D, const float *S2, const int32_t *leaf_row, int T, float *fold, cudaStream_t st) {
    if (D > 6) return cudaErrorInvalidValue;
    const int64_t total = (int64_t)T << (D - 2 + D + 1);
    k_iv_fold<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(D, S2, leaf_row, T, fold);
    count_launches(1);
    return cudaGetLastError();
}

constexpr int kIvThreads = 256;

// Index of (lo, hi), lo < hi, in the row-major upper triangle of an F x F matrix (the
// triangle is in shared memory, so it fits 32-bit arithmetic).
__device__ __forceinline__ int iv_tri(int lo, int hi, int F) {
    return lo * F - ((lo * (lo + 1)) >> 1) + (hi - lo - 1);
}

// Writes one row's full symmetric F x F matrix with a zero diagonal: from the upper
// triangle in shared memory (SMEM), or by mirroring the upper half accumulated in place.
// Thread tid takes elements tid, tid + kIvThreads, ...; their (i, j) advance without a
// division (the step is di rows and dj columns, with at most one carry).
template <bool SMEM>
__device__ __forceinline__ void iv_write_row(float *orow, const float *acc, int F, int tid) {
    const int64_t FF = (int64_t)F * F;
    int i = tid / F, j = tid - i * F;
    const int di = kIvThreads / F, dj = kIvThreads - di * F;
    for (int64_t k = tid; k < FF; k += kIvThreads) {
        if (SMEM)
            orow[k] = i == j ? 0.0f : acc[iv_tri(min(i, j), max(i, j), F)];
        else if (i > j)
            orow[k] = orow[(size_t)j * F + i];
        i += di;
        j += dj;
        if (j >= F) {
            j -= F;
            ++i;
        }
    }
}

__host__ __device__ __forceinline__ size_t iv_up16(size_t v) { return (v + 15) & ~(size_t)15; }

// One block per consumer row (grid-stride over rows).  Shared memory: the row's code
// per column (int) | every tree's decision words | (SMEM) the upper triangle of the
// row's matrix.  Without SMEM the triangle accumulates in place in out (global atomics).
template <int D, bool SMEM>
__global__ void __launch_bounds__(kIvThreads) k_explain_iv(const float *__restrict__ C, int64_t n, int64_t ldc,
                                                         int F, TreeArrays ta, int T,
                                                         const int32_t *__restrict__ group_leaf, int n_live,
                                                         const float *__restrict__ S2T, float *__restrict__ out,
                                                         int64_t ldo) {
    using S = Shape<D>;
    constexpr int NW = S::NW, NI = S::NI, NL = S::NL, K = 1 << D;
    constexpr int P = D * (D - 1) / 2, PP = (P + 3) & ~3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ncol = ta.n_cols, cshift = ta.code_bytes == 1 ? 5 : 6;  // column = col_off >> cshift
    int *scode = reinterpret_cast<int *>(smem_raw);
    uint32_t *sdw = reinterpret_cast<uint32_t *>(smem_raw + iv_up16((size_t)ncol * 4));
    float *acc = reinterpret_cast<float *>(smem_raw + iv_up16((size_t)ncol * 4) + iv_up16((size_t)T * NW * 4));
    const int tid = threadIdx.x;
    const int64_t ntri = (int64_t)F * (F - 1) / 2;
    for (int64_t row = blockIdx.x; row < n; row += gridDim.x) {
        float *orow = out + row * ldo;
        // zero the accumulator; the row's decision codes
        if (SMEM) {
            for (int64_t k = tid; k < ntri; k += kIvThreads) acc[k] = 0.0f;
        } else {
            for (int64_t k = tid; k < (int64_t)F * F; k += kIvThreads) orow[k] = 0.0f;
        }
        const float *x = C + row * ldc;
        for (int c = tid; c < ncol; c += kIvThreads) {
            const int4 cv = __ldg(reinterpret_cast<const int4 *>(ta.cols) + c);
            const CodeCol col{cv.x, cv.y, cv.z, cv.w};
            scode[c] = decision_code(__ldg(x + col.feature), ta.col_thr + col.first, col);
        }
        __syncthreads();
        // decision words of every tree (bit v of word v / 32: left at inner node v)
        for (int t = tid; t < T; t += kIvThreads) {
            const TreeMeta m = load_meta(ta.meta + t);
            const int4 *rec = reinterpret_cast<const int4 *>(ta.rec) + (size_t)t * NI;
            if (NW <= 2) {
                uint32_t lo = 0u, hi = 0u;
                for (int i = 0; i < m.wend[NW - 1]; ++i) {
                    const int4 r = __ldg(rec + i);
                    const uint32_t s = 0u - (uint32_t)(scode[r.x >> cshift] <= r.y);
                    lo |= (uint32_t)r.z & s;
                    hi |= (uint32_t)r.w & s;
                }
                sdw[t * NW] = m.pt[0] | lo;
                if (NW == 2) sdw[t * NW + 1] = m.pt[1] | hi;
            } else {
                int i = 0;
                for (int w = 0; w < NW; ++w) {
                    uint32_t bits = 0u;
                    for (; i < m.wend[w]; ++i) {
                        const int4 r = __ldg(rec + i);
                        bits |= (uint32_t)r.z & (0u - (uint32_t)(scode[r.x >> cshift] <= r.y));
                    }
                    sdw[t * NW + w] = m.pt[w] | bits;
                }
            }
        }
        __syncthreads();
        // every live leaf: its consumer pattern, its pair values and their features
        for (int i = tid; i < n_live; i += kIvThreads) {
            const int id = __ldg(group_leaf + i);
            const int t = id >> D, q = id & (NL - 1);
            int pc = 0, fk[D];
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const int h = ((NL + q) >> (D - k)) - 1;  // path node at depth k
                const uint32_t d = (sdw[t * NW + (h >> 5)] >> (h & 31)) & 1u;
                pc |= (int)((d ^ ((uint32_t)(q >> (D - 1 - k)) & 1u)) << (D - 1 - k));
                fk[k] = __ldg(&ta.nodes[(size_t)t * NI + h].x);
            }
            float v[PP];
            const float4 *src = reinterpret_cast<const float4 *>(S2T + ((size_t)i * K + pc) * PP);
#pragma unroll
            for (int u = 0; u < PP / 4; ++u) {
                const float4 w4 = __ldg(src + u);
                v[4 * u] = w4.x; v[4 * u + 1] = w4.y; v[4 * u + 2] = w4.z; v[4 * u + 3] = w4.w;
            }
            int qq = 0;
#pragma unroll
            for (int k1 = 0; k1 < D; ++k1)
#pragma unroll
                for (int k2 = k1 + 1; k2 < D; ++k2, ++qq) {
                    const int a = min(fk[k1], fk[k2]), b = max(fk[k1], fk[k2]);
                    if (v[qq] != 0.0f && b < F && a != b) {
                        if (SMEM)
                            atomicAdd(acc + iv_tri(a, b, F), v[qq]);
                        else
                            atomicAdd(orow + (size_t)a * F + b, v[qq]);
                    }
                }
        }
        __syncthreads();
        iv_write_row<SMEM>(orow, acc, F, tid);
        __syncthreads();
    }
}

// Folded consumer kernel (depth <= 6): as k_explain_iv, but after the decision words a
// thread takes a whole tree: per live bottom subtree one gathered folded vector, whose
// pairs with r or its children go straight into the triangle, while the pairs of two
// nodes above the bottom subtrees accumulate in registers (one per (node, ancestor))
// and are added once per tree.
// FB (F <= 255, one-byte codes): the node features come from a byte table, loaded as
// 64 bytes per tree into registers, instead of one scattered load per feature, and the
// decision records from the packed table (four nodes per 16-byte load).
template <int D, bool SMEM, bool FB>
__global__ void __launch_bounds__(kIvThreads) k_explain_iv_fold(const float *__restrict__ C, int64_t n, int64_t ldc,
                                                              int F, TreeArrays ta, int T,
                                                              const float *__restrict__ fold,
                                                              const uint4 *__restrict__ ftab,
                                                              const uint4 *__restrict__ prec, float *__restrict__ out,
                                                              int64_t ldo) {
    using S = Shape<D>;
    constexpr int NW = S::NW, NI = S::NI, NS = S::NS, E = S::E;
    constexpr int FPP = iv_fpp(D);
    // (node, ancestor) pairs above the bottom subtrees: node v of depth d has d of them
    constexpr int UP = (D - 4) * (1 << (D - 2)) + 2 > 1 ? (D - 4) * (1 << (D - 2)) + 2 : 1;  // sum of depths, nodes 0..NS-2
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ncol = ta.n_cols, cshift = ta.code_bytes == 1 ? 5 : 6;
    int *scode = reinterpret_cast<int *>(smem_raw);
    uint32_t *sdw = reinterpret_cast<uint32_t *>(smem_raw + iv_up16((size_t)ncol * 4));
    float *acc = reinterpret_cast<float *>(smem_raw + iv_up16((size_t)ncol * 4) + iv_up16((size_t)T * NW * 4));
    const int tid = threadIdx.x;
    const int64_t ntri = (int64_t)F * (F - 1) / 2;
    for (int64_t row = blockIdx.x; row < n; row += gridDim.x) {
        float *orow = out + row * ldo;
        if (SMEM) {
            for (int64_t k = tid; k < ntri; k += kIvThreads) acc[k] = 0.0f;
        } else {
            for (int64_t k = tid; k < (int64_t)F * F; k += kIvThreads) orow[k] = 0.0f;
        }
        const float *x = C + row * ldc;
        for (int c = tid; c < ncol; c += kIvThreads) {
            const int4 cv = __ldg(reinterpret_cast<const int4 *>(ta.cols) + c);
            const CodeCol col{cv.x, cv.y, cv.z, cv.w};
            scode[c] = decision_code(__ldg(x + col.feature), ta.col_thr + col.first, col);
        }
        __syncthreads();
        for (int t = tid; t < T; t += kIvThreads) {
            if constexpr (FB) {
                const uint4 *pr = prec + (size_t)t * (kIvPackWords / 4);
                const uint4 hd = __ldg(pr);
                uint64_t d = (uint64_t)hd.x | ((uint64_t)hd.y << 32);
                const int cnt = (int)hd.z;
                for (int i0 = 0; i0 < cnt; i0 += 4) {
                    const uint4 w4 = __ldg(pr + 1 + (i0 >> 2));
                    const uint32_t a[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (i0 + c < cnt)
                            d |= (uint64_t)(scode[a[c] >> 16] < (int)((a[c] >> 7) & 511u)) << (a[c] & 127u);
                }
                sdw[t * NW] = (uint32_t)d;
                if (NW == 2) sdw[t * NW + 1] = (uint32_t)(d >> 32);
            } else {
                const TreeMeta m = load_meta(ta.meta + t);
                const int4 *rec = reinterpret_cast<const int4 *>(ta.rec) + (size_t)t * NI;
                uint32_t lo = 0u, hi = 0u;
                for (int i = 0; i < m.wend[NW - 1]; ++i) {
                    const int4 r = __ldg(rec + i);
                    const uint32_t s = 0u - (uint32_t)(scode[r.x >> cshift] <= r.y);
                    lo |= (uint32_t)r.z & s;
                    hi |= (uint32_t)r.w & s;
                }
                sdw[t * NW] = m.pt[0] | lo;
                if (NW == 2) sdw[t * NW + 1] = m.pt[1] | hi;
            }
        }
        __syncthreads();
        auto add = [&](int fa, int fb, float v) {
            const int a = min(fa, fb), b = max(fa, fb);
            if (v != 0.0f && b < F && a != b) {
                if (SMEM)
                    atomicAdd(acc + iv_tri(a, b, F), v);
                else
                    atomicAdd(orow + (size_t)a * F + b, v);
            }
        };
        for (int t = tid; t < T; t += kIvThreads) {
            uint32_t dw[NW];
#pragma unroll
            for (int w = 0; w < NW; ++w) dw[w] = sdw[t * NW + w];
            uint32_t ent[NS];
            subtree_entries<D>(dw, ent);
            const uint64_t lv = __ldg(&ta.meta[t].live);
            const int2 *nd = ta.nodes + (size_t)t * NI;
            uint32_t fr[FB ? 16 : 1];
            if constexpr (FB) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint4 w = __ldg(ftab + (size_t)t * 4 + q);
                    fr[4 * q] = w.x; fr[4 * q + 1] = w.y; fr[4 * q + 2] = w.z; fr[4 * q + 3] = w.w;
                }
            }
            // feature of node h (h a compile-time constant in every use)
            auto feat = [&](int h) -> int {
                if constexpr (FB)
                    return (int)((fr[h >> 2] >> ((h & 3) * 8)) & 0xFFu);
                else
                    return __ldg(&nd[h].x);
            };
            float up[UP];
#pragma unroll
            for (int k = 0; k < UP; ++k) up[k] = 0.0f;
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                if (!((lv >> s) & 1ull)) continue;
                const int r = NS - 1 + s;
                const float4 *src = reinterpret_cast<const float4 *>(fold + (((size_t)t * NS + s) * E + ent[s]) * FPP);
                float v[FPP];
#pragma unroll
                for (int u = 0; u < FPP / 4; ++u) {
                    const float4 w4 = __ldg(src + u);
                    v[4 * u] = w4.x; v[4 * u + 1] = w4.y; v[4 * u + 2] = w4.z; v[4 * u + 3] = w4.w;
                }
                int fs[D + 1];  // features of the slots
#pragma unroll
                for (int k = 0; k < D - 2; ++k) fs[k] = feat(((r + 1) >> (D - 2 - k)) - 1);
                fs[D - 2] = feat(r);
                fs[D - 1] = feat(2 * r + 1);
                fs[D] = feat(2 * r + 2);
                // pairs of two ancestors: into the (node, ancestor) registers
#pragma unroll
                for (int kv = 1; kv < D - 2; ++kv) {
                    const int hv = ((r + 1) >> (D - 2 - kv)) - 1;  // ancestor at depth kv
                    // registers of node hv start at the sum of depths of nodes 0..hv-1
                    int base = 0;
#pragma unroll
                    for (int h = 0; h < NS - 1; ++h) base += h < hv ? 31 - __clz(h + 1) : 0;
#pragma unroll
                    for (int ku = 0; ku < kv; ++ku) up[base + ku] += v[iv_pidx(D, ku, kv)];
                }
                // pairs with r or one of its children: straight into the matrix
#pragma unroll
                for (int u = 0; u <= D - 2; ++u)
#pragma unroll
                    for (int w = (u < D - 2 ? D - 2 : D - 1); w <= D; ++w)
                        if (u < w) add(fs[u], fs[w], v[iv_pidx(D, u, w)]);
            }
            // the (node, ancestor) pairs above the bottom subtrees, once per tree
            int k = 0;
#pragma unroll
            for (int h = 1; h < NS - 1; ++h) {
                const int dh = 31 - __clz(h + 1);  // depth of node h
                const int fh = feat(h);
#pragma unroll
                for (int ku = 0; ku < dh; ++ku, ++k) {
                    const int anc = ((h + 1) >> (dh - ku)) - 1;
                    add(feat(anc), fh, up[k]);
                }
            }
        }
        __syncthreads();
        iv_write_row<SMEM>(orow, acc, F, tid);
        __syncthreads();
    }
}

size_t iv_smem_bytes(int D, int F, int T, int n_cols, bool smem_acc) {
    const int NW = ((1 << D) - 1 + 31) / 32;
    return iv_up16((size_t)n_cols * 4) + iv_up16((size_t)T * NW * 4) +
           (smem_acc ? iv_up16((size_t)F * (F - 1) / 2 * 4) : 0);
}

template <int D, bool SMEM>
static cudaError_t iv_t(const float *C, int64_t n, int64_t ldc, int F, const TreeArrays &ta, int T,
                        const int32_t *group_leaf, int n_live, const float *S2T, float *fold, float *out,
                        int64_t ldo, const DevInfo &dev, cudaStream_t st) {
    const size_t smem = iv_smem_bytes(D, F, T, ta.n_cols, SMEM);
    if (smem > dev.smem_optin) return cudaErrorInvalidConfiguration;
    int per_sm = 0;
    cudaError_t err;
    const int64_t cap = n;
    bool done = false;
    if constexpr (D <= 6) {
        if (fold != nullptr) {
            // node features as bytes and packed decision records when they fit (the tables
            // follow the folded vectors)
            const bool fb = F <= 255 && ta.code_bytes == 1;
            uint4 *ftab = reinterpret_cast<uint4 *>(fold + iv_fold_only(D, T));
            uint4 *prec = ftab + (size_t)T * 4;
            if (fb) {
                k_iv_feature_bytes<<<(unsigned)(((int64_t)T * 64 + 255) / 256), 256, 0, st>>>(
                    Shape<D>::NI, ta.nodes, T, reinterpret_cast<unsigned char *>(ftab));
                k_iv_pack_records<<<(unsigned)(((int64_t)T * kIvPackWords + 255) / 256), 256, 0, st>>>(
                    Shape<D>::NW, Shape<D>::NI, reinterpret_cast<const int4 *>(ta.rec), ta.meta, T,
                    reinterpret_cast<uint32_t *>(prec));
                count_launches(2);
            }
            auto kern = fb ? k_explain_iv_fold<D, SMEM, true> : k_explain_iv_fold<D, SMEM, false>;
            err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (err == cudaSuccess)
                err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kIvThreads, smem);
            if (err != cudaSuccess) return err;
            const int64_t grid = std::min<int64_t>(cap, (int64_t)dev.sms * std::max(per_sm, 1));
            kern<<<(unsigned)grid, kIvThreads, smem, st>>>(C, n, ldc, F, ta, T, fold, ftab, prec, out, ldo);
            done = true;
        }
    }
    if (!done) {
        auto kern = k_explain_iv<D, SMEM>;
        err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err == cudaSuccess) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kIvThreads, smem);
        if (err != cudaSuccess) return err;
        const int64_t grid = std::min<int64_t>(cap, (int64_t)dev.sms * std::max(per_sm, 1));
        kern<<<(unsigned)grid, kIvThreads, smem, st>>>(C, n, ldc, F, ta, T, group_leaf, n_live, S2T, out, ldo);
    }
    count_launches(1);
    return cudaGetLastError();
}

template <int D>
static cudaError_t iv_d(const float *C, int64_t n, int64_t ldc, int F, const TreeArrays &ta, int T,
                        const int32_t *group_leaf, int n_live, const float *S2T, float *fold, float *out,
                        int64_t ldo, const DevInfo &dev, cudaStream_t st) {
    // the triangle in shared memory while two blocks still fit per SM, else in place
    if (iv_smem_bytes(D, F, T, ta.n_cols, true) <= dev.smem_optin / 2)
        return iv_t<D, true>(C, n, ldc, F, ta, T, group_leaf, n_live, S2T, fold, out, ldo, dev, st);
    return iv_t<D, false>(C, n, ldc, F, ta, T, group_leaf, n_live, S2T, fold, out, ldo, dev, st);
}

cudaError_t launch_explain_iv(int D, const float *C, int64_t n, int64_t ldc, int F, const TreeArrays &ta, int T,
                              const int32_t *group_leaf, int n_live, const float *S2T, float *fold, float *out,
                              int64_t ldo, const DevInfo &dev, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    switch (D) {
        case 2: return iv_d<2>(C, n, ldc, F, ta, T, group_leaf, n_live, S2T, fold, out, ldo, dev, st);
        case 3: return iv_d<3>(C, n, ldc, F, ta, T, group_leaf, n_live, S2T, fold, out, ldo, dev, st);
        case 4: return iv_d<4>(C, n, ldc, F, ta, T, group_leaf, n_live, S2T, fold, out, ldo, dev, st);
        case 5: return iv_d<5>(C, n, ldc, F, ta, T, group_leaf, n_live, S2T, fold, out, ldo, dev, st);
        case 6: return iv_d<6>(C, n, ldc, F, ta, T, group_leaf, n_live, S2T, fold, out, ldo, dev, st);
        case 7: return iv_d<7>(C, n, ldc, F, ta, T, group_leaf, n_live, S2T, fold, out, ldo, dev, st);
        case 8: return iv_d<8>(C, n, ldc, F, ta, T, group_leaf, n_live, S2T, fold, out, ldo, dev, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace wdf
