// Steps 2 and 3 of Algorithm 3: the pattern-pair tables (built once per path
// signature, section "Algorithmic Improvements" item 2) and their contraction with the
// baseline pattern frequencies, s_{l,i} = w_l * M_{l,i} * f_l (Eq.
// "bg_shap_derivation" step (f); f from background counts or, for the path-dependent
// game, Eq. "path_dependent_estimation"), then the fold of the four leaves of every
// bottom subtree into the per-entry vectors the consumer kernel gathers.
#include "launch.h"

namespace wdf {

__device__ __forceinline__ double binom_small(int n, int k) {
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
    return r;
}

// One thread per (p_b, p_c) of one signature.  The cube of the pair follows the four
// rules of section "Constructing a WDNF Representation" (root first, bit D-1-k is
// path position k); its unit-weight value is Formula "shap_simplified_formula" (metric
// 0, Shapley, in FP64 from exact binomials) or Formula "banzhaf_simplified_formula"
// (metric 1, Banzhaf: +-1 / 2^(|S|-1)).  A feature met at several path positions is one
// variable (cubes are sets); its value sits at its first position.
__global__ void k_tables(int D, int metric, const uint32_t *__restrict__ keys, float *__restrict__ t32,
                         double *__restrict__ t64) {
    const int g = blockIdx.y;
    const int K = 1 << D, N = D << D;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= K * K) return;
    const int pb = idx >> D, pc = idx & (K - 1);
    const uint32_t key = keys[g];
    const size_t rowbase = ((size_t)g * K + pb) * N;
    uint32_t posm = 0, negm = 0;
    bool bottom = (pc | pb) != K - 1;  // some position is (0,0): rule 4
    for (int k = 0; k < D; ++k) {
        const int bc = (pc >> (D - 1 - k)) & 1, bb = (pb >> (D - 1 - k)) & 1;
        const int f = (key >> (3 * k)) & 7;
        if (bc && !bb) posm |= 1u << f;  // rule 1
        if (!bc && bb) negm |= 1u << f;  // rule 2
    }
    const bool unsat = bottom || (posm & negm);
    const int a = __popc(posm), b = __popc(negm);
    double vp, vn;
    if (metric == 1) {
        const double w = (a + b > 0) ? 1.0 / (double)(1u << (a + b - 1)) : 0.0;
        vp = w;
        vn = -w;
    } else {
        vp = (a > 0) ? 1.0 / ((double)a * binom_small(a + b, a)) : 0.0;
        vn = (b > 0) ? -1.0 / ((double)b * binom_small(a + b, b)) : 0.0;
    }
    for (int k = 0; k < D; ++k) {
        double v = 0.0;
        const int f = (key >> (3 * k)) & 7;
        if (!unsat && f == k) {
            if ((posm >> k) & 1u) v = vp;
            else if ((negm >> k) & 1u) v = vn;
        }
        t32[rowbase + ((size_t)k << D) + pc] = (float)v;
        if (t64) t64[rowbase + ((size_t)k << D) + pc] = v;
    }
}

cudaError_t launch_tables(int D, int metric, const uint32_t *sig_keys, int G, float *t32, double *t64,
                          cudaStream_t st) {
    if (G == 0) return cudaSuccess;
    const int total = 1 << (2 * D);
    dim3 grid((total + 255) / 256, G);
    k_tables<<<grid, 256, 0, st>>>(D, metric, sig_keys, t32, t64);
    count_launches(1);
    return cudaGetLastError();
}

// FP32 contraction on CUDA cores: 64 x 64 output tile per block, 4 x 4 per thread.
__global__ void __launch_bounds__(256) k_contract_fp32(int D, int N, const float *__restrict__ A,
                                                       const float *__restrict__ scale, const int4 *__restrict__ tiles,
                                                       const float *__restrict__ t32, float *__restrict__ S) {
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ float As[BK][BM + 4];
    __shared__ float Bs[BK][BN];
    const int4 tile = tiles[blockIdx.x];
    const int g = tile.x, r0 = tile.y, r1 = tile.z;
    const int K = 1 << D;
    const int c0 = blockIdx.y * BN;
    if (c0 >= N) return;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
    const float *Bg = t32 + (size_t)g * K * N;
    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int i = threadIdx.x; i < BM * BK; i += 256) {
            const int r = i / BK, kk = i % BK;
            const int row = r0 + r, k = k0 + kk;
            As[kk][r] = (row < r1 && k < K) ? __ldg(A + ((size_t)row << D) + k) : 0.0f;
        }
        for (int i = threadIdx.x; i < BK * BN; i += 256) {
            const int kk = i / BN, c = i % BN;
            const int k = k0 + kk, col = c0 + c;
            Bs[kk][c] = (k < K && col < N) ? __ldg(Bg + (size_t)k * N + col) : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int row = r0 + ty * 4 + i;
        if (row >= r1) continue;
        const float sc = __ldg(scale + row);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int col = c0 + tx * 4 + j;
            if (col < N) S[(size_t)row * N + col] = acc[i][j] * sc;
        }
    }
}

cudaError_t launch_contract_fp32(int D, const float *A, const float *scale, const int4 *tiles, int n_tiles,
                                 const float *t32, float *S, cudaStream_t st, int slots) {
    if (n_tiles == 0) return cudaSuccess;
    const int N = (slots > 0 ? slots : D) << D;
    dim3 grid(n_tiles, (N + 63) / 64);
    k_contract_fp32<<<grid, 256, 0, st>>>(D, N, A, scale, tiles, t32, S);
    count_launches(1);
    return cudaGetLastError();
}

// One thread per (tree, bottom subtree, entry e).  For each of the four leaves below
// the subtree root r the entry fixes the leaf's consumer pattern p; the slot vector
// collects sum over leaves of S[leaf][k][p] per path position k: positions above r
// (slots 0..D-3) and r itself (slot D-2) from all four leaves, the left child of r
// (slot D-1) from leaves 0-1 and the right child (slot D) from leaves 2-3.  The vector
// of entry e is stored at line_pos(e) of the subtree's line map.
__global__ void k_fold(int D, const float *__restrict__ S, const int32_t *__restrict__ leaf_row, int T,
                       const uint32_t *__restrict__ lines, float *__restrict__ sfold) {
    const int NS = 1 << (D - 2), E = 1 << (D + 1), NL = 1 << D, N = D << D;
    const int SP = (D + 1) <= 4 ? 4 : ((D + 1) <= 8 ? 8 : 12);
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)T * NS * E) return;
    const int e = (int)(idx % E);
    const int s = (int)((idx / E) % NS);
    const int t = (int)(idx / ((int64_t)E * NS));
    // entry -> pattern at the subtree root and the three decisions (wdf_internal.h)
    const uint32_t pp = ((uint32_t)e >> 3) ^ (uint32_t)s, dn = (e >> 2) & 1, dnl = e & 1, dnr = (e >> 1) & 1;
    float out[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) out[k] = 0.0f;
    for (int j = 0; j < 4; ++j) {
        const int row = __ldg(leaf_row + (size_t)t * NL + 4 * s + j);
        if (row < 0) continue;
        const uint32_t fn = (j < 2) ? dn : (dn ^ 1u);
        const uint32_t dch = (j < 2) ? dnl : dnr;
        const uint32_t fc = ((j & 1) == 0) ? dch : (dch ^ 1u);
        const uint32_t p = (pp << 2) | (fn << 1) | fc;
        const float *Sr = S + (size_t)row * N;
        for (int k = 0; k <= D - 2; ++k) out[k] += __ldg(Sr + ((size_t)k << D) + p);
        out[(j < 2) ? D - 1 : D] += __ldg(Sr + ((size_t)(D - 1) << D) + p);
    }
    const uint32_t rot = (__ldg(lines + (size_t)t * lines_words(D) + (s >> 2)) >> (8 * (s & 3))) & 0xFFu;
    const int64_t at = ((int64_t)t * NS + s) * E + line_pos((uint32_t)e, rot, D);
    float4 *dst = reinterpret_cast<float4 *>(sfold + at * SP);
    for (int k = 0; k < SP; k += 4) dst[k / 4] = make_float4(out[k], out[k + 1], out[k + 2], out[k + 3]);
}

cudaError_t launch_fold(int D, const float *S, const int32_t *leaf_row, int T, const uint32_t *lines, float *sfold,
                        cudaStream_t st) {
    const int64_t total = (int64_t)T << (D - 2 + D + 1);
    k_fold<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(D, S, leaf_row, T, lines, sfold);
    count_launches(1);
    return cudaGetLastError();
}

// One thread per (tree, map byte): for its bottom subtree s, the background frequency of
// every entry bit b (the share of rows with bit b set), and the rotation r whose low
// pair (bits r and r + 1 mod D + 1) is the least certain: the largest sum of
// min(p, 1 - p).  Ties keep the smaller r; a subtree no row reaches, and the padding
// bytes past the last subtree, keep the identity 0.
__global__ void k_line_maps(int D, const uint32_t *__restrict__ hist, int T, uint8_t *__restrict__ lines) {
    const int NS = 1 << (D - 2), E = 1 << (D + 1), B = 4 * lines_words(D), NB = D + 1;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)T * B) return;
    const int t = (int)(idx / B), s = (int)(idx % B);
    uint32_t rot = 0;
    if (s < NS && hist) {
        const uint32_t *h = hist + ((size_t)t * NS + s) * E;
        uint64_t total = 0, ones[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int e = 0; e < E; ++e) {
            const uint64_t c = __ldg(h + e);
            total += c;
            for (int b = 0; b < NB; ++b) ones[b] += ((e >> b) & 1) ? c : 0;
        }
        if (total > 0) {
            double best = -1.0;
            for (int r = 0; r < NB; ++r) {
                double u = 0.0;
                for (int k = 0; k < 2; ++k) {
                    const double p = (double)ones[(r + k) % NB] / (double)total;
                    u += p < 1.0 - p ? p : 1.0 - p;
                }
                if (u > best) {
                    best = u;
                    rot = (uint32_t)r;
                }
            }
        }
    }
    lines[idx] = (uint8_t)rot;
}

cudaError_t launch_line_maps(int D, const uint32_t *hist, int T, uint32_t *lines, cudaStream_t st) {
    const int64_t total = (int64_t)T * 4 * lines_words(D);
    if (total == 0) return cudaSuccess;
    k_line_maps<<<(unsigned)((total + 127) / 128), 128, 0, st>>>(D, hist, T, reinterpret_cast<uint8_t *>(lines));
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace wdf
