// Device helpers shared by the background-count kernel and the consumer kernel.
//
// A thread owns one row.  For one tree it evaluates the inner nodes of the complete
// layout (Def. "decision_tree": x[feature] < threshold), keeps the decisions as a
// bitmask, and derives the decision patterns of the bottom-subtree roots by the rule
// of Algorithm 1 (a child's pattern is its parent's shifted left plus 1 when the row
// takes that child).  Pass-through nodes always send a row left, so their decision
// bits come from a per-tree mask and only the nodes testing a real feature are
// evaluated, from a compacted per-tree list.  The pattern indices are compile-time
// constants of the depth D, so the per-node state stays in registers.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace wdf {

template <int D>
struct Shape {
    static constexpr int NI = (1 << D) - 1;    // inner nodes
    static constexpr int NL = 1 << D;          // leaves
    static constexpr int NS = 1 << (D - 2);    // bottom subtrees
    static constexpr int E = 1 << (D + 1);     // entries per bottom subtree
    static constexpr int NW = (NI + 63) / 64;  // 64-bit decision words
    static constexpr int SP = (D + 1) <= 4 ? 4 : ((D + 1) <= 8 ? 8 : 12);  // padded slots per entry
};

// One tree of a chunk staged in shared memory.
//   rn[i]  (i < cnt): x = (feature * XS) << 8 | heap index, y = threshold bits
//   fo[v]  feature * XS of heap node v (pass-through nodes: F * XS, a scratch row)
struct TreeMeta {
    uint64_t pt[4];  // pass-through bits
    uint64_t live;   // live bottom subtrees
    int cnt;         // real inner nodes
    uint32_t flush;  // bit b: consumer flush batch b repeats no real feature
};

// Stage trees [t0, t0 + tcn) into shared memory (all threads of the block call it).
template <int D>
__device__ __forceinline__ void stage_trees(int t0, int tcn, int XS, const int2 *__restrict__ nodes,
                                            const int32_t *__restrict__ rn_key, const float *__restrict__ rn_thr,
                                            const int32_t *__restrict__ rn_count, const uint64_t *__restrict__ pt_mask,
                                            const uint64_t *__restrict__ live, const uint32_t *__restrict__ flush_ok,
                                            int2 *srn, int *sfo, TreeMeta *smeta, int tid, int nthreads) {
    constexpr int NI = Shape<D>::NI;
    for (int i = tid; i < tcn * NI; i += nthreads) {
        const size_t gi = (size_t)t0 * NI + i;
        const int key = __ldg(rn_key + gi);
        srn[i] = make_int2((((key >> 8) * XS) << 8) | (key & 255), __float_as_int(__ldg(rn_thr + gi)));
        if (sfo != nullptr) sfo[i] = __ldg(&nodes[gi].x) * XS;
    }
    for (int i = tid; i < tcn; i += nthreads) {
        TreeMeta m;
#pragma unroll
        for (int w = 0; w < 4; ++w) m.pt[w] = __ldg(pt_mask + (size_t)(t0 + i) * 4 + w);
        m.live = __ldg(live + t0 + i);
        m.cnt = __ldg(rn_count + t0 + i);
        m.flush = flush_ok != nullptr ? __ldg(flush_ok + t0 + i) : 0u;
        smeta[i] = m;
    }
}

// Decision bitmask of row `lane` (staged at sx[f * XS + lane]) for one tree.
template <int D>
__device__ __forceinline__ void tree_decisions(const int2 *rn, const TreeMeta &m, const float *sx, int lane,
                                               uint64_t (&dm)[Shape<D>::NW]) {
    constexpr int NW = Shape<D>::NW;
    // four independent partial masks, so consecutive nodes do not wait on each other
    uint64_t part[4][NW];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int w = 0; w < NW; ++w) part[k][w] = 0ull;
    const int cnt = m.cnt;
    int i = 0;
    for (; i + 4 <= cnt; i += 4) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int2 nd = rn[i + k];
            const float x = sx[(nd.x >> 8) + lane];
            const uint64_t b = (x < __int_as_float(nd.y)) ? 1ull : 0ull;
            const int h = nd.x & 255;
            if (NW == 1) {
                part[k][0] |= b << h;
            } else {
#pragma unroll
                for (int w = 0; w < NW; ++w) part[k][w] |= ((h >> 6) == w) ? (b << (h & 63)) : 0ull;
            }
        }
    }
    for (; i < cnt; ++i) {
        const int2 nd = rn[i];
        const float x = sx[(nd.x >> 8) + lane];
        const uint64_t b = (x < __int_as_float(nd.y)) ? 1ull : 0ull;
        const int h = nd.x & 255;
#pragma unroll
        for (int w = 0; w < NW; ++w) part[0][w] |= ((h >> 6) == w) ? (b << (h & 63)) : 0ull;
    }
#pragma unroll
    for (int w = 0; w < NW; ++w) dm[w] = m.pt[w] | part[0][w] | part[1][w] | part[2][w] | part[3][w];
}

template <int D>
__device__ __forceinline__ uint32_t dbit(const uint64_t (&dm)[Shape<D>::NW], int v) {
    return (uint32_t)(dm[v >> 6] >> (v & 63)) & 1u;
}

// Entry index of the row at every bottom subtree (see wdf_internal.h).
template <int D>
__device__ __forceinline__ void subtree_entries(const uint64_t (&dm)[Shape<D>::NW], uint32_t (&ent)[Shape<D>::NS]) {
    constexpr int NS = Shape<D>::NS;
    uint32_t pat[2 * NS - 1];
    pat[0] = 0u;
#pragma unroll
    for (int v = 0; v < NS - 1; ++v) {
        const uint32_t d = dbit<D>(dm, v);
        pat[2 * v + 1] = (pat[v] << 1) | d;
        pat[2 * v + 2] = (pat[v] << 1) | (d ^ 1u);
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const int r = NS - 1 + s;
        ent[s] = (pat[r] << 3) | (dbit<D>(dm, r) << 2) | (dbit<D>(dm, 2 * r + 1) << 1) | dbit<D>(dm, 2 * r + 2);
    }
}

}  // namespace wdf
