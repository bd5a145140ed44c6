// Device helpers shared by the background-count kernel and the consumer kernel.
//
// A thread owns one row.  For one tree it evaluates every inner node of the complete
// layout (Def. "decision_tree": x[feature] < threshold), keeps the decisions as a
// bitmask, and derives the decision patterns of the bottom-subtree roots by the rule
// of Algorithm 1 (a child's pattern is its parent's shifted left plus 1 when the row
// takes that child).  All indices are compile-time constants of the depth D, so the
// per-node state stays in registers.
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
    static constexpr int NW = (NI + 31) / 32;  // decision words
    static constexpr int SP = (D + 1) <= 4 ? 4 : ((D + 1) <= 8 ? 8 : 12);  // padded slots per entry
};

// Rows are staged feature-major in shared memory: x of row `lane` at feature f is
// sx[f * XS + lane]; feature F is a virtual column of zeros used by pass-through nodes.
template <int D>
__device__ __forceinline__ void tree_decisions(const int2 *__restrict__ tn, const float *sx, int XS, int lane,
                                               uint32_t (&dm)[Shape<D>::NW]) {
#pragma unroll
    for (int w = 0; w < Shape<D>::NW; ++w) dm[w] = 0u;
#pragma unroll
    for (int v = 0; v < Shape<D>::NI; ++v) {
        const int2 nd = __ldg(tn + v);
        const float x = sx[nd.x * XS + lane];
        dm[v >> 5] |= (uint32_t)(x < __int_as_float(nd.y)) << (v & 31);
    }
}

template <int D>
__device__ __forceinline__ uint32_t dbit(const uint32_t (&dm)[Shape<D>::NW], int v) {
    return (dm[v >> 5] >> (v & 31)) & 1u;
}

// Entry index of the row at every bottom subtree (see wdf_internal.h).
template <int D>
__device__ __forceinline__ void subtree_entries(const uint32_t (&dm)[Shape<D>::NW], uint32_t (&ent)[Shape<D>::NS]) {
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
