// Device helpers shared by the background-count kernel and the consumer kernel.
//
// A thread owns one row.  For one tree it evaluates the inner nodes of the complete
// layout (Def. "decision_tree": x[feature] < threshold, here on the row's decision
// codes, tree_layout.h), keeps the decisions as a bitmask, and derives the decision
// patterns of the bottom-subtree roots by the rule of Algorithm 1 (a child's pattern is
// its parent's shifted left plus 1 when the row takes that child).  Pass-through nodes
// always send a row left, so their decision bits come from a per-tree mask and only
// the nodes testing a real feature are evaluated, from a compacted per-tree list.  The
// pattern indices are compile-time constants of the depth D, so the per-node state
// stays in registers.
//
// Code tile layout in shared memory (both kernels): blocks of 32 rows; within a block
// column c occupies 32 consecutive codes, one per row ([block][column][row of block]),
// so the 32 lanes of a warp read 32 consecutive codes of one column.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "tree_layout.h"

namespace wdf {

template <int D>
struct Shape {
    static constexpr int NI = (1 << D) - 1;    // inner nodes
    static constexpr int NL = 1 << D;          // leaves
    static constexpr int NS = 1 << (D - 2);    // bottom subtrees
    static constexpr int E = 1 << (D + 1);     // entries per bottom subtree
    static constexpr int NW = (NI + 31) / 32;  // 32-bit decision words
    static constexpr int SP = slots_per_entry(D);  // padded slots per entry
};

// Stage the node records and metadata of trees [t0, t0 + tcn) into shared memory (all
// threads of the block call it).
template <int D>
__device__ __forceinline__ void stage_trees(int t0, int tcn, const NodeRec *__restrict__ rec,
                                            const TreeMeta *__restrict__ meta, int4 *srec, TreeMeta *smeta, int tid,
                                            int nthreads) {
    constexpr int NI = Shape<D>::NI;
    const int4 *src = reinterpret_cast<const int4 *>(rec) + (size_t)t0 * NI;
    for (int i = tid; i < tcn * NI; i += nthreads) srec[i] = __ldg(src + i);
    const uint2 *msrc = reinterpret_cast<const uint2 *>(meta + t0);
    uint2 *mdst = reinterpret_cast<uint2 *>(smeta);
    constexpr int MW = sizeof(TreeMeta) / sizeof(uint2);
    for (int i = tid; i < tcn * MW; i += nthreads) mdst[i] = __ldg(msrc + i);
}

// Where a thread reads its row's codes: its own code in column 0 of its code block
// (one-byte codes: a plain byte load), or the 4-byte word holding it and the byte
// selector (__byte_perm) that extracts the code, zero-extended, for two-byte codes.
struct CodeReader {
    const unsigned char *byte, *word;
    uint32_t sel;
    __device__ __forceinline__ CodeReader(const unsigned char *block, int lane, int code_bytes) {
        const int at = lane * code_bytes;
        byte = block + at;
        word = block + (at & ~3);
        const uint32_t b = (uint32_t)(at & 3);
        sel = code_bytes == 1 ? (0x4440u | b) : (0x4400u | ((b + 1u) << 4) | b);
    }
    template <bool ONE_BYTE>
    __device__ __forceinline__ int code(int col_off) const {
        if constexpr (ONE_BYTE)
            return (int)byte[col_off];
        else
            return (int)__byte_perm(*reinterpret_cast<const uint32_t *>(word + col_off), 0u, sel);
    }
    // rec.z when the node (rec.x = column offset, rec.y = rank) sends the row left, else
    // 0; a select, not a branch (the lanes of a warp decide differently)
    template <bool ONE_BYTE>
    __device__ __forceinline__ uint32_t left_bit(const int4 &rec) const {
        return (uint32_t)rec.z & (0u - (uint32_t)(code<ONE_BYTE>(rec.x) <= rec.y));
    }
    template <bool ONE_BYTE>
    __device__ __forceinline__ uint32_t left_mask(const int4 &rec) const {
        return 0u - (uint32_t)(code<ONE_BYTE>(rec.x) <= rec.y);
    }
};

__device__ __forceinline__ TreeMeta load_meta(const TreeMeta *p) {
    TreeMeta m;
    const uint2 *src = reinterpret_cast<const uint2 *>(p);
    uint2 *dst = reinterpret_cast<uint2 *>(&m);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(TreeMeta) / sizeof(uint2)); ++i) dst[i] = __ldg(src + i);
    return m;
}

// Decision words of one row for one tree of depth <= 6 from the first eight bytes of its
// node records (code-column offset, rank), rec and the tree's expand masks mv in shared
// memory: the decisions are collected in record order, one bit per real node, then moved
// to the nodes' heap positions by the expand of Hacker's Delight section 7-5 (six masked
// shifts); pass-through nodes add their always-left bits pt, which also cover the copies
// the expand leaves outside the real positions (or past the tree's last node).  A
// 16-byte record read by a whole warp from one shared address takes two L1 wavefronts,
// an 8-byte one takes one.
template <int D, bool ONE_BYTE>
__device__ __forceinline__ void tree_decisions8(const int2 *rec, int cnt, const uint32_t *pt, const uint64_t *mv,
                                                const CodeReader &xr, uint32_t (&dw)[Shape<D>::NW]) {
    static_assert(Shape<D>::NW <= 2, "64-bit decision word");
    uint64_t x = 0ull;
    int i = 0;
    for (; i + 4 <= cnt; i += 4) {
        const int2 a = rec[i], b = rec[i + 1], c = rec[i + 2], d = rec[i + 3];
        const uint32_t nib = (uint32_t)(xr.code<ONE_BYTE>(a.x) <= a.y) |
                             ((uint32_t)(xr.code<ONE_BYTE>(b.x) <= b.y) << 1) |
                             ((uint32_t)(xr.code<ONE_BYTE>(c.x) <= c.y) << 2) |
                             ((uint32_t)(xr.code<ONE_BYTE>(d.x) <= d.y) << 3);
        x |= (uint64_t)nib << i;
    }
    for (; i < cnt; ++i) {
        const int2 a = rec[i];
        x |= (uint64_t)(xr.code<ONE_BYTE>(a.x) <= a.y) << i;
    }
#pragma unroll
    for (int k = 5; k >= 0; --k) {
        const uint64_t v = mv[k];
        x = (x & ~v) | ((x << (1 << k)) & v);
    }
    dw[0] = pt[0] | (uint32_t)x;
    if constexpr (Shape<D>::NW == 2) dw[1] = pt[1] | (uint32_t)(x >> 32);
}

// Decision words of one row for one tree: bit v of word v/32 is 1 when the row goes
// left at inner node v.  rec (shared memory) holds the tree's real inner nodes.
template <int D, bool ONE_BYTE>
__device__ __forceinline__ void tree_decisions(const int4 *rec, const TreeMeta &m, const CodeReader &xr,
                                               uint32_t (&dw)[Shape<D>::NW]) {
    constexpr int NW = Shape<D>::NW;
    if constexpr (NW <= 2) {
        // one loop over all nodes, the bit in a low and a high word (measured much faster
        // than a loop per word, which stalled on instruction fetch)
        const int cnt = m.wend[NW - 1];
        uint32_t l0 = 0u, l1 = 0u, l2 = 0u, l3 = 0u, h0 = 0u, h1 = 0u, h2 = 0u, h3 = 0u;
        int i = 0;
        for (; i + 4 <= cnt; i += 4) {
            const int4 a = rec[i], b = rec[i + 1], c = rec[i + 2], d = rec[i + 3];
            const uint32_t sa = xr.left_mask<ONE_BYTE>(a), sb = xr.left_mask<ONE_BYTE>(b);
            const uint32_t sc = xr.left_mask<ONE_BYTE>(c), sd = xr.left_mask<ONE_BYTE>(d);
            l0 |= a.z & sa; h0 |= a.w & sa;
            l1 |= b.z & sb; h1 |= b.w & sb;
            l2 |= c.z & sc; h2 |= c.w & sc;
            l3 |= d.z & sd; h3 |= d.w & sd;
        }
        for (; i < cnt; ++i) {
            const int4 a = rec[i];
            const uint32_t sa = xr.left_mask<ONE_BYTE>(a);
            l0 |= a.z & sa; h0 |= a.w & sa;
        }
        dw[0] = m.pt[0] | l0 | l1 | l2 | l3;
        if constexpr (NW == 2) dw[1] = m.pt[1] | h0 | h1 | h2 | h3;
    } else {
        // deep trees: one (rolled) loop per 32-node word
        int lo = 0;
#pragma unroll 1
        for (int w = 0; w < NW; ++w) {
            const int hi = m.wend[w];
            uint32_t p0 = 0u, p1 = 0u, p2 = 0u, p3 = 0u;
            int i = lo;
            for (; i + 4 <= hi; i += 4) {
                p0 |= xr.left_bit<ONE_BYTE>(rec[i]);
                p1 |= xr.left_bit<ONE_BYTE>(rec[i + 1]);
                p2 |= xr.left_bit<ONE_BYTE>(rec[i + 2]);
                p3 |= xr.left_bit<ONE_BYTE>(rec[i + 3]);
            }
            for (; i < hi; ++i) p0 |= xr.left_bit<ONE_BYTE>(rec[i]);
            dw[w] = m.pt[w] | p0 | p1 | p2 | p3;
            lo = hi;
        }
    }
}

template <int D>
__device__ __forceinline__ uint32_t dbit(const uint32_t (&dw)[Shape<D>::NW], int v) {
    return (dw[v >> 5] >> (v & 31)) & 1u;
}

// Two adjacent decision bits, v and v + 1 (bit 0 = node v), of the decision words.
template <int D>
__device__ __forceinline__ uint32_t dbit2(const uint32_t (&dw)[Shape<D>::NW], int v) {
    if ((v & 31) != 31) return (dw[v >> 5] >> (v & 31)) & 3u;
    return ((dw[v >> 5] >> 31) | (dw[(v >> 5) + 1] << 1)) & 3u;
}

// Entry index of the row at every bottom subtree (wdf_internal.h): the ancestors' raw
// decisions R are built once per node of depth < D-2 (siblings share them), then each
// entry takes d_r and the adjacent pair d_{2r+1}, d_{2r+2} in one extraction.
template <int D>
__device__ __forceinline__ void subtree_entries(const uint32_t (&dw)[Shape<D>::NW], uint32_t (&ent)[Shape<D>::NS]) {
    constexpr int NS = Shape<D>::NS;
    uint32_t R[NS > 1 ? NS - 1 : 1];  // R of the children of node v, v < NS - 1
#pragma unroll
    for (int v = 0; v < NS - 1; ++v) R[v] = ((v == 0 ? 0u : R[(v - 1) >> 1]) << 1) | dbit<D>(dw, v);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const int r = NS - 1 + s;
        const uint32_t Rr = r == 0 ? 0u : R[(r - 1) >> 1];
        ent[s] = (Rr << 3) | (dbit<D>(dw, r) << 2) | dbit2<D>(dw, 2 * r + 1);
    }
}

// Decision code of value x in one code column (tree_layout.h): the number of the
// column's sorted thresholds u with u <= x, by binary search; the count for NaN.
__device__ __forceinline__ int decision_code(float x, const float *__restrict__ u, const CodeCol &c) {
    if (x != x) return c.count;
    int pos = 0;
    for (int step = c.top; step > 0; step >>= 1)
        if (pos + step <= c.count && __ldg(u + pos + step - 1) <= x) pos += step;
    return pos;
}

}  // namespace wdf
