// Per-tree records shared by the host packer and the kernels (plain structs, no device
// code), and the order in which the consumer kernel adds a tree's node values into phi.
//
// Decision codes.  Every real inner node tests x[f] < thr (Def. "decision_tree").  The
// packer sorts the distinct thresholds of each feature and cuts the sorted list into
// "code columns" of at most 255 (one-byte codes) or 65535 (two-byte codes) thresholds.
// A row's code in column c is the number of the column's thresholds u with u <= x (the
// column's threshold count when x is NaN).  A node whose threshold is the k-th of its
// column (rank k, 0-based) sends the row left exactly when code <= k, because the
// thresholds are sorted: x < u_k  <=>  fewer than k + 1 of them are <= x.  A NaN
// threshold never sends a row left (rank -1).  The kernels stage codes instead of
// floats: one or two bytes per column and row instead of four per feature.
//
// Flush sequence of a tree of depth D (NS = 2^(D-2) bottom subtrees, cut into NG groups
// of GS = gather_group(D) consecutive subtrees, the gather groups of the consumer
// kernel).  Per group g: the three inner nodes r, 2r+1, 2r+2 of each of its subtrees (r =
// NS - 1 + s), padded to a multiple of 8; then the GS - 1 inner nodes of the height-
// log2(GS) subtree whose leaves are the group's subtree roots (heap order within it),
// padded to a multiple of 8.  After the groups: the NG - 1 nodes above them (heap 0 ..
// NG - 2), padded to a multiple of 8.  With one group (D <= 6) this is all bottom nodes,
// then all nodes above them.  Batch b is positions [8b, 8b + 8).  A batch whose real
// features are all distinct can read all its phi values before writing any.
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define WDF_HD __host__ __device__
#else
#define WDF_HD
#endif

namespace wdf {

// One real inner node of a tree, in the order the decision loop visits them (heap
// order, so the nodes of each 32-node word of the heap index are contiguous).
struct NodeRec {
    int32_t col_off;  // byte offset of the node's code column in a 32-row code block
    int32_t rank;     // left when code <= rank; -1 for a NaN threshold
    // the node's decision bit: trees of at most 64 inner nodes (depth <= 6) carry it in
    // two words (bit_lo: heap index < 32, bit_hi: the rest), deeper trees as the bit
    // within its word (bit_lo, bit_hi = 0)
    uint32_t bit_lo, bit_hi;
};

struct TreeMeta {
    uint32_t pt[8];   // bit v of word v/32: inner node v is a pass-through node (always left)
    uint64_t live;    // bit s: bottom subtree s has a non-zero leaf
    uint64_t flush;   // bit b: consumer flush batch b repeats no real feature
    uint8_t wend[8];  // NodeRec index one past the last node of word w
    uint64_t real;    // bit b: consumer flush batch b holds a real (not pass-through) node
};
static_assert(sizeof(NodeRec) == 16, "NodeRec is one 16-byte load");
static_assert(sizeof(TreeMeta) == 64, "TreeMeta layout");

// One code column: source feature, first threshold in the sorted threshold array,
// threshold count, and the largest power of two <= count (0 when count is 0).  With
// one-byte codes every column occupies 255 entries of the array (NaN after its count).
struct CodeCol {
    int32_t feature, first, count, top;
};

// Floats per entry of the folded slot vectors: D - 2 ancestors and the three nodes of the
// bottom subtree, padded to 4, 8 or 12.
WDF_HD constexpr int slots_per_entry(int D) { return (D + 1) <= 4 ? 4 : ((D + 1) <= 8 ? 8 : 12); }
// Bottom subtrees per gather group: the largest power of two <= NS whose slot vectors fit
// in 128 registers.
WDF_HD constexpr int gather_group(int D) {
    int g = 1 << (D - 2);
    while (g > 1 && g * slots_per_entry(D) > 128) g /= 2;
    return g;
}
WDF_HD constexpr int pad8(int n) { return (n + 7) & ~7; }
WDF_HD constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }
WDF_HD constexpr int flush_groups(int D) { return (1 << (D - 2)) / gather_group(D); }
WDF_HD constexpr int flush_group_bottom(int D) { return pad8(3 * gather_group(D)); }
WDF_HD constexpr int flush_group_len(int D) { return flush_group_bottom(D) + pad8(gather_group(D) - 1); }
WDF_HD constexpr int flush_len(int D) { return flush_groups(D) * flush_group_len(D) + pad8(flush_groups(D) - 1); }
WDF_HD constexpr int flush_batches(int D) { return flush_len(D) / 8; }

// Heap index of the node at flush position i, -1 for padding.
WDF_HD inline int flush_node(int D, int i) {
    const int NS = 1 << (D - 2), GS = gather_group(D), NG = NS / GS, GL = flush_group_len(D);
    if (i >= NG * GL) {
        const int u = i - NG * GL;
        return u < NG - 1 ? u : -1;
    }
    const int g = i / GL, k = i - g * GL;
    if (k < 3 * GS) {
        const int r = NS - 1 + g * GS + k / 3, c = k % 3;
        return c == 0 ? r : 2 * r + c;
    }
    const int u = k - flush_group_bottom(D);  // node of the group's upper subtree, heap order
    if (u < 0 || u >= GS - 1) return -1;
    const int l = ilog2(u + 1);          // level of u within the group's subtree
    const int lg = D - 2 - ilog2(GS) + l;  // its level in the tree
    return (1 << lg) - 1 + g * (1 << l) + (u - ((1 << l) - 1));
}

static_assert(flush_batches(8) <= 64, "batch flags are one 64-bit word per tree");

}  // namespace wdf
