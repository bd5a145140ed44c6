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
// Flush sequence of a tree of depth D (NS = 2^(D-2) bottom subtrees): the three inner
// nodes r, 2r+1, 2r+2 of every bottom subtree (r = NS - 1 + s, s = 0..NS-1), padded to a
// multiple of 8; then the inner nodes above the bottom subtrees (0..NS-2), padded to a
// multiple of 8.  Batch b is positions [8b, 8b + 8).  A batch whose real features are
// all distinct can read all its phi values before writing any.
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
    uint32_t flush;   // bit b: consumer flush batch b repeats no real feature
    uint8_t wend[8];  // NodeRec index one past the last node of word w
    uint32_t real;    // bit b: consumer flush batch b holds a real (not pass-through) node
};
static_assert(sizeof(NodeRec) == 16, "NodeRec is one 16-byte load");
static_assert(sizeof(TreeMeta) == 56, "TreeMeta layout");

// One code column: source feature, first threshold in the sorted threshold array,
// threshold count, and the largest power of two <= count (0 when count is 0).  With
// one-byte codes every column occupies 255 entries of the array (NaN after its count).
struct CodeCol {
    int32_t feature, first, count, top;
};

WDF_HD constexpr int flush_len_bottom(int D) { return (3 * (1 << (D - 2)) + 7) & ~7; }
WDF_HD constexpr int flush_len_upper(int D) { return ((1 << (D - 2)) - 1 + 7) & ~7; }
WDF_HD constexpr int flush_len(int D) { return flush_len_bottom(D) + flush_len_upper(D); }
WDF_HD constexpr int flush_batches(int D) { return flush_len(D) / 8; }

// Heap index of the node at flush position i, -1 for padding.
WDF_HD inline int flush_node(int D, int i) {
    const int NS = 1 << (D - 2);
    if (i < 3 * NS) {
        const int r = NS - 1 + i / 3, c = i % 3;
        return c == 0 ? r : 2 * r + c;
    }
    if (i < flush_len_bottom(D)) return -1;
    const int u = i - flush_len_bottom(D);
    return u < NS - 1 ? u : -1;
}

static_assert(flush_batches(8) <= 32, "batch flags are one 32-bit word per tree");

}  // namespace wdf
