// Internal declarations of the GB300 Background-SHAP library (not part of the ABI).
//
// Layout used by every kernel ("complete layout"): each tree is re-laid out as a
// complete binary tree of the ensemble's depth D (2 <= D <= 8) in heap order -- inner
// node v has children 2v+1 (left) and 2v+2 (right); leaf q (0-based from the left) is
// heap position NI + q.  A leaf of the input at depth d < D is pushed down to depth D
// through "pass-through" nodes that send every row left (they test a virtual feature
// column F that is always 0 against threshold 1); the pushed-down leaf keeps the
// output, the other leaves below a pass-through node get output 0.  This changes no
// value: on a pass-through node both the consumer and the baseline follow the path to
// the kept leaf, which is rule 3 of the cube construction (no literal), and leaves
// of output 0 add nothing.
//
// "Bottom subtree" s (0 <= s < NS = 2^(D-2)) is the complete subtree of height 2 rooted
// at heap node r = NS - 1 + s: three inner nodes r, 2r+1, 2r+2 and four leaves 4s..4s+3.
// Everything consumer-side is indexed by the "entry" of a row at a bottom subtree:
//   e = (R << 3) | (d_r << 2) | (d_{2r+2} << 1) | d_{2r+1},
// d_v = 1 when the row goes left at node v, R = the d of the D-2 ancestors of r (root
// first).  The row's decision pattern at r (Algorithm 1: bit = the row follows the
// path to r) is R ^ s, since s's bits root first are the path's turns (1 = right).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "tree_layout.h"

namespace wdf {

constexpr int kMaxDepth = 8;
constexpr int kMinDepth = 2;

struct Packed {
    int F = 0, T = 0, D = 0;
    int NI = 0, NL = 0, NS = 0;
    std::vector<int32_t> node_feat;   // [T][NI]  F for pass-through nodes
    std::vector<float> node_thr;      // [T][NI]
    std::vector<float> leaf_w;        // [T][NL]
    std::vector<uint64_t> live;       // [T] bit s: bottom subtree s has a non-zero leaf
    // decision records of the kernels (tree_layout.h): per tree the real inner nodes
    // (rec[t * NI ...], meta[t].wend[7] of them) and the tree's metadata; the code
    // columns and their sorted thresholds
    std::vector<NodeRec> rec;         // [T][NI]
    std::vector<TreeMeta> meta;       // [T]
    std::vector<int32_t> flush_feat;  // [T][flush_len(D)] feature at each consumer flush position (F: padding
                                      // and pass-through nodes)
    std::vector<uint64_t> xmask;      // [T][6] (depth <= 6) expand_masks of the tree's real nodes
    std::vector<CodeCol> cols;        // [n_cols]
    std::vector<float> col_thr;       // column segments of the sorted distinct thresholds
    int code_bytes = 1;               // 1 or 2
    // live leaves grouped by path signature (first-occurrence positions)
    std::vector<uint32_t> sig_key;    // [G] 3 bits per path position
    std::vector<int32_t> group_off;   // [G+1]
    std::vector<int32_t> group_leaf;  // [n_live] t * NL + q, grouped
    std::vector<int32_t> leaf_row;    // [T][NL] row of the leaf in group_leaf, -1 if not live
    // per tree and complete-layout position (inner nodes then leaves): the local input
    // node whose cover the position carries, -1 for a zero cover; and the input offsets
    std::vector<int32_t> heap_src;    // [T][NI + NL]
    std::vector<int64_t> in_off;      // [T + 1]
};

// Path-dependent cover ratios of every live leaf row (group_leaf order): ratio[row][k] =
// cover(path node k+1) / cover(path node k) (0 where the node's cover is 0), from the
// covers of the input nodes (indexed like the input arrays).  Returns a wdf_status.
int pd_ratios(const Packed &p, const double *cover, std::vector<double> *ratio, std::string *err);

// Validates and lays out an ensemble; returns a wdf_status value and fills err.
int pack_ensemble(int F, int T, const int64_t *off, const int32_t *feat, const float *thr, const int32_t *left,
                  const int32_t *right, const float *val, Packed *out, std::string *err);

// Sets the thread-local message returned by wdf_last_error.
void set_last_error(const std::string &msg);

// A named range on the NVTX timeline (Nsight Systems, ncu's range filters) for the
// duration of one C-ABI call or one server wave; a no-op when no tool is attached.
struct TraceRange {
    explicit TraceRange(const char *name);
    ~TraceRange();
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

// Move masks of the expand of Hacker's Delight section 7-5 for mask m: expanding x with
// them puts bit k of x at the position of the k-th set bit of m (bits of x at or above
// popcount(m) must be zero) and leaves copies of bits only at positions outside m, which
// the consumer kernel ORs with the pass-through bits (all ones there) instead of
// masking.  Six steps, for shifts of 32, 16, ..., 1.
inline void expand_masks(uint64_t m, uint64_t mv[6]) {
    uint64_t mk = ~m << 1;  // bit p: the number of zeros of m below p is odd, after the prefix steps
    for (int i = 0; i < 6; ++i) {
        uint64_t mp = mk ^ (mk << 1);
        for (int s = 2; s < 64; s <<= 1) mp ^= mp << s;
        const uint64_t v = mp & m;  // the bits of m that move 2^i further in this step
        mv[i] = v;
        m = (m ^ v) | (v >> (1 << i));
        mk &= ~mp;
    }
}

}  // namespace wdf
