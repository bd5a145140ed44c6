// Order in which the consumer kernel adds a tree's per-node values into phi (shared by
// the host, which marks the batches that repeat no feature, and the device).
//
// Flush sequence of a tree of depth D (NS = 2^(D-2) bottom subtrees): the three inner
// nodes r, 2r+1, 2r+2 of every bottom subtree (r = NS - 1 + s, s = 0..NS-1), padded to a
// multiple of 8; then the inner nodes above the bottom subtrees (0..NS-2), padded to a
// multiple of 8.  Batch b is positions [8b, 8b + 8).  A batch whose real features are
// all distinct can read all its phi values before writing any.
#pragma once

#if defined(__CUDACC__)
#define WDF_HD __host__ __device__
#else
#define WDF_HD
#endif

namespace wdf {

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
