// Kernel launchers (internal).  Every launcher enqueues on the given stream and
// returns the launch status; none of them allocates.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "tree_layout.h"

namespace wdf {

// Counts kernel launches (every launcher adds the kernels it enqueued).
void count_launches(int k);

// Device arrays describing the complete layout of an ensemble (see wdf_internal.h and
// tree_layout.h).
struct TreeArrays {
    const int2 *nodes;        // [T][NI] (feature, threshold bits); feature F = pass-through
    const NodeRec *rec;       // [T][NI] real inner nodes of every tree
    const TreeMeta *meta;     // [T]
    const CodeCol *cols;      // [n_cols] decision-code columns
    const float *col_thr;     // their sorted thresholds
    int n_cols, code_bytes;   // code_bytes: 1 or 2
    const unsigned long long *xmask;  // [T][6] (depth <= 6) expand masks of the real nodes
};

// Everything the consumer kernel needs about one ensemble.
struct ExplainJob {
    TreeArrays ta;
    const float *sfold;     // folded slot vectors [T][NS][2^(D+1)][SP], entry e at line_pos(e)
    const uint32_t *lines;  // per tree lines_words(D) words: byte s = line map of subtree s
    const int32_t *flfeat;  // [T][flush_len(D)] feature of the node at each flush position (F: none)
    int T, F;
};

// Where the consumer gathers land.  A warp's 32-byte gathers of one bottom subtree are
// served a quarter warp at a time, one L1 wavefront per distinct 128-byte line, and a
// line holds four consecutive entries.  Entries are formed from D + 1 decision bits;
// the entry of subtree s is stored rotated right by r_s bits, r_s chosen so that the two
// bits that land in the two lowest positions (within a line) are the adjacent pair
// (cyclically) whose background frequencies are closest to one half: the rows of a
// quarter warp mostly agree on the more certain decisions, so they land in fewer lines.
// The map of subtree s is the byte r_s (0 is the identity).  A rotation keeps nearly all
// of the gain of moving the best two bits anywhere, for a third of the instructions.
__host__ __device__ __forceinline__ uint32_t line_pos(uint32_t e, uint32_t r, int D) {
    const uint32_t nb = (uint32_t)D + 1u;
    return ((e >> r) | (e << (nb - r))) & ((1u << nb) - 1u);
}
// 32-bit words of line maps per tree: one byte per bottom subtree, at least four words
// so that a tree's maps are whole 16-byte loads.
__host__ __device__ constexpr int lines_words(int D) { return (1 << (D - 2)) / 4 < 4 ? 4 : (1 << (D - 2)) / 4; }

// One request of a ragged batch: n consumer rows at C (row stride ldc), phi out; codes
// receives the rows' decision code blocks (rows padded to a multiple of 128), job is
// the slot of the request's ensemble among its class's jobs.
struct BatchRequest {
    const float *C;
    float *phi;
    unsigned char *codes;
    int64_t n, ldc, ldp;
    int job;
};

struct DevInfo {
    int sms = 0;
    size_t smem_optin = 0;  // max dynamic shared memory per block
};

// Step 1 of Algorithm 3 (background): joint entry counts hist[T][NS][2^(D+1)] (u32,
// must be zeroed by the caller) of the background rows at every bottom subtree.  The
// rows are encoded to decision codes (tree_layout.h) in chunks of code_rows rows into
// codes (code_rows * n_cols * code_bytes bytes; code_rows a positive multiple of
// kBgMaxTileRows), each chunk then counted.
constexpr int kBgMaxTileRows = 512;

// Decision codes of rows [0, rows) of X (row stride ldx) into codes, in 32-row code
// blocks (wdf_device.cuh); rows up to rows_pad (a multiple of 32) get code 0.
cudaError_t launch_encode_codes(const float *X, int64_t rows, int64_t ldx, const TreeArrays &ta, int64_t rows_pad,
                                unsigned char *codes, cudaStream_t st);
// With ov, chunks alternate between codes and ov->codes1 and are encoded on ov->side, so
// the encode of chunk k + 1 overlaps the count of chunk k (events order each buffer's
// encode after its previous count and each count after its encode); st still ends
// after all of it.
struct BgOverlap {
    unsigned char *codes1;
    cudaStream_t side;
    cudaEvent_t enc[2], cnt[2];
};
cudaError_t launch_bg_hist(int D, const float *B, int64_t m, int64_t ldb, const TreeArrays &ta, int T,
                           unsigned char *codes, int64_t code_rows, uint32_t *hist, const DevInfo &dev,
                           cudaStream_t st, const BgOverlap *ov = nullptr);

// Per-leaf pattern counts vc[row][p] (u32, 2^D per row) of the live leaves, marginals of
// the joint entry counts; A (nullable) receives them as FP32.
cudaError_t launch_leaf_counts(int D, const uint32_t *hist, const int32_t *group_leaf, int n_live, uint32_t *vc,
                               float *A, cudaStream_t st);

// Path-dependent pattern frequencies A[row][p] (FP32, 2^D per row) from the per-leaf
// cover ratios ratio[row][k] (FP64, D per row).
cudaError_t launch_pd_freq(int D, const double *ratio, int n_live, float *A, cudaStream_t st);

// Step 2: FP64 pattern-pair tables of G path signatures; t32 (and t64 when non-null)
// laid out [G][2^D][D * 2^D].  metric 0: Shapley values, 1: Banzhaf values.
cudaError_t launch_tables(int D, int metric, const uint32_t *sig_keys, int G, float *t32, double *t64,
                          cudaStream_t st);

// Step 3 on CUDA cores: S[row][k * 2^D + p_c] = scale[row] * sum_p A[row][p] *
// T[g][p][k * 2^D + p_c] for every live leaf row of group g (A: background counts or
// path-dependent frequencies).  tiles: (group, row0, row_end, 0) items of up to 64 rows.
// slots: output slots per pattern (0: D, one per path position; D(D-1)/2 for pairs).
cudaError_t launch_contract_fp32(int D, const float *A, const float *scale, const int4 *tiles, int n_tiles,
                                 const float *t32, float *S, cudaStream_t st, int slots = 0);

// Step 3 on the tensor cores (tcgen05, TMEM accumulators): the same S as
// launch_contract_fp32 from split-precision operands: mode 0 = TF32 hi+lo, 1 = BF16
// hi+lo (three products each), 2 = BF16 hi+mid+lo (six products).  The operands are
// split once into the core-matrix stages the MMAs read: B (the tables, per signature) by
// launch_pack_b into bpk (contract_tc_b_bytes), A (the frequencies) by the contraction
// itself into apk (contract_tc_a_bytes: room for any mode).  tiles: (group, row0,
// row_end, 0) work items of up to 128 rows.  err is set to 1 if a bounded wait expired.
struct TcGeom {
    int NT, NB, nk, ring, np;  // N per CTA, column blocks, K steps, ring stages, operand parts
    uint32_t a_stage, b_stage;  // bytes of one stage of A and of B
    size_t smem;
};
TcGeom tc_geom(int D, int mode);
size_t contract_tc_a_bytes(int D, int n_tiles);
size_t contract_tc_b_bytes(int D, int mode, int G);
cudaError_t launch_pack_b(int D, int mode, const float *t32, int G, unsigned char *bpk, cudaStream_t st);
cudaError_t launch_contract_tc(int D, int mode, const float *A, const float *scale, const int4 *tiles, int n_tiles,
                               unsigned char *apk, const unsigned char *bpk, float *S, int *err, cudaStream_t st);
// Test hook: poll limit of the first mbarrier wait of every CTA of later launches (0
// restores the normal limit).
void set_contract_first_wait_limit(uint32_t polls);

// Folds the per-leaf S rows of every bottom subtree into per-entry slot vectors
// sfold[T][NS][2^(D+1)][SP] (see wdf_internal.h).
cudaError_t launch_fold(int D, const float *S, const int32_t *leaf_row, int T, const uint32_t *lines, float *sfold,
                        cudaStream_t st);
// Line maps of every bottom subtree from the joint background counts hist (hist null:
// the identity map, used for the path-dependent frequencies).
cudaError_t launch_line_maps(int D, const uint32_t *hist, int T, uint32_t *lines, cudaStream_t st);

// scale[row] = w[row] / m.
cudaError_t launch_scale(const double *w, int n_live, int64_t m, float *scale, cudaStream_t st);

// v({}) in FP64 (one block): sum over live leaves of w * vc[all ones] / m, or, when
// ratio is non-null (path-dependent game), of w * (product of the leaf's cover ratios).
cudaError_t launch_base_value(int D, const uint32_t *vc, const double *ratio, const double *leaf_w_rows, int n_live,
                              int64_t m, double *out, cudaStream_t st);

// Step 4: phi of n consumer rows, tile_rows consumer rows per block (32, 64 or 128;
// 0 picks the default for the shared-memory budget).
cudaError_t launch_explain(int D, const float *C, int64_t n, int64_t ldc, const ExplainJob &job, float *phi,
                           int64_t ldp, int tile_rows, const DevInfo &dev, cudaStream_t st);
// Consumer-kernel timing (process-wide): while on, launch_explain brackets every
// consumer-kernel launch with a pair of CUDA events on its stream; explain_timing_read
// waits for the recorded pairs, returns the summed milliseconds and the launch count, and
// forgets them.  Turning it on or off also forgets them.
void explain_timing(bool on);
cudaError_t explain_timing_read(double *ms, int64_t *launches);
// xb: decision-code bytes per row (code columns x code bytes).
int default_tile_rows(int D, int F, int xb, const DevInfo &dev);
size_t explain_smem_bytes(int D, int F, int xb, int tile_rows);

// Decision codes of a ragged batch's rows: items (request, 32-row block), *n_items read on
// the device; a grid of `grid` blocks walks them.
cudaError_t launch_encode_batch(const ExplainJob *jobs, const BatchRequest *reqs, const int2 *items,
                                const int *n_items, int grid, cudaStream_t st);

// Step 4 for a ragged batch of one depth: a persistent grid (grid <= 0: one wave at full
// occupancy) walks the work items (job, request, first row split as hi/lo words);
// *n_items is read on the device; the rows' codes come from launch_encode_batch.  F_max and xb_max bound the feature count and the
// decision-code bytes per row of every job.
cudaError_t launch_explain_batch(int D, const ExplainJob *jobs, const BatchRequest *reqs, const int4 *items,
                                 int *n_items, int F_max, int xb_max, int tile_rows, int grid, const DevInfo &dev,
                                 cudaStream_t st);

// Interaction values (k_interactions.cu).  Pair tables t2 [G][2^D][P * 2^D] (P =
// D(D-1)/2 position pairs) for metric 0 (Shapley) or 1 (Banzhaf); the contraction is
// launch_contract_fp32 with slots = P; S2T [n_live][2^D][PP] (PP = P rounded up to 4);
// out [n][F][F] at row stride ldo.
cudaError_t launch_tables_iv(int D, int metric, const uint32_t *sig_keys, int G, float *t2, cudaStream_t st);
cudaError_t launch_iv_pack(int D, int PP, const float *S2, int n_live, float *S2T, cudaStream_t st);
// depth <= 6: the pair values folded per (tree, bottom subtree, entry), followed by a
// byte table of node features (iv_fold_floats words in all; launch_explain_iv writes the
// table); the consumer kernel then takes whole trees (fold non-null) instead of leaves
size_t iv_fold_floats(int D, int T);
cudaError_t launch_iv_fold(int D, const float *S2, const int32_t *leaf_row, int T, float *fold, cudaStream_t st);
cudaError_t launch_explain_iv(int D, const float *C, int64_t n, int64_t ldc, int F, const TreeArrays &ta, int T,
                              const int32_t *group_leaf, int n_live, const float *S2T, float *fold, float *out,
                              int64_t ldo, const DevInfo &dev, cudaStream_t st);

// FP64 column means of |phi| and phi: partial sums per row block, then a fixed-order
// final sum.  partial holds global_attr_partial_doubles(n, F) doubles.
int64_t global_attr_blocks(int64_t n);
int64_t global_attr_partial_doubles(int64_t n, int F);
cudaError_t launch_global_attr(const float *phi, int64_t n, int64_t ldp, int F, double *partial,
                               double *mean_abs, double *mean, cudaStream_t st);

}  // namespace wdf
