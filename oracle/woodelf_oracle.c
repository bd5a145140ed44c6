/*
 * woodelf_oracle.c -- plain FP64 CPU oracle for Background (interventional) SHAP
 * and Banzhaf values of decision-tree ensembles.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code, header,
 * table or helper with the CUDA path, and it never reads anything the CUDA path
 * produced.
 *
 * What it computes (paper section "Efficient Background SHAP Equation"): for a
 * consumer row c and a background matrix B of m rows, the interventional game
 *     v_c(S) = (1/m) sum_{b in B} f(x^S),   x^S_i = c_i if i in S else b_i,
 * where f(x) is the plain sum of the trees' leaf outputs (section "WOODELF
 * Algorithm": run per tree and sum), and its Shapley value (Eq. "s") or Banzhaf
 * value (Eq. "banzhaf_combinatorial_def") for every feature.
 *
 * Three tiers, each pinned by the tests against the others and against the paper:
 *   O0  orc_values_bruteforce -- the definition written out: v_c(S) for all 2^F
 *       coalitions, then Eq. "s" (or the Banzhaf sum).  Tiny F only.
 *   O1  orc_values_pairs -- Eq. "trival_bg": for every (consumer, background row)
 *       pair the leaf cube is built by the four construction rules of section
 *       "Constructing a WDNF Representation" and valued by Formula
 *       "shap_simplified_formula" (or "banzhaf_simplified_formula").  Leaves whose
 *       cube is bottom by rule 4 are not visited.
 *   O2  orc_bg_hist + orc_values_hist -- Eq. "bg_shap_derivation" steps (c)-(d): the
 *       background is reduced to exact per-leaf pattern counts vc[l][p_b] computed by
 *       CalcDecisionPatterns (Algorithm 1), then every (consumer pattern, counted
 *       background pattern) cube is valued and weighted by vc/m.
 * Interaction values (section "Beyond SHAP": Def. "shap_iv_def" for Shapley, Def.
 * "banzhaf_iv_def" for Banzhaf) of every feature pair of the same background game:
 *   orc_iv_bruteforce -- v_c(S) for all coalitions, then the definitions written out;
 *   orc_iv_hist -- the counts of O2 with Table "table_shap_iv" (or Formula
 *       "banzhaf_simplified_formula_interactions") in place of the value formula.
 * The path-dependent game (covers instead of a background) has the same two ends:
 *   orc_pd_values_bruteforce -- v_c(S) as the cover-weighted expectation walk for all
 *       coalitions, then Eq. "s";
 *   orc_pd_values -- the frequency form of section "Efficient Path-Dependent SHAP
 *       Equation" (Eq. "path_dependent_estimation") in place of vc/m.
 *
 * Conventions read from the paper:
 *   - split(x) = x[feature] < threshold, strict, True goes left (Def. "decision_tree");
 *     a NaN compares false and goes right.
 *   - a decision pattern has one bit per inner node on the root-to-leaf path, root
 *     first as the most significant bit (Algorithm 1 shifts left; the path-dependent
 *     example reads pattern 5 = 101 root first).
 *   - cubes are feature sets: a feature met at several nodes of one path enters once;
 *     a cube holding a feature and its negation is unsatisfiable and dropped.
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC woodelf_oracle.c -o liboracle.so -lm
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXD 24
#define ORC_SHAPLEY 0
#define ORC_BANZHAF 1

typedef struct {
    int32_t n_trees;
    const int64_t *off;
    const int32_t *feat;
    const float *thr;
    const int32_t *left;
    const int32_t *right;
    const float *val;
} ens_t;

typedef struct {
    int32_t tree, node, depth;
    int32_t path[ORC_MAXD];      /* local ids of the inner nodes on the root-to-leaf path */
    uint8_t goes_left[ORC_MAXD]; /* 1 when the path continues to that node's left child */
    double w;                    /* leaf output */
    int64_t hoff;                /* offset of this leaf's 2^depth pattern counts */
} leaf_t;

typedef struct {
    int64_t n;
    int64_t hist_size;
    int32_t max_tree_nodes;
    leaf_t *v;
    int32_t *leaf_of_node; /* global node index -> leaf index, -1 for inner nodes */
} leafset_t;

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Def. "decision_tree": split(c) = c[n.feature] < theta_n. */
static int split_true(const float *x, int32_t f, float th) { return x[f] < th; }

static uint64_t binom(int n, int k) {
    if (k < 0 || k > n) return 0;
    if (k > n - k) k = n - k;
    uint64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (uint64_t)(n - k + i) / (uint64_t)i;
    return r;
}

/* ---------------------------------------------------------------- leaves */

static int collect_rec(const ens_t *e, int t, int32_t node, int depth, int32_t *path, uint8_t *gl,
                       leafset_t *ls, int64_t tree_size) {
    if (node < 0 || node >= tree_size || depth > ORC_MAXD) return -1;
    int64_t g = e->off[t] + node;
    if (e->feat[g] < 0) {
        leaf_t *L = &ls->v[ls->n];
        L->tree = t; L->node = node; L->depth = depth; L->w = (double)e->val[g];
        memcpy(L->path, path, sizeof(int32_t) * (size_t)depth);
        memcpy(L->goes_left, gl, (size_t)depth);
        L->hoff = ls->hist_size;
        ls->hist_size += (int64_t)1 << depth;
        ls->leaf_of_node[g] = (int32_t)ls->n;
        ls->n++;
        return 0;
    }
    if (depth == ORC_MAXD) return -1;
    path[depth] = node;
    gl[depth] = 1;
    if (collect_rec(e, t, e->left[g], depth + 1, path, gl, ls, tree_size)) return -1;
    gl[depth] = 0;
    if (collect_rec(e, t, e->right[g], depth + 1, path, gl, ls, tree_size)) return -1;
    return 0;
}

/* All leaves, tree by tree, each tree depth first with the left child first. */
static int collect_leaves(const ens_t *e, leafset_t *ls) {
    int64_t total = e->off[e->n_trees];
    memset(ls, 0, sizeof(*ls));
    ls->v = (leaf_t *)calloc((size_t)(total > 0 ? total : 1), sizeof(leaf_t));
    ls->leaf_of_node = (int32_t *)malloc(sizeof(int32_t) * (size_t)(total > 0 ? total : 1));
    if (!ls->v || !ls->leaf_of_node) return -1;
    for (int64_t i = 0; i < total; ++i) ls->leaf_of_node[i] = -1;
    int32_t path[ORC_MAXD];
    uint8_t gl[ORC_MAXD];
    for (int t = 0; t < e->n_trees; ++t) {
        int64_t sz = e->off[t + 1] - e->off[t];
        if (sz > ls->max_tree_nodes) ls->max_tree_nodes = (int32_t)sz;
        if (collect_rec(e, t, 0, 0, path, gl, ls, sz)) return -1;
    }
    return 0;
}

static void free_leaves(leafset_t *ls) {
    free(ls->v);
    free(ls->leaf_of_node);
}

int64_t orc_leaf_count(int32_t n_trees, const int64_t *off, const int32_t *feat, const float *thr,
                       const int32_t *left, const int32_t *right, const float *val) {
    ens_t e = {n_trees, off, feat, thr, left, right, val};
    leafset_t ls;
    if (collect_leaves(&e, &ls)) { free_leaves(&ls); return -1; }
    int64_t n = ls.n;
    free_leaves(&ls);
    return n;
}

/* Leaf table in the oracle's order: tree, local node id, depth, and the offset of the
 * leaf's pattern counts in orc_bg_hist's output.  Returns the total count size. */
int64_t orc_leaf_table(int32_t n_trees, const int64_t *off, const int32_t *feat, const float *thr,
                       const int32_t *left, const int32_t *right, const float *val,
                       int32_t *leaf_tree, int32_t *leaf_node, int32_t *leaf_depth, int64_t *leaf_hoff) {
    ens_t e = {n_trees, off, feat, thr, left, right, val};
    leafset_t ls;
    if (collect_leaves(&e, &ls)) { free_leaves(&ls); return -1; }
    for (int64_t i = 0; i < ls.n; ++i) {
        leaf_tree[i] = ls.v[i].tree;
        leaf_node[i] = ls.v[i].node;
        leaf_depth[i] = ls.v[i].depth;
        leaf_hoff[i] = ls.v[i].hoff;
    }
    int64_t hs = ls.hist_size;
    free_leaves(&ls);
    return hs;
}

/* ---------------------------------------------------------------- prediction */

static double tree_value(const ens_t *e, int t, const float *x) {
    int64_t o = e->off[t];
    int32_t v = 0;
    while (e->feat[o + v] >= 0) v = split_true(x, e->feat[o + v], e->thr[o + v]) ? e->left[o + v] : e->right[o + v];
    return (double)e->val[o + v];
}

static double ens_value(const ens_t *e, const float *x) {
    double s = 0.0;
    for (int t = 0; t < e->n_trees; ++t) s += tree_value(e, t, x);
    return s;
}

/* f(x) for every row: the sum of the leaf outputs the row reaches. */
int orc_predict(int32_t n_trees, const int64_t *off, const int32_t *feat, const float *thr,
                const int32_t *left, const int32_t *right, const float *val,
                const float *X, int64_t n, int64_t ld, double *out) {
    ens_t e = {n_trees, off, feat, thr, left, right, val};
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < n; ++r) out[r] = ens_value(&e, X + r * ld);
    return 0;
}

/* ---------------------------------------------------------------- cube values */

/* Distinct positive / negated feature sets of a cube; returns 0 when unsatisfiable. */
static int cube_sets(const int32_t *pos, int np, const int32_t *neg, int nn, int32_t *P, int *a, int32_t *N, int *b) {
    *a = 0; *b = 0;
    for (int i = 0; i < np; ++i) {
        int dup = 0;
        for (int j = 0; j < *a; ++j) dup |= (P[j] == pos[i]);
        if (!dup) P[(*a)++] = pos[i];
    }
    for (int i = 0; i < nn; ++i) {
        int dup = 0;
        for (int j = 0; j < *b; ++j) dup |= (N[j] == neg[i]);
        if (!dup) N[(*b)++] = neg[i];
    }
    for (int i = 0; i < *a; ++i)
        for (int j = 0; j < *b; ++j)
            if (P[i] == N[j]) return 0;
    return 1;
}

/* Formula "shap_simplified_formula" (metric 0) or "banzhaf_simplified_formula"
 * (metric 1) for one satisfiable weighted cube with distinct sets P and N. */
static void cube_value(const int32_t *P, int a, const int32_t *N, int b, double w, int metric, double *phi) {
    int s = a + b;
    if (s == 0) return;
    if (metric == ORC_SHAPLEY) {
        if (a > 0) {
            double v = w / ((double)a * (double)binom(s, a));
            for (int i = 0; i < a; ++i) phi[P[i]] += v;
        }
        if (b > 0) {
            double v = w / ((double)b * (double)binom(s, b));
            for (int i = 0; i < b; ++i) phi[N[i]] -= v;
        }
    } else {
        double v = w / ldexp(1.0, s - 1);
        for (int i = 0; i < a; ++i) phi[P[i]] += v;
        for (int i = 0; i < b; ++i) phi[N[i]] -= v;
    }
}

/* ---------------------------------------------------------------- WDNF level */

/* WDNF evaluation (Def. "WDNF"): sum of the weights of the satisfied cubes. */
int orc_wdnf_eval(int32_t h, int32_t K, const double *w, const int64_t *lit_off, const int32_t *lit_var,
                  const uint8_t *lit_neg, const uint8_t *x, double *out) {
    (void)h;
    double s = 0.0;
    for (int k = 0; k < K; ++k) {
        int sat = 1;
        for (int64_t j = lit_off[k]; j < lit_off[k + 1]; ++j) sat &= (x[lit_var[j]] == (uint8_t)(!lit_neg[j]));
        if (sat) s += w[k];
    }
    *out = s;
    return 0;
}

/* Linear-time values on a WDNF: drop unsatisfiable cubes, then per cube the
 * closed form.  phi has h entries. */
int orc_wdnf_values(int32_t h, int32_t K, const double *w, const int64_t *lit_off, const int32_t *lit_var,
                    const uint8_t *lit_neg, int32_t metric, double *phi) {
    for (int i = 0; i < h; ++i) phi[i] = 0.0;
    int32_t pos[64], neg[64], P[64], N[64];
    for (int k = 0; k < K; ++k) {
        int np = 0, nn = 0, a, b;
        if (lit_off[k + 1] - lit_off[k] > 64) return -1;
        for (int64_t j = lit_off[k]; j < lit_off[k + 1]; ++j) {
            if (lit_neg[j]) neg[nn++] = lit_var[j];
            else pos[np++] = lit_var[j];
        }
        if (!cube_sets(pos, np, neg, nn, P, &a, N, &b)) continue;
        cube_value(P, a, N, b, w[k], metric, phi);
    }
    return 0;
}

/* Exponential-time values on a WDNF: Eq. "PB_shap" (metric 0) or Eq. "PB_banzhaf"
 * (metric 1), enumerating every assignment of the other h-1 variables. */
int orc_wdnf_values_bruteforce(int32_t h, int32_t K, const double *w, const int64_t *lit_off,
                               const int32_t *lit_var, const uint8_t *lit_neg, int32_t metric, double *phi) {
    if (h > 24) return -1;
    uint8_t x[24];
    for (int i = 0; i < h; ++i) {
        double acc = 0.0;
        for (uint32_t a = 0; a < (1u << (h - 1)); ++a) {
            int ones = 0, bit = 0;
            for (int j = 0; j < h; ++j) {
                if (j == i) continue;
                x[j] = (uint8_t)((a >> bit) & 1u);
                ones += x[j];
                ++bit;
            }
            double f1, f0;
            x[i] = 1; orc_wdnf_eval(h, K, w, lit_off, lit_var, lit_neg, x, &f1);
            x[i] = 0; orc_wdnf_eval(h, K, w, lit_off, lit_var, lit_neg, x, &f0);
            double wt = metric == ORC_SHAPLEY ? 1.0 / ((double)h * (double)binom(h - 1, ones)) : 1.0 / ldexp(1.0, h - 1);
            acc += wt * (f1 - f0);
        }
        phi[i] = acc;
    }
    return 0;
}

/* The cube of one (consumer pattern, baseline pattern) pair on a path with the given
 * features (the four rules of section "Constructing a WDNF Representation", applied
 * root first; bit D-1-i of a pattern belongs to path position i), valued with unit
 * weight.  out is indexed by feature id (n_out entries).  Returns 1 when the cube is
 * satisfiable, 0 when it is bottom or unsatisfiable (out left at zero). */
int orc_path_cube(int32_t D, const int32_t *feats, uint64_t pc, uint64_t pb, int32_t metric,
                  double *out, int32_t n_out) {
    for (int i = 0; i < n_out; ++i) out[i] = 0.0;
    int32_t pos[ORC_MAXD], neg[ORC_MAXD], P[ORC_MAXD], N[ORC_MAXD];
    int np = 0, nn = 0, a, b;
    for (int i = 0; i < D; ++i) {
        int bc = (int)((pc >> (D - 1 - i)) & 1u), bb = (int)((pb >> (D - 1 - i)) & 1u);
        if (!bc && !bb) return 0;           /* rule 4: bottom */
        if (bc && !bb) pos[np++] = feats[i]; /* rule 1: f */
        if (!bc && bb) neg[nn++] = feats[i]; /* rule 2: not f */
    }                                       /* rule 3: (1,1) leaves the cube unchanged */
    if (!cube_sets(pos, np, neg, nn, P, &a, N, &b)) return 0;
    for (int i = 0; i < a; ++i) if (P[i] >= n_out) return -1;
    for (int i = 0; i < b; ++i) if (N[i] >= n_out) return -1;
    cube_value(P, a, N, b, 1.0, metric, out);
    return 1;
}

/* ---------------------------------------------------------------- O0: brute force */

/* v_c(S) for every coalition S of the F features, then Eq. "s" (metric 0) or the
 * Banzhaf sum (metric 1).  vempty[c] = v_c({}) = mean_b f(b). */
int orc_values_bruteforce(int32_t n_trees, const int64_t *off, const int32_t *feat, const float *thr,
                          const int32_t *left, const int32_t *right, const float *val, int32_t F,
                          const float *C, int64_t n, int64_t ldc, const float *B, int64_t m, int64_t ldb,
                          int32_t metric, double *phi, double *vempty) {
    if (F > 20 || F < 1 || m < 1) return -1;
    ens_t e = {n_trees, off, feat, thr, left, right, val};
    const uint32_t NS = 1u << F;
    int err = 0;
#pragma omp parallel
    {
        double *v = (double *)malloc(sizeof(double) * NS);
        float *x = (float *)malloc(sizeof(float) * (size_t)F);
        if (!v || !x) err = 1;
#pragma omp for schedule(dynamic)
        for (int64_t c = 0; c < n; ++c) {
            if (!v || !x) continue;
            const float *cr = C + c * ldc;
            for (uint32_t S = 0; S < NS; ++S) {
                double acc = 0.0;
                for (int64_t r = 0; r < m; ++r) {
                    const float *br = B + r * ldb;
                    for (int i = 0; i < F; ++i) x[i] = ((S >> i) & 1u) ? cr[i] : br[i];
                    acc += ens_value(&e, x);
                }
                v[S] = acc / (double)m;
            }
            for (int i = 0; i < F; ++i) {
                double acc = 0.0;
                for (uint32_t S = 0; S < NS; ++S) {
                    if ((S >> i) & 1u) continue;
                    int sz = __builtin_popcount(S);
                    double wt = metric == ORC_SHAPLEY ? 1.0 / ((double)F * (double)binom(F - 1, sz))
                                                      : 1.0 / ldexp(1.0, F - 1);
                    acc += wt * (v[S | (1u << i)] - v[S]);
                }
                phi[c * F + i] = acc;
            }
            vempty[c] = v[0];
        }
        free(v);
        free(x);
    }
    return err ? -1 : 0;
}

/* ---------------------------------------------------------------- O1: per pair */

typedef struct {
    const ens_t *e;
    const float *c, *b;
    int32_t pos[ORC_MAXD], neg[ORC_MAXD];
    int np, nn;
    double scale;
    int metric;
    double *phi;
} pair_walk_t;

/* Walk the tree along every branch that the consumer or the baseline takes; a branch
 * neither takes makes the cube bottom (rule 4) and is not entered. */
static void pair_rec(pair_walk_t *pw, int64_t o, int32_t node) {
    const ens_t *e = pw->e;
    int64_t g = o + node;
    if (e->feat[g] < 0) {
        int32_t P[ORC_MAXD], N[ORC_MAXD];
        int a, b;
        if (cube_sets(pw->pos, pw->np, pw->neg, pw->nn, P, &a, N, &b))
            cube_value(P, a, N, b, (double)e->val[g] * pw->scale, pw->metric, pw->phi);
        return;
    }
    int sc = split_true(pw->c, e->feat[g], e->thr[g]);
    int sb = split_true(pw->b, e->feat[g], e->thr[g]);
    for (int side = 0; side < 2; ++side) {
        int fc = side == 0 ? sc : !sc; /* consumer's pattern bit for this branch */
        int fb = side == 0 ? sb : !sb; /* baseline's pattern bit */
        if (!fc && !fb) continue;      /* rule 4 */
        if (fc && !fb) pw->pos[pw->np++] = e->feat[g]; /* rule 1 */
        if (!fc && fb) pw->neg[pw->nn++] = e->feat[g]; /* rule 2 */
        pair_rec(pw, o, side == 0 ? e->left[g] : e->right[g]);
        if (fc && !fb) pw->np--;
        if (!fc && fb) pw->nn--;
    }
}

/* Eq. "trival_bg": phi_i(c) = (1/m) sum_b sum_l w_l * value_i(d_l[P[l][c]][P[l][b]]).
 * base = mean_b f(b) = v_c({}). */
int orc_values_pairs(int32_t n_trees, const int64_t *off, const int32_t *feat, const float *thr,
                     const int32_t *left, const int32_t *right, const float *val, int32_t F,
                     const float *C, int64_t n, int64_t ldc, const float *B, int64_t m, int64_t ldb,
                     int32_t metric, double *phi, double *base) {
    if (m < 1) return -1;
    ens_t e = {n_trees, off, feat, thr, left, right, val};
    double fb = 0.0;
    for (int64_t r = 0; r < m; ++r) fb += ens_value(&e, B + r * ldb);
    *base = fb / (double)m;
#pragma omp parallel for schedule(dynamic)
    for (int64_t c = 0; c < n; ++c) {
        pair_walk_t pw;
        pw.e = &e; pw.c = C + c * ldc; pw.metric = metric; pw.phi = phi + c * F; pw.scale = 1.0 / (double)m;
        for (int i = 0; i < F; ++i) pw.phi[i] = 0.0;
        for (int64_t r = 0; r < m; ++r) {
            pw.b = B + r * ldb;
            for (int t = 0; t < n_trees; ++t) {
                pw.np = pw.nn = 0;
                pair_rec(&pw, off[t], 0);
            }
        }
    }
    return 0;
}

/* ---------------------------------------------------------------- O2: regrouped */

/* Algorithm 1 for one row and one tree: the decision pattern of every node, by a
 * breadth-first walk; a child's pattern is the parent's shifted left plus 1 when the
 * row would take that child. */
static void row_patterns(const ens_t *e, int t, const float *x, uint64_t *pat, int32_t *queue) {
    int64_t o = e->off[t];
    int head = 0, tail = 0;
    pat[0] = 0;
    queue[tail++] = 0;
    while (head < tail) {
        int32_t v = queue[head++];
        if (e->feat[o + v] < 0) continue;
        uint64_t s = (uint64_t)split_true(x, e->feat[o + v], e->thr[o + v]);
        int32_t l = e->left[o + v], r = e->right[o + v];
        pat[l] = (pat[v] << 1) + s;
        pat[r] = (pat[v] << 1) + (1u - s);
        queue[tail++] = l;
        queue[tail++] = r;
    }
}

int64_t orc_hist_size(int32_t n_trees, const int64_t *off, const int32_t *feat, const float *thr,
                      const int32_t *left, const int32_t *right, const float *val) {
    ens_t e = {n_trees, off, feat, thr, left, right, val};
    leafset_t ls;
    if (collect_leaves(&e, &ls)) { free_leaves(&ls); return -1; }
    int64_t hs = ls.hist_size;
    free_leaves(&ls);
    return hs;
}

/* vc[l][p_b] = |{b in B : P[l][b] = p_b}| for every leaf (Eq. "bg_shap_derivation"
 * step (d)); counts laid out per leaf in orc_leaf_table order, 2^depth bins each.
 * Threads take disjoint trees (so each writes only its own trees' counts) over blocks
 * of rows small enough to stay in cache while every tree reads them. */
int orc_bg_hist(int32_t n_trees, const int64_t *off, const int32_t *feat, const float *thr,
                const int32_t *left, const int32_t *right, const float *val,
                const float *B, int64_t m, int64_t ldb, uint64_t *counts) {
    ens_t e = {n_trees, off, feat, thr, left, right, val};
    leafset_t ls;
    if (collect_leaves(&e, &ls)) { free_leaves(&ls); return -1; }
    const int64_t hs = ls.hist_size;
    const int64_t rows_per_block = 2048;
    memset(counts, 0, sizeof(uint64_t) * (size_t)hs);
    int err = 0;
#pragma omp parallel
    {
        uint64_t *pat = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)ls.max_tree_nodes);
        int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)ls.max_tree_nodes);
        if (!pat || !queue) {
#pragma omp atomic write
            err = 1;
        }
        for (int64_t r0 = 0; r0 < m; r0 += rows_per_block) {
            const int64_t r1 = r0 + rows_per_block < m ? r0 + rows_per_block : m;
#pragma omp for schedule(static)
            for (int t = 0; t < n_trees; ++t) {
                if (!pat || !queue) continue;
                const int64_t o = off[t], sz = off[t + 1] - off[t];
                for (int64_t r = r0; r < r1; ++r) {
                    row_patterns(&e, t, B + r * ldb, pat, queue);
                    for (int64_t v = 0; v < sz; ++v) {
                        int32_t li = ls.leaf_of_node[o + v];
                        if (li >= 0) counts[ls.v[li].hoff + (int64_t)pat[v]] += 1;
                    }
                }
            }
        }
        free(pat);
        free(queue);
    }
    free_leaves(&ls);
    return err ? -1 : 0;
}

/* Eq. "bg_shap_derivation" step (d): for each consumer, leaf and counted background
 * pattern, the cube d_l[P[l][c]][p_b] weighted by w_l * vc[l][p_b] / m. */
int orc_values_hist(int32_t n_trees, const int64_t *off, const int32_t *feat, const float *thr,
                    const int32_t *left, const int32_t *right, const float *val, int32_t F,
                    const uint64_t *counts, int64_t m, const float *C, int64_t n, int64_t ldc,
                    int32_t metric, double *phi) {
    if (m < 1) return -1;
    ens_t e = {n_trees, off, feat, thr, left, right, val};
    leafset_t ls;
    if (collect_leaves(&e, &ls)) { free_leaves(&ls); return -1; }
    int err = 0;
#pragma omp parallel
    {
        uint64_t *pat = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)ls.max_tree_nodes);
        int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)ls.max_tree_nodes);
        if (!pat || !queue) err = 1;
#pragma omp for schedule(dynamic, 16)
        for (int64_t c = 0; c < n; ++c) {
            if (!pat || !queue) continue;
            const float *x = C + c * ldc;
            double *ph = phi + c * F;
            for (int i = 0; i < F; ++i) ph[i] = 0.0;
            int64_t li = 0;
            for (int t = 0; t < n_trees; ++t) {
                row_patterns(&e, t, x, pat, queue);
                for (; li < ls.n && ls.v[li].tree == t; ++li) {
                    const leaf_t *L = &ls.v[li];
                    const int D = L->depth;
                    const uint64_t full = D == 0 ? 0 : (((uint64_t)1 << D) - 1);
                    const uint64_t pc = pat[L->node];
                    int32_t pf[ORC_MAXD];
                    for (int i = 0; i < D; ++i) pf[i] = feat[off[t] + L->path[i]];
                    for (uint64_t pb = 0; pb <= full; ++pb) {
                        uint64_t cnt = counts[L->hoff + (int64_t)pb];
                        if (cnt == 0) continue;
                        if ((pc | pb) != full) continue; /* some bit is (0,0): rule 4 */
                        int32_t pos[ORC_MAXD], neg[ORC_MAXD], P[ORC_MAXD], N[ORC_MAXD];
                        int np = 0, nn = 0, a, b;
                        for (int i = 0; i < D; ++i) {
                            int bc = (int)((pc >> (D - 1 - i)) & 1u), bb = (int)((pb >> (D - 1 - i)) & 1u);
                            if (bc && !bb) pos[np++] = pf[i];
                            if (!bc && bb) neg[nn++] = pf[i];
                        }
                        if (!cube_sets(pos, np, neg, nn, P, &a, N, &b)) continue;
                        cube_value(P, a, N, b, L->w * (double)cnt / (double)m, metric, ph);
                    }
                }
            }
        }
        free(pat);
        free(queue);
    }
    free_leaves(&ls);
    return err ? -1 : 0;
}

/* E_b f(b) from the counts: a background row reaches leaf l exactly when its pattern
 * there is all ones. */
int orc_base_from_hist(int32_t n_trees, const int64_t *off, const int32_t *feat, const float *thr,
                       const int32_t *left, const int32_t *right, const float *val,
                       const uint64_t *counts, int64_t m, double *out) {
    ens_t e = {n_trees, off, feat, thr, left, right, val};
    leafset_t ls;
    if (collect_leaves(&e, &ls)) { free_leaves(&ls); return -1; }
    double s = 0.0;
    for (int64_t i = 0; i < ls.n; ++i) {
        int64_t full = ((int64_t)1 << ls.v[i].depth) - 1;
        s += ls.v[i].w * (double)counts[ls.v[i].hoff + full];
    }
    *out = s / (double)m;
    free_leaves(&ls);
    return 0;
}

/* ---------------------------------------------------------------- path-dependent */

/* The path-dependent game (section "Feature Importance Using Shapley Values": the cover
 * of a node, the number of training rows that reached it, stands in for the missing
 * features): v_c(S) = sum over trees of E(root), where E(leaf) = w_leaf and at an inner
 * node splitting on feature i, E = E(child c follows) when i is in S, else
 * cover(left)/cover(node) * E(left) + cover(right)/cover(node) * E(right) (a node of
 * zero cover contributes 0). */
static double pd_expect(const ens_t *e, const double *cover, int64_t o, int32_t node, const float *x, uint32_t S) {
    int64_t g = o + node;
    if (e->feat[g] < 0) return (double)e->val[g];
    int32_t f = e->feat[g];
    if ((S >> f) & 1u) {
        int32_t nx = split_true(x, f, e->thr[g]) ? e->left[g] : e->right[g];
        return pd_expect(e, cover, o, nx, x, S);
    }
    double cn = cover[g];
    if (cn <= 0.0) return 0.0;
    int32_t l = e->left[g], r = e->right[g];
    return (cover[o + l] / cn) * pd_expect(e, cover, o, l, x, S) + (cover[o + r] / cn) * pd_expect(e, cover, o, r, x, S);
}

/* O0 for the path-dependent game: v_c(S) for all 2^F coalitions, then Eq. "s" (or the
 * Banzhaf sum).  vempty[c] = v_c({}). */
int orc_pd_values_bruteforce(int32_t n_trees, const int64_t *off, const int32_t *feat, const float *thr,
                             const int32_t *left, const int32_t *right, const float *val, const double *cover,
                             int32_t F, const float *C, int64_t n, int64_t ldc, int32_t metric, double *phi,
                             double *vempty) {
    if (F > 20 || F < 1) return -1;
    ens_t e = {n_trees, off, feat, thr, left, right, val};
    const uint32_t NS = 1u << F;
    int err = 0;
#pragma omp parallel
    {
        double *v = (double *)malloc(sizeof(double) * NS);
        if (!v) err = 1;
#pragma omp for schedule(dynamic)
        for (int64_t c = 0; c < n; ++c) {
            if (!v) continue;
            const float *x = C + c * ldc;
            for (uint32_t S = 0; S < NS; ++S) {
                double acc = 0.0;
                for (int t = 0; t < n_trees; ++t) acc += pd_expect(&e, cover, off[t], 0, x, S);
                v[S] = acc;
            }
            for (int i = 0; i < F; ++i) {
                double acc = 0.0;
                for (uint32_t S = 0; S < NS; ++S) {
                    if ((S >> i) & 1u) continue;
                    int sz = __builtin_popcount(S);
                    double wt = metric == ORC_SHAPLEY ? 1.0 / ((double)F * (double)binom(F - 1, sz))
                                                      : 1.0 / ldexp(1.0, F - 1);
                    acc += wt * (v[S | (1u << i)] - v[S]);
                }
                phi[c * F + i] = acc;
            }
            vempty[c] = v[0];
        }
        free(v);
    }
    return err ? -1 : 0;
}

/* Eq. "path_dependent_estimation": for the leaf with index `leaf` (orc_leaf_table order)
 * the frequency of every baseline pattern p_b, the product over the path nodes of the
 * cover ratio r_i = cover(n_{i+1}) / cover(n_i) where bit i of p_b is 1 and of 1 - r_i
 * where it is 0 (root first, bit D-1-i).  out has 2^depth entries. */
static void pd_freq_leaf(const ens_t *e, const double *cover, const leaf_t *L, double *out) {
    const int D = L->depth;
    const int64_t o = e->off[L->tree];
    double r[ORC_MAXD];
    for (int i = 0; i < D; ++i) {
        int32_t nd = L->path[i];
        int32_t nx = (i + 1 < D) ? L->path[i + 1] : L->node;
        double cn = cover[o + nd];
        r[i] = cn > 0.0 ? cover[o + nx] / cn : 0.0;
    }
    for (uint64_t p = 0; p < ((uint64_t)1 << D); ++p) {
        double f = 1.0;
        for (int i = 0; i < D; ++i) f *= ((p >> (D - 1 - i)) & 1u) ? r[i] : 1.0 - r[i];
        out[p] = f;
    }
}

int orc_pd_freq(int32_t n_trees, const int64_t *off, const int32_t *feat, const float *thr, const int32_t *left,
                const int32_t *right, const float *val, const double *cover, double *out) {
    ens_t e = {n_trees, off, feat, thr, left, right, val};
    leafset_t ls;
    if (collect_leaves(&e, &ls)) { free_leaves(&ls); return -1; }
    for (int64_t i = 0; i < ls.n; ++i) pd_freq_leaf(&e, cover, &ls.v[i], out + ls.v[i].hoff);
    free_leaves(&ls);
    return 0;
}

/* O2 for the path-dependent game: as orc_values_hist with the background frequencies
 * vc / m replaced by the path-dependent frequencies (section "Efficient Path-Dependent
 * SHAP Equation").  base = sum_l w_l * f_pd[l][all ones] = v_c({}). */
int orc_pd_values(int32_t n_trees, const int64_t *off, const int32_t *feat, const float *thr, const int32_t *left,
                  const int32_t *right, const float *val, const double *cover, int32_t F, const float *C, int64_t n,
                  int64_t ldc, int32_t metric, double *phi, double *base) {
    ens_t e = {n_trees, off, feat, thr, left, right, val};
    leafset_t ls;
    if (collect_leaves(&e, &ls)) { free_leaves(&ls); return -1; }
    double *freq = (double *)malloc(sizeof(double) * (size_t)(ls.hist_size > 0 ? ls.hist_size : 1));
    if (!freq) { free_leaves(&ls); return -1; }
    double b = 0.0;
    for (int64_t i = 0; i < ls.n; ++i) {
        pd_freq_leaf(&e, cover, &ls.v[i], freq + ls.v[i].hoff);
        b += ls.v[i].w * freq[ls.v[i].hoff + ((int64_t)1 << ls.v[i].depth) - 1];
    }
    *base = b;
    int err = 0;
#pragma omp parallel
    {
        uint64_t *pat = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)ls.max_tree_nodes);
        int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)ls.max_tree_nodes);
        if (!pat || !queue) err = 1;
#pragma omp for schedule(dynamic, 16)
        for (int64_t c = 0; c < n; ++c) {
            if (!pat || !queue) continue;
            const float *x = C + c * ldc;
            double *ph = phi + c * F;
            for (int i = 0; i < F; ++i) ph[i] = 0.0;
            int64_t li = 0;
            for (int t = 0; t < n_trees; ++t) {
                row_patterns(&e, t, x, pat, queue);
                for (; li < ls.n && ls.v[li].tree == t; ++li) {
                    const leaf_t *L = &ls.v[li];
                    const int D = L->depth;
                    const uint64_t full = D == 0 ? 0 : (((uint64_t)1 << D) - 1);
                    const uint64_t pc = pat[L->node];
                    int32_t pf[ORC_MAXD];
                    for (int i = 0; i < D; ++i) pf[i] = feat[off[t] + L->path[i]];
                    for (uint64_t pb = 0; pb <= full; ++pb) {
                        double fr = freq[L->hoff + (int64_t)pb];
                        if (fr == 0.0) continue;
                        if ((pc | pb) != full) continue; /* rule 4 */
                        int32_t pos[ORC_MAXD], neg[ORC_MAXD], P[ORC_MAXD], N[ORC_MAXD];
                        int np = 0, nn = 0, a, bb;
                        for (int i = 0; i < D; ++i) {
                            int bc = (int)((pc >> (D - 1 - i)) & 1u), bv = (int)((pb >> (D - 1 - i)) & 1u);
                            if (bc && !bv) pos[np++] = pf[i];
                            if (!bc && bv) neg[nn++] = pf[i];
                        }
                        if (!cube_sets(pos, np, neg, nn, P, &a, N, &bb)) continue;
                        cube_value(P, a, N, bb, L->w * fr, metric, ph);
                    }
                }
            }
        }
        free(pat);
        free(queue);
    }
    free(freq);
    free_leaves(&ls);
    return err ? -1 : 0;
}

/* ---------------------------------------------------------------- interaction values */

/* One satisfiable weighted cube with distinct sets P (a variables) and N (b): for every
 * ordered pair of its variables i != j, Table "table_shap_iv" (metric 0, cells indexed
 * by where i and j sit) or Formula "banzhaf_simplified_formula_interactions" (metric
 * 1, +-w / 2^(|S|-2)), added to out[i * h + j].  Pairs with a variable outside the
 * cube get 0; the diagonal is not touched. */
static void cube_iv(const int32_t *P, int a, const int32_t *N, int b, double w, int metric, int32_t h, double *out) {
    const int s = a + b;
    if (s < 2) return;
    double pp, nn, pn, np_;  /* (i in P, j in P), (N, N), (i in P, j in N), (i in N, j in P) */
    if (metric == ORC_SHAPLEY) {
        pp = a >= 2 ? w / ((double)(a - 1) * (double)binom(s - 1, a - 1)) : 0.0;
        nn = b >= 2 ? w / ((double)(b - 1) * (double)binom(s - 1, b - 1)) : 0.0;
        pn = b >= 1 ? -w / ((double)b * (double)binom(s - 1, b)) : 0.0;
        np_ = a >= 1 ? -w / ((double)a * (double)binom(s - 1, a)) : 0.0;
    } else {
        const double v = w / ldexp(1.0, s - 2);
        pp = nn = v;
        pn = np_ = -v;
    }
    for (int x = 0; x < a; ++x)
        for (int y = 0; y < a; ++y)
            if (x != y) out[(int64_t)P[x] * h + P[y]] += pp;
    for (int x = 0; x < b; ++x)
        for (int y = 0; y < b; ++y)
            if (x != y) out[(int64_t)N[x] * h + N[y]] += nn;
    for (int x = 0; x < a; ++x)
        for (int y = 0; y < b; ++y) {
            out[(int64_t)P[x] * h + N[y]] += pn;
            out[(int64_t)N[y] * h + P[x]] += np_;
        }
}

/* Interaction values of a WDNF by the per-cube closed forms (out is h x h). */
int orc_wdnf_iv(int32_t h, int32_t K, const double *w, const int64_t *lit_off, const int32_t *lit_var,
                const uint8_t *lit_neg, int32_t metric, double *out) {
    for (int64_t i = 0; i < (int64_t)h * h; ++i) out[i] = 0.0;
    int32_t pos[64], neg[64], P[64], N[64];
    for (int k = 0; k < K; ++k) {
        int np = 0, nn = 0, a, b;
        if (lit_off[k + 1] - lit_off[k] > 64) return -1;
        for (int64_t j = lit_off[k]; j < lit_off[k + 1]; ++j) {
            if (lit_neg[j]) neg[nn++] = lit_var[j];
            else pos[np++] = lit_var[j];
        }
        if (!cube_sets(pos, np, neg, nn, P, &a, N, &b)) continue;
        cube_iv(P, a, N, b, w[k], metric, h, out);
    }
    return 0;
}

/* The pair weight of a coalition of s other players out of h - 2: Def. "shap_iv_def"
 * is the Shapley value of j in the (h-1)-player game with i held in or out, whose
 * weight is 1 / ((h-1) C(h-2, s)); Def. "banzhaf_iv_def" takes the uniform average. */
static double pair_weight(int h, int s, int metric) {
    return metric == ORC_SHAPLEY ? 1.0 / ((double)(h - 1) * (double)binom(h - 2, s)) : 1.0 / ldexp(1.0, h - 2);
}

/* Interaction values of a WDNF by the definitions, enumerating the other h-2
 * variables: sum of weight * (f(i,j) - f(i) - f(j) + f()) over their assignments. */
int orc_wdnf_iv_bruteforce(int32_t h, int32_t K, const double *w, const int64_t *lit_off, const int32_t *lit_var,
                           const uint8_t *lit_neg, int32_t metric, double *out) {
    if (h > 22 || h < 2) return -1;
    uint8_t x[24];
    for (int i = 0; i < h; ++i)
        for (int j = 0; j < h; ++j) {
            out[(int64_t)i * h + j] = 0.0;
            if (i == j) continue;
            double acc = 0.0;
            for (uint32_t asg = 0; asg < (1u << (h - 2)); ++asg) {
                int ones = 0, bit = 0;
                for (int k = 0; k < h; ++k) {
                    if (k == i || k == j) continue;
                    x[k] = (uint8_t)((asg >> bit) & 1u);
                    ones += x[k];
                    ++bit;
                }
                double f11, f10, f01, f00;
                x[i] = 1; x[j] = 1; orc_wdnf_eval(h, K, w, lit_off, lit_var, lit_neg, x, &f11);
                x[i] = 1; x[j] = 0; orc_wdnf_eval(h, K, w, lit_off, lit_var, lit_neg, x, &f10);
                x[i] = 0; x[j] = 1; orc_wdnf_eval(h, K, w, lit_off, lit_var, lit_neg, x, &f01);
                x[i] = 0; x[j] = 0; orc_wdnf_eval(h, K, w, lit_off, lit_var, lit_neg, x, &f00);
                acc += pair_weight(h, ones, metric) * (f11 - f10 - f01 + f00);
            }
            out[(int64_t)i * h + j] = acc;
        }
    return 0;
}

/* Def. "shap_iv_def" / "banzhaf_iv_def" on the background game, written out: v_c(S) for
 * every coalition of the F features, then for every ordered pair i != j the weighted
 * sum over coalitions S of the other features of v(S+i+j) - v(S+i) - v(S+j) + v(S).
 * out is n x F x F (diagonal 0).  Tiny F only. */
int orc_iv_bruteforce(int32_t n_trees, const int64_t *off, const int32_t *feat, const float *thr,
                      const int32_t *left, const int32_t *right, const float *val, int32_t F,
                      const float *C, int64_t n, int64_t ldc, const float *B, int64_t m, int64_t ldb,
                      int32_t metric, double *out) {
    if (F > 16 || F < 2 || m < 1) return -1;
    ens_t e = {n_trees, off, feat, thr, left, right, val};
    const uint32_t NS = 1u << F;
    int err = 0;
#pragma omp parallel
    {
        double *v = (double *)malloc(sizeof(double) * NS);
        float *x = (float *)malloc(sizeof(float) * (size_t)F);
        if (!v || !x) err = 1;
#pragma omp for schedule(dynamic)
        for (int64_t c = 0; c < n; ++c) {
            if (!v || !x) continue;
            const float *cr = C + c * ldc;
            for (uint32_t S = 0; S < NS; ++S) {
                double acc = 0.0;
                for (int64_t r = 0; r < m; ++r) {
                    const float *br = B + r * ldb;
                    for (int i = 0; i < F; ++i) x[i] = ((S >> i) & 1u) ? cr[i] : br[i];
                    acc += ens_value(&e, x);
                }
                v[S] = acc / (double)m;
            }
            double *o = out + c * F * F;
            for (int i = 0; i < F; ++i)
                for (int j = 0; j < F; ++j) {
                    double acc = 0.0;
                    if (i != j) {
                        const uint32_t bi = 1u << i, bj = 1u << j;
                        for (uint32_t S = 0; S < NS; ++S) {
                            if (S & (bi | bj)) continue;
                            acc += pair_weight(F, __builtin_popcount(S), metric) *
                                   (v[S | bi | bj] - v[S | bi] - v[S | bj] + v[S]);
                        }
                    }
                    o[i * F + j] = acc;
                }
        }
        free(v);
        free(x);
    }
    return err ? -1 : 0;
}

/* Interaction values from per-leaf baseline-pattern weights: as orc_values_hist, each
 * (consumer pattern, weighted baseline pattern) cube weighted by w_l times the bin's
 * weight -- vc[l][p_b] / m from exact background counts (counts non-null), or the
 * path-dependent frequency f_pd[l][p_b] (freq) -- valued by Table "table_shap_iv" (or
 * the Banzhaf pair formula).  out is n x F x F. */
static int iv_from_weights(const ens_t *ep, int32_t F, const uint64_t *counts, int64_t m, const double *freq,
                           const float *C, int64_t n, int64_t ldc, int32_t metric, double *out) {
    const ens_t e = *ep;
    const int64_t *off = e.off;
    const int32_t *feat = e.feat;
    const int32_t n_trees = e.n_trees;
    leafset_t ls;
    if (collect_leaves(&e, &ls)) { free_leaves(&ls); return -1; }
    int err = 0;
#pragma omp parallel
    {
        uint64_t *pat = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)ls.max_tree_nodes);
        int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)ls.max_tree_nodes);
        if (!pat || !queue) err = 1;
#pragma omp for schedule(dynamic, 4)
        for (int64_t c = 0; c < n; ++c) {
            if (!pat || !queue) continue;
            const float *x = C + c * ldc;
            double *o = out + c * F * F;
            for (int64_t i = 0; i < (int64_t)F * F; ++i) o[i] = 0.0;
            int64_t li = 0;
            for (int t = 0; t < n_trees; ++t) {
                row_patterns(&e, t, x, pat, queue);
                for (; li < ls.n && ls.v[li].tree == t; ++li) {
                    const leaf_t *L = &ls.v[li];
                    const int D = L->depth;
                    const uint64_t full = D == 0 ? 0 : (((uint64_t)1 << D) - 1);
                    const uint64_t pc = pat[L->node];
                    int32_t pf[ORC_MAXD];
                    for (int i = 0; i < D; ++i) pf[i] = feat[off[t] + L->path[i]];
                    for (uint64_t pb = 0; pb <= full; ++pb) {
                        const double wt = counts ? (double)counts[L->hoff + (int64_t)pb] / (double)m
                                                 : freq[L->hoff + (int64_t)pb];
                        if (wt == 0.0) continue;
                        if ((pc | pb) != full) continue; /* rule 4 */
                        int32_t pos[ORC_MAXD], neg[ORC_MAXD], P[ORC_MAXD], N[ORC_MAXD];
                        int np = 0, nn = 0, a, b;
                        for (int i = 0; i < D; ++i) {
                            int bc = (int)((pc >> (D - 1 - i)) & 1u), bb = (int)((pb >> (D - 1 - i)) & 1u);
                            if (bc && !bb) pos[np++] = pf[i];
                            if (!bc && bb) neg[nn++] = pf[i];
                        }
                        if (!cube_sets(pos, np, neg, nn, P, &a, N, &b)) continue;
                        cube_iv(P, a, N, b, L->w * wt, metric, F, o);
                    }
                }
            }
        }
        free(pat);
        free(queue);
    }
    free_leaves(&ls);
    return err ? -1 : 0;
}

int orc_iv_hist(int32_t n_trees, const int64_t *off, const int32_t *feat, const float *thr,
                const int32_t *left, const int32_t *right, const float *val, int32_t F,
                const uint64_t *counts, int64_t m, const float *C, int64_t n, int64_t ldc,
                int32_t metric, double *out) {
    if (m < 1) return -1;
    ens_t e = {n_trees, off, feat, thr, left, right, val};
    return iv_from_weights(&e, F, counts, m, NULL, C, n, ldc, metric, out);
}

/* Path-dependent interaction values: the frequency form (Eq.
 * "path_dependent_estimation") in place of the counts. */
int orc_pd_iv(int32_t n_trees, const int64_t *off, const int32_t *feat, const float *thr, const int32_t *left,
              const int32_t *right, const float *val, const double *cover, int32_t F, const float *C, int64_t n,
              int64_t ldc, int32_t metric, double *out) {
    ens_t e = {n_trees, off, feat, thr, left, right, val};
    leafset_t ls;
    if (collect_leaves(&e, &ls)) { free_leaves(&ls); return -1; }
    double *freq = (double *)calloc((size_t)(ls.hist_size > 0 ? ls.hist_size : 1), sizeof(double));
    if (!freq) { free_leaves(&ls); return -1; }
    for (int64_t i = 0; i < ls.n; ++i) pd_freq_leaf(&e, cover, &ls.v[i], freq + ls.v[i].hoff);
    free_leaves(&ls);
    int rc = iv_from_weights(&e, F, NULL, 0, freq, C, n, ldc, metric, out);
    free(freq);
    return rc;
}

/* Path-dependent interaction values by the definitions: v_c(S) from the cover-weighted
 * expectation walk for all coalitions, then the pair sums of orc_iv_bruteforce. */
int orc_pd_iv_bruteforce(int32_t n_trees, const int64_t *off, const int32_t *feat, const float *thr,
                         const int32_t *left, const int32_t *right, const float *val, const double *cover,
                         int32_t F, const float *C, int64_t n, int64_t ldc, int32_t metric, double *out) {
    if (F > 16 || F < 2) return -1;
    ens_t e = {n_trees, off, feat, thr, left, right, val};
    const uint32_t NS = 1u << F;
    int err = 0;
#pragma omp parallel
    {
        double *v = (double *)malloc(sizeof(double) * NS);
        if (!v) err = 1;
#pragma omp for schedule(dynamic)
        for (int64_t c = 0; c < n; ++c) {
            if (!v) continue;
            const float *x = C + c * ldc;
            for (uint32_t S = 0; S < NS; ++S) {
                double acc = 0.0;
                for (int t = 0; t < n_trees; ++t) acc += pd_expect(&e, cover, off[t], 0, x, S);
                v[S] = acc;
            }
            double *o = out + c * F * F;
            for (int i = 0; i < F; ++i)
                for (int j = 0; j < F; ++j) {
                    double acc = 0.0;
                    if (i != j) {
                        const uint32_t bi = 1u << i, bj = 1u << j;
                        for (uint32_t S = 0; S < NS; ++S) {
                            if (S & (bi | bj)) continue;
                            acc += pair_weight(F, __builtin_popcount(S), metric) *
                                   (v[S | bi | bj] - v[S | bi] - v[S | bj] + v[S]);
                        }
                    }
                    o[i * F + j] = acc;
                }
        }
        free(v);
    }
    return err ? -1 : 0;
}
