// Host-side validation and complete-layout packing of a tree ensemble.
//
// Input format: Def. "decision_tree" (binary inner nodes with feature and threshold,
// leaves with outputs).  The complete layout and why it changes no value are
// described in wdf_internal.h.  Leaves are grouped by the path signature of section
// "Algorithmic Improvements" item 2 (the pattern-pair matrices depend only on the
// path length and on which features repeat along the path), so each group shares one
// pattern-pair table.
#include <algorithm>
#include <cstring>
#include <limits>
#include <map>

#include "tree_layout.h"
#include "wdf_internal.h"

namespace wdf {

namespace {

struct Src {
    int F;
    const int64_t *off;
    const int32_t *feat;
    const float *thr;
    const int32_t *left, *right;
    const float *val;
};

// Writes the subtree of input node `node` (local to tree t) at heap position h of
// depth `depth`; pass-through when node < 0 ("send left") and `keep` says whether the
// leftmost leaf below keeps output w.  csrc: the input node whose cover a pass-through
// position carries (the pushed-down leaf on the kept path, -1 elsewhere).
void place(const Src &s, int t, int32_t node, int h, int depth, float w, bool keep, Packed *p, int32_t csrc) {
    const int D = p->D;
    p->heap_src[(size_t)t * (p->NI + p->NL) + h] = (node >= 0) ? node : csrc;
    if (depth == D) {
        const int q = h - p->NI;
        p->leaf_w[(size_t)t * p->NL + q] = (node >= 0) ? s.val[s.off[t] + node] : (keep ? w : 0.0f);
        return;
    }
    const size_t k = (size_t)t * p->NI + h;
    if (node >= 0 && s.feat[s.off[t] + node] >= 0) {
        const int64_t g = s.off[t] + node;
        p->node_feat[k] = s.feat[g];
        p->node_thr[k] = s.thr[g];
        place(s, t, s.left[g], 2 * h + 1, depth + 1, 0.0f, false, p, -1);
        place(s, t, s.right[g], 2 * h + 2, depth + 1, 0.0f, false, p, -1);
        return;
    }
    // an input leaf above depth D, or a node under a pass-through: route every row left
    float wl = w;
    bool kl = keep;
    int32_t cl = csrc;
    if (node >= 0) {  // input leaf: its output (and cover) move to the leftmost leaf below
        wl = s.val[s.off[t] + node];
        kl = true;
        cl = node;
    }
    p->node_feat[k] = p->F;  // virtual column, always 0
    p->node_thr[k] = 1.0f;   // 0 < 1: left
    place(s, t, -1, 2 * h + 1, depth + 1, wl, kl, p, cl);
    place(s, t, -1, 2 * h + 2, depth + 1, 0.0f, false, p, -1);
}

// Code columns, node records and tree metadata of the decision kernels (tree_layout.h).
void build_records(Packed *pp) {
    Packed &p = *pp;
    const int F = p.F, T = p.T, D = p.D, NI = p.NI;
    // distinct thresholds of every feature, sorted (NaN thresholds send every row right
    // and take no part in the codes)
    std::vector<std::vector<float>> thr(F);
    for (size_t k = 0; k < p.node_feat.size(); ++k) {
        const int f = p.node_feat[k];
        if (f < F && p.node_thr[k] == p.node_thr[k]) thr[(size_t)f].push_back(p.node_thr[k]);
    }
    int64_t cols8 = 0, cols16 = 0;
    for (auto &v : thr) {
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end(), [](float a, float b) { return a == b; }), v.end());
        cols8 += ((int64_t)v.size() + 254) / 255;
        cols16 += ((int64_t)v.size() + 65534) / 65535;
    }
    // one-byte codes unless they would take more shared memory than two-byte codes
    p.code_bytes = cols8 <= 2 * cols16 ? 1 : 2;
    const int cap = p.code_bytes == 1 ? 255 : 65535;
    std::vector<int32_t> first_col((size_t)F, -1);
    p.cols.clear();
    p.col_thr.clear();
    for (int f = 0; f < F; ++f) {
        const auto &v = thr[(size_t)f];
        if (v.empty()) continue;
        first_col[(size_t)f] = (int32_t)p.cols.size();
        for (size_t lo = 0; lo < v.size(); lo += (size_t)cap) {
            const int cnt = (int)std::min(v.size() - lo, (size_t)cap);
            int top = 1;
            while (2 * top <= cnt) top *= 2;
            p.cols.push_back(CodeCol{f, (int32_t)p.col_thr.size(), cnt, top});
            p.col_thr.insert(p.col_thr.end(), v.begin() + (int64_t)lo, v.begin() + (int64_t)lo + cnt);
            // one-byte columns are padded to 255 entries with NaN (u <= x is false for a NaN
            // u), so the encoder can search them in 8 fixed steps without bound checks
            if (p.code_bytes == 1)
                p.col_thr.insert(p.col_thr.end(), (size_t)(255 - cnt), std::numeric_limits<float>::quiet_NaN());
        }
    }
    if (p.cols.empty()) {  // no real threshold at all: one empty column
        p.cols.push_back(CodeCol{0, 0, 0, 0});
        if (p.code_bytes == 1) p.col_thr.assign(255, std::numeric_limits<float>::quiet_NaN());
    }
    const int64_t blk = 32 * (int64_t)p.code_bytes;             // bytes of one column in a code block
    p.rec.assign((size_t)T * NI, NodeRec{0, -1, 0u, 0u});
    p.meta.assign((size_t)T, TreeMeta{});
    const int FL = flush_len(D);
    p.flush_feat.assign((size_t)T * FL, F);
    if (D <= 6) p.xmask.assign((size_t)T * 6, 0ull);
    for (int t = 0; t < T; ++t) {
        TreeMeta &m = p.meta[(size_t)t];
        int c = 0;
        for (int v = 0; v < NI; ++v) {  // heap order, so the nodes of word v/32 are contiguous
            const size_t k = (size_t)t * NI + v;
            const int f = p.node_feat[k];
            if (f == F) {
                m.pt[v >> 5] |= 1u << (v & 31);
            } else {
                NodeRec r{0, -1, (D >= 7 || v < 32) ? 1u << (v & 31) : 0u, (D <= 6 && v >= 32) ? 1u << (v - 32) : 0u};
                const float x = p.node_thr[k];
                if (x == x) {
                    const auto &u = thr[(size_t)f];
                    const int64_t j = std::lower_bound(u.begin(), u.end(), x) - u.begin();
                    r.col_off = (int32_t)((first_col[(size_t)f] + j / cap) * blk);
                    r.rank = (int32_t)(j % cap);
                }
                p.rec[(size_t)t * NI + c++] = r;
            }
            if ((v & 31) == 31 || v == NI - 1) m.wend[v >> 5] = (uint8_t)c;
        }
        for (int w = (NI - 1) / 32 + 1; w < 8; ++w) m.wend[w] = (uint8_t)c;
        m.live = p.live[(size_t)t];
        if (D <= 6) {  // the real (not pass-through) nodes, one bit per heap position
            const uint64_t all = NI == 64 ? ~0ull : ((1ull << NI) - 1ull);
            const uint64_t real = ~((uint64_t)m.pt[0] | ((uint64_t)m.pt[1] << 32)) & all;
            expand_masks(real, &p.xmask[(size_t)t * 6]);
        }
        for (int i = 0; i < FL; ++i) {
            const int v = flush_node(D, i);
            if (v >= 0) p.flush_feat[(size_t)t * FL + i] = p.node_feat[(size_t)t * NI + v];
        }
        // flush batches of the consumer kernel whose real features are all distinct
        for (int b = 0; b < flush_batches(D); ++b) {
            bool ok = true;
            for (int i = 8 * b; i < 8 * b + 8 && ok; ++i)
                for (int j = 8 * b; j < i && ok; ++j) {
                    const int vi = flush_node(D, i), vj = flush_node(D, j);
                    if (vi < 0 || vj < 0) continue;
                    const int32_t fi = p.node_feat[(size_t)t * NI + vi], fj = p.node_feat[(size_t)t * NI + vj];
                    ok = fi == F || fi != fj;  // pass-through nodes all write the scratch row
                }
            if (ok) m.flush |= 1ull << b;
            for (int i = 8 * b; i < 8 * b + 8; ++i) {
                const int v = flush_node(D, i);
                if (v >= 0 && p.node_feat[(size_t)t * NI + v] != F) m.real |= 1ull << b;
            }
        }
    }
}

}  // namespace

int pack_ensemble(int F, int T, const int64_t *off, const int32_t *feat, const float *thr, const int32_t *left,
                  const int32_t *right, const float *val, Packed *out, std::string *err) {
    if (F < 1 || T < 1 || !off || !feat || !thr || !left || !right || !val) {
        *err = "n_features and n_trees must be >= 1 and all arrays non-null";
        return 1;
    }
    if (off[0] != 0) {
        *err = "tree_offset[0] must be 0";
        return 1;
    }
    int max_depth = 0;
    std::vector<int> depth_of, seen;
    for (int t = 0; t < T; ++t) {
        const int64_t o = off[t], sz = off[t + 1] - off[t];
        if (sz < 1 || sz > (1 << 20)) {
            *err = "tree " + std::to_string(t) + ": node count must be in [1, 2^20]";
            return 1;
        }
        depth_of.assign((size_t)sz, -1);
        seen.assign((size_t)sz, 0);
        std::vector<int32_t> queue;
        queue.push_back(0);
        depth_of[0] = 0;
        seen[0] = 1;
        size_t head = 0;
        while (head < queue.size()) {
            const int32_t v = queue[head++];
            const int64_t g = o + v;
            if (feat[g] < 0) {
                max_depth = std::max(max_depth, depth_of[(size_t)v]);
                continue;
            }
            if (feat[g] >= F) {
                *err = "tree " + std::to_string(t) + " node " + std::to_string(v) + ": feature out of range";
                return 1;
            }
            for (int32_t c : {left[g], right[g]}) {
                if (c <= 0 || c >= sz) {
                    *err = "tree " + std::to_string(t) + " node " + std::to_string(v) + ": child index out of range";
                    return 1;
                }
                if (seen[(size_t)c]) {
                    *err = "tree " + std::to_string(t) + " node " + std::to_string(c) + ": reached twice";
                    return 1;
                }
                seen[(size_t)c] = 1;
                depth_of[(size_t)c] = depth_of[(size_t)v] + 1;
                if (depth_of[(size_t)c] > kMaxDepth) {
                    *err = "tree " + std::to_string(t) + ": depth above 8 is not supported";
                    return 4;
                }
                queue.push_back(c);
            }
        }
        if ((int64_t)queue.size() != sz) {
            *err = "tree " + std::to_string(t) + ": " + std::to_string(sz - (int64_t)queue.size()) +
                   " node(s) not reachable from the root";
            return 1;
        }
    }
    Packed &p = *out;
    p = Packed();
    p.F = F;
    p.T = T;
    p.D = std::max(kMinDepth, max_depth);
    p.NI = (1 << p.D) - 1;
    p.NL = 1 << p.D;
    p.NS = 1 << (p.D - 2);
    p.node_feat.assign((size_t)T * p.NI, 0);
    p.node_thr.assign((size_t)T * p.NI, 0.0f);
    p.leaf_w.assign((size_t)T * p.NL, 0.0f);
    p.live.assign((size_t)T, 0);
    p.leaf_row.assign((size_t)T * p.NL, -1);
    p.heap_src.assign((size_t)T * (p.NI + p.NL), -1);
    p.in_off.assign(off, off + T + 1);
    Src s{F, off, feat, thr, left, right, val};
    for (int t = 0; t < T; ++t) place(s, t, 0, 0, 0, 0.0f, false, &p, -1);

    // live bottom subtrees and signature groups of the live leaves
    std::map<uint32_t, std::vector<int32_t>> groups;
    const int D = p.D;
    for (int t = 0; t < T; ++t) {
        for (int q = 0; q < p.NL; ++q) {
            if (p.leaf_w[(size_t)t * p.NL + q] == 0.0f) continue;
            p.live[(size_t)t] |= (uint64_t)1 << (q >> 2);
            int32_t pf[kMaxDepth];
            uint32_t key = 0;
            for (int k = 0; k < D; ++k) {
                const int h = ((p.NL + q) >> (D - k)) - 1;  // heap index of the depth-k node on the path
                const int32_t f = p.node_feat[(size_t)t * p.NI + h];
                pf[k] = (f == F) ? -(k + 1) : f;  // pass-through positions never repeat
                int first = k;
                for (int j = 0; j < k; ++j)
                    if (pf[j] == pf[k]) { first = j; break; }
                key |= (uint32_t)first << (3 * k);
            }
            groups[key].push_back(t * p.NL + q);
        }
    }
    p.group_off.push_back(0);
    for (auto &kv : groups) {
        p.sig_key.push_back(kv.first);
        for (int32_t leaf : kv.second) {
            p.leaf_row[(size_t)leaf] = (int32_t)p.group_leaf.size();
            p.group_leaf.push_back(leaf);
        }
        p.group_off.push_back((int32_t)p.group_leaf.size());
    }
    build_records(&p);
    return 0;
}

int pd_ratios(const Packed &p, const double *cover, std::vector<double> *ratio, std::string *err) {
    if (!cover) {
        *err = "cover is null";
        return 1;
    }
    const int64_t total = p.in_off[(size_t)p.T];
    for (int64_t i = 0; i < total; ++i)
        if (!(cover[i] >= 0.0) || cover[i] > 1e300) {
            *err = "covers must be finite and non-negative (node " + std::to_string(i) + ")";
            return 1;
        }
    const int D = p.D;
    ratio->assign(p.group_leaf.size() * (size_t)D, 0.0);
    for (size_t row = 0; row < p.group_leaf.size(); ++row) {
        const int leaf = p.group_leaf[row];
        const int t = leaf / p.NL, q = leaf % p.NL;
        auto cov = [&](int h) {
            const int32_t src = p.heap_src[(size_t)t * (p.NI + p.NL) + h];
            return src >= 0 ? cover[p.in_off[(size_t)t] + src] : 0.0;
        };
        for (int k = 0; k < D; ++k) {
            const int h = ((p.NL + q) >> (D - k)) - 1;          // path node at depth k
            const int hn = ((p.NL + q) >> (D - k - 1)) - 1;     // the next one on the path
            if (p.node_feat[(size_t)t * p.NI + h] == p.F) {      // pass-through: every row goes left
                (*ratio)[row * D + k] = 1.0;
                continue;
            }
            const double cn = cov(h);
            (*ratio)[row * D + k] = cn > 0.0 ? cov(hn) / cn : 0.0;
        }
    }
    return 0;
}

}  // namespace wdf
