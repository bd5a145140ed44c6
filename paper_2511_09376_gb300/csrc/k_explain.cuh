// Consumer side of Algorithm 3, step 4 (Eq. "bg_shap_derivation" step (g)):
// phi[c, i] = sum over trees and leaves of s_{l,i}[P[l][c]].
//
// One thread per consumer row.  The block stages its rows' decision codes in shared
// memory together with a per-row phi accumulator (feature-major), and the real inner
// nodes of a chunk of trees.  Per tree the thread evaluates those nodes (decision
// bitmask in registers), forms its entry at every bottom subtree, and gathers one slot
// vector per subtree from the folded table -- all gathers of a group of subtrees are
// issued before any is used, so their L2 latency overlaps; a dead subtree issues no load
// (its slots are zero).  The slots of the nodes above the bottom subtrees
// accumulate in registers (one per node, the node-level form of the NumPy indexing of
// section "Algorithmic Improvements" item 6); every node's value is then added into
// phi[feature of the node] in the fixed flush order of tree_layout.h, eight at a time:
// a batch that repeats no feature reads its eight phi values before writing any, so
// the shared-memory round trips overlap; any other batch adds one by one.  Pass-through
// nodes add into a scratch row.  The order of every floating-point addition into a
// row's phi depends only on the ensemble, never on which rows share a block.
//
// The kernels are templates of the depth; every depth is instantiated in its own
// translation unit so that they compile in parallel.
#pragma once
#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include "tree_layout.h"
#include "launch.h"
#include "wdf_device.cuh"

namespace wdf {

template <int D>
struct ExplainCfg {
    // trees per shared-memory chunk: two keeps the block small (five blocks of 64 rows
    // per SM at 127 features), measured faster than eight despite four times the barriers
    // (and than one or three, within 1 %); one for deep trees, whose node records would
    // otherwise cost a block per SM (depth 8: four instead of three 64-row blocks at 134
    // features; depth 7: 2 % faster)
    static constexpr int TCH = D >= 7 ? 1 : 2;
    // bottom subtrees gathered together (tree_layout.h); deep trees have several groups
    static constexpr int GS = gather_group(D);
    static constexpr int NG = Shape<D>::NS / GS;
    static_assert(Shape<D>::NS % GS == 0, "gather groups must tile the bottom subtrees");
    // the group loop is unrolled: rolled (group index in a register, its decision fields
    // and ancestor slots selected at run time) it had no instruction-cache misses at
    // depth 8 but more instructions; alone it measured within 2 %, in the server (beside
    // the other depths' kernels) its p99 was 10 % worse
    static constexpr int GUNROLL = NG;
    // phi offsets of the flush positions: 16 bits for deep trees (every offset is below
    // the 58,112 floats a block's shared memory can hold), 32 bits otherwise
    using Off = typename std::conditional<(D >= 7), uint16_t, int>::type;
    // node records staged as their first eight bytes (column offset, rank) with the
    // tree's expand masks, decisions collected in record order (tree_decisions8): up to
    // depth 6, where a tree's decisions fit one 64-bit word
    static constexpr bool R8 = D <= 6;
    using Rec = typename std::conditional<R8, int2, int4>::type;
};

// Shared memory of one block: code tile (TC rows x xb bytes) | phi tile ((F + 1) x (TC + 1)
// floats, feature-major, row F a scratch row) | tree metadata | expand masks (depth <= 6)
// | node records | phi offsets of the trees' nodes in flush order.
template <int D>
struct ExLayout {
    size_t x, p, meta, xm, rec, fl, total;
    static __host__ __device__ size_t up(size_t v) { return (v + 15) & ~(size_t)15; }
    __host__ __device__ ExLayout(int F, int xb, int TC) {
        using X = ExplainCfg<D>;
        x = up((size_t)TC * xb);
        p = up((size_t)(F + 1) * (TC + 1) * 4);
        meta = up((size_t)X::TCH * sizeof(TreeMeta));
        xm = X::R8 ? up((size_t)X::TCH * 6 * 8) : 0;
        rec = up((size_t)X::TCH * Shape<D>::NI * sizeof(typename X::Rec));
        fl = up((size_t)X::TCH * flush_len(D) * sizeof(typename X::Off));
        total = x + p + meta + xm + rec + fl;
    }
};

// 16-byte and 32-byte read-only loads predicated on `on` (the outputs keep their values
// when off): a dead bottom subtree issues no load, so it costs no L1 data-pipe wavefronts.
__device__ __forceinline__ void ldg_f4_if(const float4 *p, float4 &r, uint32_t on) {
    asm volatile(
        "{\n.reg .pred q;\nsetp.ne.u32 q, %5, 0;\n@q ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];\n}\n"
        : "+f"(r.x), "+f"(r.y), "+f"(r.z), "+f"(r.w)
        : "l"(p), "r"(on));
}

// One 32-byte entry in a single 256-bit load (the address is 32-byte aligned).
__device__ __forceinline__ void ldg_f8_if(const float4 *p, float4 &a, float4 &b, uint32_t on) {
    asm volatile(
        "{\n.reg .pred q;\nsetp.ne.u32 q, %9, 0;\n@q ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n}\n"
        : "+f"(a.x), "+f"(a.y), "+f"(a.z), "+f"(a.w), "+f"(b.x), "+f"(b.y), "+f"(b.z), "+f"(b.w)
        : "l"(p), "r"(on));
}

// phi[o[q]] += val[q], q < cnt, one after another: the rare batch that repeats a
// feature.  Kept out of line so the per-tree loop stays small in the instruction cache.
static __device__ __noinline__ void flush_serial(float *myphi, int4 oa, int4 ob, float4 va, float4 vb, int cnt) {
    const int o[8] = {oa.x, oa.y, oa.z, oa.w, ob.x, ob.y, ob.z, ob.w};
    const float v[8] = {va.x, va.y, va.z, va.w, vb.x, vb.y, vb.z, vb.w};
    for (int q = 0; q < cnt; ++q) myphi[o[q]] += v[q];
}

// phi[o[q]] += val[q] for the first cnt positions of one flush batch.  fast: the batch
// repeats no real feature, so all reads may precede all writes.  Pass-through positions
// (the scratch row) are not skipped: a predicated-off shared access still takes an L1
// data-pipe wavefront (ncu), so a test per position only added instructions.
__device__ __forceinline__ void flush_batch(float *myphi, const int (&o)[8], const float (&val)[8], int cnt,
                                            bool fast) {
    if (fast) {
        float a[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (q < cnt) a[q] = myphi[o[q]];
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (q < cnt) myphi[o[q]] = a[q] + val[q];
    } else {
        flush_serial(myphi, make_int4(o[0], o[1], o[2], o[3]), make_int4(o[4], o[5], o[6], o[7]),
                     make_float4(val[0], val[1], val[2], val[3]), make_float4(val[4], val[5], val[6], val[7]), cnt);
    }
}

__device__ __forceinline__ void load_offsets8(const int *p, int (&o)[8]) {
    const int4 a = *reinterpret_cast<const int4 *>(p), b = *reinterpret_cast<const int4 *>(p + 4);
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
    o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
}
__device__ __forceinline__ void load_offsets8(const uint16_t *p, int (&o)[8]) {
    const uint4 a = *reinterpret_cast<const uint4 *>(p);
    o[0] = (int)(a.x & 0xFFFFu); o[1] = (int)(a.x >> 16); o[2] = (int)(a.y & 0xFFFFu); o[3] = (int)(a.y >> 16);
    o[4] = (int)(a.z & 0xFFFFu); o[5] = (int)(a.z >> 16); o[6] = (int)(a.w & 0xFFFFu); o[7] = (int)(a.w >> 16);
}

// phi[offset of flush position i] += val[i] for the N positions that follow fl, in
// batches of eight (batch b0 first); the next batch's offsets are read before this
// batch's phi writes, so the offset loads stay off the chain of dependent shared-memory
// round trips.  A batch of pass-through nodes only is skipped (real), a batch that
// repeats no feature reads before it writes (fok).
template <int N, class Off, class Val>
__device__ __forceinline__ void flush_run(float *myphi, const Off *fl, const Val &value, uint64_t real, uint64_t fok,
                                          int b0) {
    int o[8];
    load_offsets8(fl, o);
#pragma unroll
    for (int i0 = 0; i0 < N; i0 += 8) {
        int on[8];
        if (i0 + 8 < N) load_offsets8(fl + i0 + 8, on);
        float vv[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) vv[q] = i0 + q < N ? value(i0 + q) : 0.0f;
        const int b = b0 + i0 / 8;
        if ((real >> b) & 1u) flush_batch(myphi, o, vv, N - i0 < 8 ? N - i0 : 8, (fok >> b) & 1u);
        if (i0 + 8 < N) {
#pragma unroll
            for (int q = 0; q < 8; ++q) o[q] = on[q];
        }
    }
}

// Slot k of a gathered slot vector held as Q float4 registers (k a compile-time constant
// after unrolling; a float pointer into the float4 array kept it in local memory).
template <int Q>
__device__ __forceinline__ float slot_of(const float4 (&vj)[Q], int k) {
    const float4 &x = vj[k >> 2];
    return (k & 3) == 0 ? x.x : (k & 3) == 1 ? x.y : (k & 3) == 2 ? x.z : x.w;
}

// Decision bits of tree level l (heap nodes 2^l - 1 .. 2^(l+1) - 2), aligned to the
// level's first node: word k holds nodes 2^l - 1 + 32k ... (levels of fewer than 32 nodes:
// one word, high bits beyond the level undefined).
template <int D, int l>
struct LevelBits {
    static constexpr int W = (1 << l) / 32 > 0 ? (1 << l) / 32 : 1;
    uint32_t w[W];
    __device__ __forceinline__ explicit LevelBits(const uint32_t (&dw)[Shape<D>::NW]) {
        constexpr int NW = Shape<D>::NW;
#pragma unroll
        for (int k = 0; k < W; ++k) {
            const int s = (1 << l) - 1 + 32 * k, a = s >> 5, sh = s & 31;
            const uint32_t hi = a + 1 < NW ? dw[a + 1 < NW ? a + 1 : 0] : 0u;
            w[k] = sh == 0 ? dw[a] : __funnelshift_r(dw[a], hi, sh);
        }
    }
    // the `width` bits of nodes g * width .. g * width + width - 1 of the level (width a
    // power of two <= 32, so a field never straddles two words)
    template <int width>
    __device__ __forceinline__ uint32_t field(int g) const {
        const uint32_t at = (uint32_t)g * width;
        uint32_t x = w[0];
#pragma unroll
        for (int k = 1; k < W; ++k) x = (at >> 5) == (uint32_t)k ? w[k] : x;
        if constexpr (width == 32) return x;
        else return (x >> (at & 31u)) & ((1u << width) - 1u);
    }
};

// One tile of TC consumer rows starting at row c0 (of n rows), for one ensemble.  The
// rows' decision codes are copied from codes, the code blocks of all n rows written by
// k_encode_codes or k_encode_batch (padded to a multiple of TC rows).  Encoding inside
// the tile measured 1.9 ms per 1M rows slower at the large workload: ten warps per SM
// cannot hide the dependent threshold loads of the searches, which the encode kernels
// run at full occupancy.
template <int D, int TC>
__device__ __forceinline__ void explain_tile(const ExplainJob &job, const unsigned char *__restrict__ codes,
                                             int64_t n, float *__restrict__ phi, int64_t ldp, int64_t c0,
                                             unsigned char *smem_raw) {
    using S = Shape<D>;
    using X = ExplainCfg<D>;
    constexpr int XS = TC + 1;
    constexpr int NA = S::NS > 1 ? S::NS - 1 : 1;
    constexpr int GS = X::GS;
    constexpr int Q = S::SP / 4;
    constexpr int FL = flush_len(D), FLB = flush_group_bottom(D);
    using Off = typename X::Off;
    const int F = job.F, T = job.T;
    const TreeArrays &ta = job.ta;
    const float *__restrict__ sfold = job.sfold;
    const int cb = ta.code_bytes, xb = ta.n_cols * cb;
    const ExLayout<D> L(F, xb, TC);
    unsigned char *sx = smem_raw;
    float *sp = reinterpret_cast<float *>(smem_raw + L.x);
    TreeMeta *smeta = reinterpret_cast<TreeMeta *>(smem_raw + L.x + L.p);
    using Rec = typename X::Rec;
    unsigned long long *sxm = reinterpret_cast<unsigned long long *>(smem_raw + L.x + L.p + L.meta);
    Rec *srec = reinterpret_cast<Rec *>(smem_raw + L.x + L.p + L.meta + L.xm);
    Off *sfl = reinterpret_cast<Off *>(smem_raw + L.x + L.p + L.meta + L.xm + L.rec);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(codes + c0 * xb);
        for (int i = tid; i < TC * xb / 16; i += TC) reinterpret_cast<uint4 *>(sx)[i] = __ldg(src + i);
    }
    for (int i = tid; i < (F + 1) * XS; i += TC) sp[i] = 0.0f;
    float *myphi = sp + tid;
    const CodeReader xr(sx + (size_t)warp * 32 * xb, lane, cb);
    // The next chunk's node records, metadata and flush features are loaded into
    // registers while this chunk's trees are processed, so staging a chunk costs only
    // shared-memory stores between two barriers (a block alone on its SM -- a small
    // request -- would otherwise wait for a global round trip per chunk).
    constexpr int MW = (int)(sizeof(TreeMeta) / sizeof(uint2));
    constexpr int RPT = (X::TCH * S::NI + TC - 1) / TC, MPT = (X::TCH * MW + TC - 1) / TC;
    constexpr int FPT = (X::TCH * FL + TC - 1) / TC, XPT = X::R8 ? (X::TCH * 6 + TC - 1) / TC : 0;
    Rec prec[RPT];
    uint2 pmeta[MPT];
    int pfl[FPT];
    unsigned long long pxm[XPT > 0 ? XPT : 1];
    auto fetch = [&](int t0) {
        const int n = min(X::TCH, T - t0);
        // a record's first eight bytes are its column offset and rank (NodeRec)
        const Rec *rsrc = reinterpret_cast<const Rec *>(ta.rec) + (size_t)t0 * S::NI * (X::R8 ? 2 : 1);
        const uint2 *msrc = reinterpret_cast<const uint2 *>(ta.meta + t0);
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            const int i = tid + r * TC;
            if (i < n * S::NI) prec[r] = __ldg(rsrc + (X::R8 ? 2 * i : i));
        }
#pragma unroll
        for (int k = 0; k < XPT; ++k) {
            const int i = tid + k * TC;
            if (i < n * 6) pxm[k] = __ldg(ta.xmask + (size_t)t0 * 6 + i);
        }
#pragma unroll
        for (int m = 0; m < MPT; ++m) {
            const int i = tid + m * TC;
            if (i < n * MW) pmeta[m] = __ldg(msrc + i);
        }
#pragma unroll
        for (int f = 0; f < FPT; ++f) {
            const int i = tid + f * TC;
            if (i < n * FL) pfl[f] = __ldg(job.flfeat + (size_t)t0 * FL + i);
        }
    };
    fetch(0);
    for (int tc0 = 0; tc0 < T; tc0 += X::TCH) {
        const int tcn = min(X::TCH, T - tc0);
        __syncthreads();
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            const int i = tid + r * TC;
            if (i < tcn * S::NI) srec[i] = prec[r];
        }
#pragma unroll
        for (int m = 0; m < MPT; ++m) {
            const int i = tid + m * TC;
            if (i < tcn * MW) reinterpret_cast<uint2 *>(smeta)[i] = pmeta[m];
        }
#pragma unroll
        for (int k = 0; k < XPT; ++k) {
            const int i = tid + k * TC;
            if (i < tcn * 6) sxm[i] = pxm[k];
        }
        // phi offsets of every tree in flush order (padding and pass-through nodes: the
        // scratch row F), from the features the host lists in flush order
#pragma unroll
        for (int f = 0; f < FPT; ++f) {
            const int i = tid + f * TC;
            if (i < tcn * FL) sfl[i] = (Off)(pfl[f] * XS);
        }
        __syncthreads();
        if (tc0 + X::TCH < T) fetch(tc0 + X::TCH);
        for (int g = 0; g < tcn; ++g) {
            const int t = tc0 + g;
            const TreeMeta &mt = smeta[g];
            const Off *fl = sfl + g * FL;
            uint32_t dw[S::NW];
            // one generic decision loop for both code widths (a second, one-byte copy in
            // this loop measured slower here, unlike in the counting kernel; node words
            // packed four to a 16-byte load measured slower too: the decoding cost more
            // issue slots than the shared-memory wavefronts it saved)
            if constexpr (X::R8)
                tree_decisions8<D, false>(srec + g * S::NI, mt.wend[S::NW - 1], mt.pt,
                                          reinterpret_cast<const uint64_t *>(sxm + g * 6), xr, dw);
            else
                tree_decisions<D, false>(srec + g * S::NI, mt, xr, dw);
            const uint64_t lv = mt.live;
            const float4 *tf = reinterpret_cast<const float4 *>(sfold + (size_t)t * S::NS * S::E * S::SP);
            constexpr int LW = lines_words(D);
            if constexpr (X::NG == 1) {
                const uint32_t fok = (uint32_t)mt.flush, real = (uint32_t)mt.real;
                uint32_t ent[S::NS];
                subtree_entries<D>(dw, ent);
                // the tree's line maps (launch.h), one byte per bottom subtree
                uint32_t lmap[LW];
#pragma unroll
                for (int w = 0; w < LW; w += 4) {
                    const uint4 v4 = __ldg(reinterpret_cast<const uint4 *>(job.lines + (size_t)t * LW) + w / 4);
                    lmap[w] = v4.x; lmap[w + 1] = v4.y; lmap[w + 2] = v4.z; lmap[w + 3] = v4.w;
                }
                float acc[NA];
#pragma unroll
                for (int a = 0; a < NA; ++a) acc[a] = 0.0f;
                constexpr int s0 = 0;
                if (lv) {  // else every subtree is dead (warp-uniform)
                    float4 v[GS][Q];
#pragma unroll
                    for (int j = 0; j < GS; ++j) {
                        const uint32_t lj = (uint32_t)(lv >> (s0 + j)) & 1u;
                        const uint32_t rot = (lmap[(s0 + j) >> 2] >> (8 * ((s0 + j) & 3))) & 0xFFu;
                        const float4 *src = tf + ((size_t)(s0 + j) * S::E + line_pos(ent[s0 + j], rot, D)) * Q;
#pragma unroll
                        for (int k = 0; k < Q; ++k) v[j][k] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                        if (Q == 2) {
                            ldg_f8_if(src, v[j][0], v[j][Q > 1 ? 1 : 0], lj);
                        } else {
#pragma unroll
                            for (int k = 0; k < Q; ++k) ldg_f4_if(src + k, v[j][k], lj);
                        }
                    }
#pragma unroll
                    for (int j = 0; j < GS; ++j) {
                        const int r = S::NS - 1 + s0 + j;
                        const float *vj = reinterpret_cast<const float *>(&v[j][0]);
#pragma unroll
                        for (int k = 0; k < D - 2; ++k) acc[((r + 1) >> (D - 2 - k)) - 1] += vj[k];
                    }
                    // the three inner nodes of each subtree, in flush order; the next
                    // batch's phi offsets are read before this batch's phi writes, so the
                    // offset loads stay off the chain of dependent shared-memory round trips
                    int o[8];
                    load_offsets8(fl + 3 * s0, o);
#pragma unroll
                    for (int i0 = 0; i0 < 3 * GS; i0 += 8) {
                        const int fb = 3 * s0 + i0;
                        int on[8];
                        if (i0 + 8 < 3 * GS) load_offsets8(fl + fb + 8, on);
                        float val[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const int i = i0 + q;
                            val[q] = i < 3 * GS ? reinterpret_cast<const float *>(&v[i / 3][0])[D - 2 + i % 3] : 0.0f;
                        }
                        if ((real >> (fb >> 3)) & 1u)  // a batch of pass-through nodes only adds nothing
                            flush_batch(myphi, o, val, min(8, 3 * GS - i0), (fok >> (fb >> 3)) & 1u);
                        if (i0 + 8 < 3 * GS) {
#pragma unroll
                            for (int q = 0; q < 8; ++q) o[q] = on[q];
                        }
                    }
                }
                // the nodes above the bottom subtrees
                if (S::NS > 1) {
                    int o[8];
                    load_offsets8(fl + FLB, o);
#pragma unroll
                    for (int u0 = 0; u0 < S::NS - 1; u0 += 8) {
                        int on[8];
                        if (u0 + 8 < S::NS - 1) load_offsets8(fl + FLB + u0 + 8, on);
                        float val[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) val[q] = u0 + q < S::NS - 1 ? acc[u0 + q] : 0.0f;
                        if ((real >> ((FLB + u0) >> 3)) & 1u)
                            flush_batch(myphi, o, val, min(8, S::NS - 1 - u0), (fok >> ((FLB + u0) >> 3)) & 1u);
                        if (u0 + 8 < S::NS - 1) {
#pragma unroll
                            for (int q = 0; q < 8; ++q) o[q] = on[q];
                        }
                    }
                }
            } else {
                // Deep trees: a loop over the NG gather groups.  Group g holds the subtrees
                // g*GS .. g*GS + GS - 1, whose roots are the leaves of the group's own
                // upper subtree (GS - 1 nodes, rooted at level L0); its nodes accumulate
                // in registers and are flushed with the group, so no accumulator lives
                // across groups but the NG - 1 nodes above them, each fed one sum per
                // group (selects that fold away when the loop is unrolled).
                constexpr int NG = X::NG, GL = flush_group_len(D);
                constexpr int LG = ilog2(GS), L0 = D - 2 - LG, NU = GS - 1;
                const uint64_t fok = mt.flush, real = mt.real;
                // decision bits per level, from the groups' roots down (word 0 also holds
                // the levels above them)
                LevelBits<D, L0> lb0(dw);
                LevelBits<D, L0 + 1 < D ? L0 + 1 : D - 1> lb1(dw);
                LevelBits<D, L0 + 2 < D ? L0 + 2 : D - 1> lb2(dw);
                LevelBits<D, L0 + 3 < D ? L0 + 3 : D - 1> lb3(dw);
                LevelBits<D, D - 2> lbr(dw);
                LevelBits<D, D - 1> lbc(dw);
                static_assert(LG <= 4 && L0 <= 3, "group subtrees of at most 4 levels below at most 3 top levels");
                float top[NG - 1];
#pragma unroll
                for (int u = 0; u < NG - 1; ++u) top[u] = 0.0f;
                const unsigned char *lines = reinterpret_cast<const unsigned char *>(job.lines + (size_t)t * LW);
#pragma unroll X::GUNROLL
                for (int g = 0; g < NG; ++g) {
                    if (!((lv >> (g * GS)) & ((1ull << GS) - 1ull))) continue;  // all dead (warp-uniform)
                    // the group's line maps, one byte per subtree
                    uint32_t lm[GS / 4];
                    if constexpr (GS == 16) {
                        const uint4 q = __ldg(reinterpret_cast<const uint4 *>(lines) + g);
                        lm[0] = q.x; lm[1] = q.y; lm[2] = q.z; lm[3] = q.w;
                    } else {
                        static_assert(GS == 8, "groups of 8 or 16 subtrees");
                        const uint2 q = __ldg(reinterpret_cast<const uint2 *>(lines) + g);
                        lm[0] = q.x; lm[1] = q.y;
                    }
                    // path bits from the root to the group's root (exclusive), then the
                    // raw decisions of the group's upper nodes, as in subtree_entries
                    uint32_t P = 0u;
#pragma unroll
                    for (int k = 0; k < L0; ++k) P = (P << 1) | ((dw[0] >> ((1 << k) - 1 + (g >> (L0 - k)))) & 1u);
                    uint32_t ub = lb0.template field<1>(g);
                    if constexpr (LG > 1) ub |= lb1.template field<(LG > 1 ? 2 : 1)>(g) << 1;
                    if constexpr (LG > 2) ub |= lb2.template field<(LG > 2 ? 4 : 1)>(g) << 3;
                    if constexpr (LG > 3) ub |= lb3.template field<(LG > 3 ? 8 : 1)>(g) << 7;
                    const uint32_t rb = lbr.template field<GS>(g);
                    const uint32_t cb = lbc.template field<2 * GS>(g);
                    uint32_t R[NU];
#pragma unroll
                    for (int u = 0; u < NU; ++u) R[u] = ((u == 0 ? P : R[(u - 1) >> 1]) << 1) | ((ub >> u) & 1u);
                    float4 v[GS][Q];
#pragma unroll
                    for (int j = 0; j < GS; ++j) {
                        const int s = g * GS + j;
                        const uint32_t ent = (R[(GS - 2 + j) >> 1] << 3) | (((rb >> j) & 1u) << 2) | ((cb >> (2 * j)) & 3u);
                        const uint32_t lj = (uint32_t)(lv >> s) & 1u;
                        const uint32_t rot = (lm[j >> 2] >> (8 * (j & 3))) & 0xFFu;
                        const float4 *src = tf + ((size_t)s * S::E + line_pos(ent, rot, D)) * Q;
#pragma unroll
                        for (int k = 0; k < Q; ++k) v[j][k] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                        if (Q == 2) {
                            ldg_f8_if(src, v[j][0], v[j][Q > 1 ? 1 : 0], lj);
                        } else {
#pragma unroll
                            for (int k = 0; k < Q; ++k) ldg_f4_if(src + k, v[j][k], lj);
                        }
                    }
                    // the group's upper nodes (local heap order) and the per-group sums of
                    // the levels above it
                    float gl[NU], xk[L0];
#pragma unroll
                    for (int u = 0; u < NU; ++u) gl[u] = 0.0f;
#pragma unroll
                    for (int j = 0; j < GS; ++j) {
#pragma unroll
                        for (int k = 0; k < L0; ++k) xk[k] = j == 0 ? slot_of(v[j], k) : xk[k] + slot_of(v[j], k);
#pragma unroll
                        for (int l = 0; l < LG; ++l) gl[(1 << l) - 1 + (j >> (LG - l))] += slot_of(v[j], L0 + l);
                    }
#pragma unroll
                    for (int k = 0; k < L0; ++k) {
                        const int at = g >> (L0 - k);
#pragma unroll
                        for (int p = 0; p < (1 << k); ++p) top[(1 << k) - 1 + p] += p == at ? xk[k] : 0.0f;
                    }
                    const Off *gfl = fl + g * GL;
                    flush_run<3 * GS>(myphi, gfl, [&](int i) { return slot_of(v[i / 3], D - 2 + i % 3); }, real, fok,
                                      g * (GL / 8));
                    flush_run<NU>(myphi, gfl + FLB, [&](int i) { return gl[i]; }, real, fok, g * (GL / 8) + FLB / 8);
                }
                flush_run<NG - 1>(myphi, fl + NG * GL, [&](int i) { return top[i]; }, real, fok, NG * GL / 8);
            }
        }
    }
    __syncthreads();
    for (int r = warp; r < TC; r += TC / 32) {
        const int64_t row = c0 + r;
        if (row >= n) break;
        float *dst = phi + row * ldp;
        for (int f = lane; f < F; f += 32) dst[f] = sp[f * XS + r];
    }
}

// 1 block per SM is enough (shared memory limits residency anyway): the register
// budget then covers a whole gather group in flight.
template <int D, int TC>
__global__ void __launch_bounds__(TC, 1) k_explain(const unsigned char *__restrict__ codes, int64_t n,
                                                   ExplainJob job, float *__restrict__ phi, int64_t ldp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    explain_tile<D, TC>(job, codes, n, phi, ldp, (int64_t)blockIdx.x * TC, smem_raw);
}

// Persistent form over a ragged batch: work item i is (job, request, first row).  Blocks
// claim items in order from a counter (n_items[1], zero at launch), so expensive items,
// which the host puts first, spread over the whole grid and cheap ones fill the tail.
// The item count n_items[0] is read from device memory, so one captured graph serves
// batches of any size up to its capacity.  Which block computes a tile does not change
// any row's arithmetic.
template <int D, int TC>
__global__ void __launch_bounds__(TC, 1) k_explain_batch(const ExplainJob *__restrict__ jobs,
                                                         const BatchRequest *__restrict__ reqs,
                                                         const int4 *__restrict__ items, int *__restrict__ n_items) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int claimed;
    const int count = n_items[0];
    for (;;) {
        if (threadIdx.x == 0) claimed = atomicAdd(n_items + 1, 1);
        __syncthreads();
        const int i = claimed;
        if (i >= count) break;
        const int4 it = items[i];
        const ExplainJob job = jobs[it.x];
        const BatchRequest rq = reqs[it.y];
        const int64_t c0 = ((int64_t)it.z << 31) | (uint32_t)it.w;
        explain_tile<D, TC>(job, rq.codes, rq.n, rq.phi, rq.ldp, c0, smem_raw);
        __syncthreads();
    }
}

template <int D, int TC>
cudaError_t explain_t(const unsigned char *codes, int64_t n, const ExplainJob &job, float *phi, int64_t ldp,
                      const DevInfo &dev, cudaStream_t st) {
    const size_t smem = ExLayout<D>(job.F, job.ta.n_cols * job.ta.code_bytes, TC).total;
    if (smem > dev.smem_optin) return cudaErrorInvalidConfiguration;
    auto kern = k_explain<D, TC>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    const int64_t blocks = (n + TC - 1) / TC;
    kern<<<(unsigned)blocks, TC, smem, st>>>(codes, n, job, phi, ldp);
    count_launches(1);
    return cudaGetLastError();
}

template <int D, int TC>
cudaError_t batch_t(const ExplainJob *jobs, const BatchRequest *reqs, const int4 *items, int *n_items, int F_max,
                    int xb_max, int grid, const DevInfo &dev, cudaStream_t st) {
    const size_t smem = ExLayout<D>(F_max, xb_max, TC).total;
    if (smem > dev.smem_optin) return cudaErrorInvalidConfiguration;
    auto kern = k_explain_batch<D, TC>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    if (grid <= 0) {
        int per_sm = 0;
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TC, smem);
        if (err != cudaSuccess) return err;
        grid = dev.sms * (per_sm > 0 ? per_sm : 1);
    }
    kern<<<grid, TC, smem, st>>>(jobs, reqs, items, n_items);
    count_launches(1);
    return cudaGetLastError();
}

// Explicit instantiation of the kernels of one (depth, tile rows) pair; each pair is
// compiled in one of the k_explain_d*.cu translation units.
#define WDF_EXPLAIN_TILE(d, tc, spec)                                                                            \
    spec template cudaError_t explain_t<d, tc>(const unsigned char *, int64_t, const ExplainJob &, float *,       \
                                               int64_t, const DevInfo &, cudaStream_t);                          \
    spec template cudaError_t batch_t<d, tc>(const ExplainJob *, const BatchRequest *, const int4 *, int *, int,  \
                                             int, int, const DevInfo &, cudaStream_t);
#define WDF_EXPLAIN_DEPTH(d, spec) WDF_EXPLAIN_TILE(d, 32, spec) WDF_EXPLAIN_TILE(d, 64, spec) \
    WDF_EXPLAIN_TILE(d, 128, spec)

}  // namespace wdf
