// Step 3 of Algorithm 3 on the 5th-generation tensor cores: the stacked contraction
// S[row][k * 2^D + p_c] = scale[row] * sum_p A[row][p] * T[g][p][k * 2^D + p_c]
// (Eq. "bg_shap_derivation" step (f) for every leaf of one path signature at once) with
// split-precision operands accumulated in FP32 in tensor memory.  Two-part splits
// X = X_0 + X_1 (both parts rounded to TF32, kind::tf32, or to BF16, kind::f16) take
// three products A_0 B_0 + A_0 B_1 + A_1 B_0; the dropped A_1 B_1 term is below the
// rounding of the rest, so the result carries the parts' 2 x 11 (TF32) or 2 x 8 (BF16)
// significant bits.  The three-part BF16 split X = X_0 + X_1 + X_2 holds every FP32
// value exactly (3 x 8 bits) and takes the six products A_i B_j with i + j <= 2; the
// dropped ones are below 2^-24 relative, FP32 accuracy.
//
// The operands are split once, outside the GEMM, straight into the shared-memory image
// the MMAs read: the K-major, no-swizzle core-matrix layout (8 rows x 16 bytes per core
// matrix; LBO = 128 B between the two core matrices of a 32-byte K step, SBO = 256 B
// between 8-row groups).  One "stage" is one K step (32 bytes of K per row and part) of
// every part of the A tile (128 rows) and the B tile (NT <= 256 columns), contiguous in
// global memory, so it arrives with two bulk copies (cp.async.bulk, the TMA engine's
// linear form) that signal a "full" mbarrier by transaction count.  A ring of stages is
// kept in flight: one thread issues the copies of stage i while the tensor cores work
// on stage i - (ring - 1); each stage's MMAs end with tcgen05.commit on its "empty"
// mbarrier, which the copy of the stage that reuses the slot waits for.  A last commit
// signals "done"; the four warps then read the accumulator with tcgen05.ld for the
// scaled FP32 epilogue.  The ring is sized so that two CTAs fit on an SM, which lets
// one CTA's epilogue overlap the other's MMAs.
//
// Every wait is bounded.  When one gives up, the CTA raises the error flag, still waits
// at the normal limit for the copies and MMAs it has started (so no copy lands in shared
// memory and no MMA reads it after the CTA has left), frees its tensor memory and
// returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cstdint>

#include "launch.h"

namespace wdf {

// Poll limit of the first mbarrier wait of every CTA (0: the normal limit).  Tests set it
// to make that wait expire on purpose; the waits that drain the copies and MMAs in flight
// before the tensor memory is freed always keep the normal limit.
static std::atomic<uint32_t> g_first_wait_limit{0};
void set_contract_first_wait_limit(uint32_t polls) { g_first_wait_limit.store(polls); }

namespace {

constexpr int kRows = 128;                  // M of one CTA tile (TMEM lanes)
constexpr int kStepBytes = 32;              // K bytes per row and part of one stage (one MMA K step)
constexpr int kMaxNT = 256;                 // N of one CTA tile
constexpr int kRingBudget = 110 * 1024;     // shared memory of a CTA's ring: two CTAs per SM
constexpr uint32_t kWaitLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Shared-memory matrix descriptor: start address, LBO, SBO (all >> 4), descriptor
// version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor: FP32 accumulator, A/B format (TF32 = 2, BF16 = 1), both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t instr_desc(bool bf16, int n, int m) {
    const uint32_t fmt = bf16 ? 1u : 2u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

template <bool BF16>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if (BF16) {
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    }
}

__device__ __forceinline__ void commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// Bounded wait for the phase of an mbarrier.  At the normal limit it polls with
// try_wait (which may suspend the thread for a short while between polls); a shorter
// limit (the test hook) polls with the non-suspending test_wait, so that the limit
// counts polls and nothing else.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, uint32_t limit = kWaitLimit) {
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t ok;
        if (limit >= kWaitLimit)
            asm volatile(
                "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(ok)
                : "r"(bar), "r"(phase)
                : "memory");
        else
            asm volatile(
                "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(ok)
                : "r"(bar), "r"(phase)
                : "memory");
        if (ok) return true;
    }
    return false;
}

// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from global to
// shared memory, completing `bytes` transactions on the mbarrier.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Byte offset of element (row, kbyte) inside one part of a stage: rows in 8-row groups of
// 256 bytes (two core matrices of 8 rows x 16 bytes along K).
__host__ __device__ __forceinline__ uint32_t core_off(int row, int kbyte) {
    return (uint32_t)((row >> 3) * 256 + (kbyte >> 4) * 128 + (row & 7) * 16 + (kbyte & 15));
}

// Writes the NP parts of x at part[0] + j * stride + off.  Each remainder x - (sum of
// the earlier parts) is exact in FP32 (the parts are x's leading bits).
template <bool BF16, int NP>
__device__ __forceinline__ void put_split(unsigned char *part, uint32_t stride, uint32_t off, float x) {
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        if (BF16) {
            const __nv_bfloat16 h = __float2bfloat16_rn(x);
            *reinterpret_cast<__nv_bfloat16 *>(part + j * stride + off) = h;
            x -= __bfloat162float(h);
        } else {
            const float h = tf32_rna(x);
            *reinterpret_cast<float *>(part + j * stride + off) = h;
            x -= h;
        }
    }
}

}  // namespace

// A operand: rows [r0, r1) of group tile t (A row-major [row][2^D] FP32), split into
// stages [tile][step][part][128 x 32 B].  One thread per (tile, step, row, element).
template <bool BF16, int NP>
__global__ void k_pack_a(int D, const float *__restrict__ A, const int4 *__restrict__ tiles, int n_tiles, int nk,
                         unsigned char *__restrict__ out) {
    constexpr int EB = BF16 ? 2 : 4, KS = kStepBytes / EB;
    const int64_t total = (int64_t)n_tiles * nk * kRows * KS;
    const int K = 1 << D;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int kk = (int)(i % KS);
        const int row = (int)((i / KS) % kRows);
        const int64_t ts = i / ((int64_t)KS * kRows);  // tile * nk + step
        const int t = (int)(ts / nk), ks = (int)(ts % nk);
        const int4 tile = tiles[t];
        const int gr = tile.y + row, gk = ks * KS + kk;
        const float x = (gr < tile.z && gk < K) ? __ldg(A + ((size_t)gr << D) + gk) : 0.0f;
        unsigned char *stage = out + (size_t)ts * NP * kRows * kStepBytes;
        put_split<BF16, NP>(stage, kRows * kStepBytes, core_off(row, kk * EB), x);
    }
}

// B operand: the FP32 tables t32 [G][2^D][D * 2^D] as N x K (K-major) tiles of NT
// columns, split into stages [group][column block][step][part][NT x 32 B].
template <bool BF16, int NP>
__global__ void k_pack_b(int D, const float *__restrict__ t32, int G, int NT, int NB, int nk,
                         unsigned char *__restrict__ out) {
    constexpr int EB = BF16 ? 2 : 4, KS = kStepBytes / EB;
    const int K = 1 << D, N = D << D;
    const int64_t total = (int64_t)G * NB * nk * NT * KS;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int kk = (int)(i % KS);
        const int col = (int)((i / KS) % NT);
        const int64_t gbs = i / ((int64_t)KS * NT);  // (group * NB + block) * nk + step
        const int ks = (int)(gbs % nk);
        const int64_t gb = gbs / nk;
        const int nb = (int)(gb % NB), g = (int)(gb / NB);
        const int n = nb * NT + col, pb = ks * KS + kk;
        const float x = (n < N && pb < K) ? __ldg(t32 + ((size_t)g * K + pb) * N + n) : 0.0f;
        unsigned char *stage = out + (size_t)gbs * NP * NT * kStepBytes;
        put_split<BF16, NP>(stage, (uint32_t)NT * kStepBytes, core_off(col, kk * EB), x);
    }
}

// One CTA: a 128-row tile (of signature group tiles[.].x) times a column block of NT
// columns, over nk K steps through a ring of `ring` stages.  The column blocks of one
// tile are consecutive CTAs (blockIdx.x = tile * NB + block), so they run together and
// read the tile's A stages from L2 rather than each from HBM.
template <bool BF16, int NP>
__global__ void __launch_bounds__(128) k_contract_tc(int D, const unsigned char *__restrict__ apk,
                                                     const unsigned char *__restrict__ bpk,
                                                     const float *__restrict__ scale, const int4 *__restrict__ tiles,
                                                     float *__restrict__ S, int NT, int NB, int nk, int ring,
                                                     int *__restrict__ err, uint32_t first_limit) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int N = D << D;
    const int ti = (int)(blockIdx.x / (unsigned)NB), nb = (int)(blockIdx.x % (unsigned)NB);
    const int4 tile = tiles[ti];
    const int g = tile.x, r0 = tile.y, r1 = tile.z;
    const int n0 = nb * NT;
    const uint32_t a_bytes = (uint32_t)NP * kRows * kStepBytes, b_bytes = (uint32_t)NP * NT * kStepBytes;
    const uint32_t stage_bytes = a_bytes + b_bytes;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)ring * stage_bytes);
    uint64_t *empty = full + ring;
    uint64_t *done = empty + ring;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int ncols = 32;
    while (ncols < NT) ncols <<= 1;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < ring; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(full + s)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(empty + s)));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(done)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    bool failed = false;
    if (tid == 0) {
        // copies run ring - 1 stages ahead of the MMAs
        const unsigned char *asrc = apk + (size_t)ti * nk * a_bytes;
        const unsigned char *bsrc = bpk + ((size_t)g * NB + nb) * nk * b_bytes;
        const uint32_t idesc = instr_desc(BF16, NT, kRows);
        const uint32_t smem0 = smem_u32(smem);
        int produced = 0, consumed = 0;
        bool first = true;
        for (int i = 0; i < nk + ring - 1; ++i) {
            if (i < nk) {
                const int s = i % ring;
                if (i >= ring && !mbar_wait(smem_u32(empty + s), (uint32_t)((i / ring) - 1) & 1u)) {
                    failed = true;
                    break;
                }
                const uint32_t fb = smem_u32(full + s), dst = smem0 + (uint32_t)s * stage_bytes;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(stage_bytes)
                             : "memory");
                bulk_g2s(dst, asrc + (size_t)i * a_bytes, a_bytes, fb);
                bulk_g2s(dst + a_bytes, bsrc + (size_t)i * b_bytes, b_bytes, fb);
                ++produced;
            }
            const int j = i - (ring - 1);
            if (j >= 0) {
                const int s = j % ring;
                if (!mbar_wait(smem_u32(full + s), (uint32_t)(j / ring) & 1u, first ? first_limit : kWaitLimit)) {
                    failed = true;
                    break;
                }
                first = false;
                ++consumed;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t abase = smem0 + (uint32_t)s * stage_bytes, bbase = abase + a_bytes;
#pragma unroll
                for (int pa = 0; pa < NP; ++pa) {
#pragma unroll
                    for (int pb = 0; pa + pb < NP; ++pb) {
                        const uint64_t da = smem_desc(abase + (uint32_t)pa * kRows * kStepBytes, 128, 256);
                        const uint64_t db = smem_desc(bbase + (uint32_t)pb * NT * kStepBytes, 128, 256);
                        mma<BF16>(tmem, da, db, idesc, (j > 0 || pa + pb > 0) ? 1u : 0u);
                    }
                }
                commit(smem_u32(empty + s));
            }
        }
        if (failed) {
            // let every copy already started land before the shared memory is given back
            for (int c = consumed; c < produced; ++c) mbar_wait(smem_u32(full + c % ring), (uint32_t)(c / ring) & 1u);
        }
        commit(smem_u32(done));  // arrives once every MMA issued above has completed
    }
    const bool done_ok = mbar_wait(smem_u32(done), 0u);
    const bool bad = __syncthreads_or(failed || !done_ok) != 0;
    if (bad) {
        if (tid == 0) atomicExch(err, 1);
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int row = warp * 32 + lane;  // accumulator lane = tile row
        const int grow = r0 + row;
        const float sc = (grow < r1) ? __ldg(scale + grow) : 0.0f;
        float *dst = S + (size_t)grow * N + n0;
        for (int c = 0; c < NT; c += 16) {
            uint32_t v[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (grow < r1) {
                if (n0 + c + 16 <= N) {
                    // N is a multiple of 8 floats and c of 16: 16-byte aligned stores
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        *reinterpret_cast<float4 *>(dst + c + 4 * q) =
                            make_float4(__uint_as_float(v[4 * q]) * sc, __uint_as_float(v[4 * q + 1]) * sc,
                                        __uint_as_float(v[4 * q + 2]) * sc, __uint_as_float(v[4 * q + 3]) * sc);
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        if (n0 + c + q < N) dst[c + q] = __uint_as_float(v[q]) * sc;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
    }
}

TcGeom tc_geom(int D, int mode) {
    TcGeom g;
    const int K = 1 << D, N = D << D;
    const int eb = mode ? 2 : 4;
    g.np = mode == 2 ? 3 : 2;
    const int ks = kStepBytes / eb;
    g.nk = std::max(K, ks) / ks;
    const int nt = std::min(N, kMaxNT);
    g.NT = (nt + 15) / 16 * 16;
    g.NB = (N + g.NT - 1) / g.NT;
    g.a_stage = (uint32_t)g.np * kRows * kStepBytes;
    g.b_stage = (uint32_t)g.np * g.NT * kStepBytes;
    g.ring = std::max(1, std::min(g.nk, kRingBudget / (int)(g.a_stage + g.b_stage)));
    g.smem = (size_t)g.ring * (g.a_stage + g.b_stage) + (size_t)(2 * g.ring + 1) * 8 + 16;
    return g;
}

size_t contract_tc_a_bytes(int D, int n_tiles) {
    size_t best = 0;
    for (int mode = 0; mode < 3; ++mode) {
        const TcGeom g = tc_geom(D, mode);
        best = std::max(best, (size_t)n_tiles * g.nk * g.a_stage);
    }
    return best;
}

size_t contract_tc_b_bytes(int D, int mode, int G) {
    const TcGeom g = tc_geom(D, mode);
    return (size_t)G * g.NB * g.nk * g.b_stage;
}

static int pack_grid(int64_t total) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 32));
}

cudaError_t launch_pack_b(int D, int mode, const float *t32, int G, unsigned char *bpk, cudaStream_t st) {
    if (G == 0) return cudaSuccess;
    if (mode < 0 || mode > 2) return cudaErrorInvalidValue;
    const TcGeom g = tc_geom(D, mode);
    const int64_t total = (int64_t)G * g.NB * g.nk * g.NT * (kStepBytes / (mode ? 2 : 4));
    auto kern = mode == 0 ? k_pack_b<false, 2> : (mode == 1 ? k_pack_b<true, 2> : k_pack_b<true, 3>);
    kern<<<pack_grid(total), 256, 0, st>>>(D, t32, G, g.NT, g.NB, g.nk, bpk);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_contract_tc(int D, int mode, const float *A, const float *scale, const int4 *tiles, int n_tiles,
                               unsigned char *apk, const unsigned char *bpk, float *S, int *err, cudaStream_t st) {
    if (n_tiles == 0) return cudaSuccess;
    if (mode < 0 || mode > 2) return cudaErrorInvalidValue;
    const TcGeom g = tc_geom(D, mode);
    const int64_t total = (int64_t)n_tiles * g.nk * kRows * (kStepBytes / (mode ? 2 : 4));
    auto pack = mode == 0 ? k_pack_a<false, 2> : (mode == 1 ? k_pack_a<true, 2> : k_pack_a<true, 3>);
    pack<<<pack_grid(total), 256, 0, st>>>(D, A, tiles, n_tiles, g.nk, apk);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    auto kern = mode == 0 ? k_contract_tc<false, 2> : (mode == 1 ? k_contract_tc<true, 2> : k_contract_tc<true, 3>);
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
    if (e != cudaSuccess) return e;
    const uint32_t first = g_first_wait_limit.load();
    kern<<<(unsigned)((int64_t)n_tiles * g.NB), 128, g.smem, st>>>(D, apk, bpk, scale, tiles, S, g.NT, g.NB, g.nk, g.ring, err,
                                    first ? first : kWaitLimit);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace wdf
