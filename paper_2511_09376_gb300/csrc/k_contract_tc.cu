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
// One CTA computes a 128-row tile of one signature group and up to 256 columns.  Operands
// are converted while being staged into shared memory in the K-major, no-swizzle
// core-matrix layout (8 rows x 16 bytes per core matrix; LBO = 128 B between core
// matrices along K, SBO between 8-row groups).  One elected thread issues
// tcgen05.mma for each K step, tcgen05.commit signals an mbarrier, and the four warps
// read the accumulator back with tcgen05.ld for the scaled FP32 epilogue.  Every wait is
// bounded: on expiry the kernel raises the error flag, waits once more (bounded) for its
// own MMAs, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <cstdint>

#include "launch.h"

namespace wdf {

namespace {

constexpr int kRows = 128;
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

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
    for (uint32_t it = 0; it < kWaitLimit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(phase)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Element (row, k) of a kRows x KC operand tile in the core-matrix layout.
template <int EB>
__device__ __forceinline__ uint32_t tile_off(int row, int k, int KC) {
    const int kcb = KC * EB / 16;  // core matrices along K
    return (uint32_t)((row >> 3) * kcb * 128 + ((k * EB) >> 4) * 128 + (row & 7) * 16 + ((k * EB) & 15));
}

// Writes the NP parts of x, part j at part[0] + j * stride.  Each remainder x - sum of
// the earlier parts is exact in FP32 (the parts are x's leading bits).
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

template <bool BF16, int NP>
__global__ void __launch_bounds__(128) k_contract_tc(int D, const float *__restrict__ A,
                                                     const float *__restrict__ scale, const int4 *__restrict__ tiles,
                                                     const float *__restrict__ t32t, float *__restrict__ S, int NT,
                                                     int KC, int *__restrict__ err) {
    constexpr int EB = BF16 ? 2 : 4;
    constexpr int KSTEP = 32 / EB;  // K per MMA: 32 bytes
    extern __shared__ __align__(1024) unsigned char smem[];
    const int K = 1 << D, N = D << D;
    const int KP = K < 16 ? 16 : K;
    const int4 tile = tiles[blockIdx.x];
    const int g = tile.x, r0 = tile.y, r1 = tile.z;
    const int n0 = blockIdx.y * NT;
    const uint32_t a_bytes = (uint32_t)kRows * KC * EB, b_bytes = (uint32_t)NT * KC * EB;
    unsigned char *a_part = smem;                  // NP parts of the A tile, a_bytes apart
    unsigned char *b_part = smem + NP * a_bytes;  // NP parts of the B tile, b_bytes apart
    uint64_t *bar = reinterpret_cast<uint64_t *>(b_part + NP * b_bytes);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int ncols = 32;
    while (ncols < NT) ncols <<= 1;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = instr_desc(BF16, NT, kRows);
    uint32_t phase = 0;
    bool ok = true;
    for (int kc0 = 0; kc0 < KP && ok; kc0 += KC) {
        // stage the split operands of this K chunk
        for (int i = tid; i < kRows * KC; i += 128) {
            const int row = i / KC, k = i % KC;
            const int gr = r0 + row, gk = kc0 + k;
            const float x = (gr < r1 && gk < K) ? __ldg(A + ((size_t)gr << D) + gk) : 0.0f;
            put_split<BF16, NP>(a_part, a_bytes, tile_off<EB>(row, k, KC), x);
        }
        for (int i = tid; i < NT * KC; i += 128) {
            const int col = i / KC, k = i % KC;
            const int gc = n0 + col, gk = kc0 + k;
            const float x = (gc < N && gk < K) ? __ldg(t32t + ((size_t)g * N + gc) * K + gk) : 0.0f;
            put_split<BF16, NP>(b_part, b_bytes, tile_off<EB>(col, k, KC), x);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t sbo_a = (uint32_t)(KC * EB / 16) * 128, sbo_b = sbo_a;
            for (int ks = 0; ks < KC; ks += KSTEP) {
                const uint32_t koff = (uint32_t)(ks / KSTEP) * 256;
                const uint32_t acc = (kc0 > 0 || ks > 0) ? 1u : 0u;
#pragma unroll
                for (int i = 0; i < NP; ++i) {
#pragma unroll
                    for (int j = 0; i + j < NP; ++j) {
                        const uint64_t da = smem_desc(smem_u32(a_part + i * a_bytes) + koff, 128, sbo_a);
                        const uint64_t db = smem_desc(smem_u32(b_part + j * b_bytes) + koff, 128, sbo_b);
                        mma<BF16>(tmem, da, db, idesc, (i + j) ? 1u : acc);
                    }
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(bar)));
        }
        // the MMAs read shared memory asynchronously: wait before restaging it
        ok = __syncthreads_and(mbar_wait(smem_u32(bar), phase)) != 0;
        phase ^= 1u;
    }
    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
        mbar_wait(smem_u32(bar), phase ^ 1u);  // one more bounded wait for the MMAs in flight
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int row = warp * 32 + lane;  // accumulator lane = tile row
        const int grow = r0 + row;
        const float sc = (grow < r1) ? __ldg(scale + grow) : 0.0f;
        for (int c = 0; c < NT; c += 8) {
            uint32_t v[8];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (grow < r1) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int col = n0 + c + j;
                    if (col < N && c + j < NT) S[(size_t)grow * N + col] = __uint_as_float(v[j]) * sc;
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

// mode: 0 = TF32 two parts, 1 = BF16 two parts, 2 = BF16 three parts.
size_t contract_tc_smem(int D, int mode, int *NT, int *KC) {
    const int K = 1 << D, N = D << D;
    const int KP = K < 16 ? 16 : K;
    int nt = N < 256 ? N : 256;
    nt = (nt + 15) / 16 * 16;
    const int eb = mode ? 2 : 4, np = mode == 2 ? 3 : 2;
    int kc = mode == 1 ? 128 : 64;  // 256 bytes of K per row and part (128 B with three parts)
    if (kc > KP) kc = KP;
    *NT = nt;
    *KC = kc;
    return (size_t)np * (kRows + nt) * kc * eb + 16;
}

cudaError_t launch_contract_tc(int D, int mode, const float *A, const float *scale, const int4 *tiles, int n_tiles,
                               const float *t32t, float *S, int *err, cudaStream_t st) {
    if (n_tiles == 0) return cudaSuccess;
    if (mode < 0 || mode > 2) return cudaErrorInvalidValue;
    int NT = 0, KC = 0;
    const size_t smem = contract_tc_smem(D, mode, &NT, &KC);
    const int N = D << D;
    dim3 grid(n_tiles, (N + NT - 1) / NT);
    auto kern = mode == 0 ? k_contract_tc<false, 2> : (mode == 1 ? k_contract_tc<true, 2> : k_contract_tc<true, 3>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, 128, smem, st>>>(D, A, scale, tiles, t32t, S, NT, KC, err);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace wdf
