// sre_tc.cuh -- tensor-core Hadamard stage (tcgen05, sm_100+/sm_103a).
//
// One round of the tile transform -- the butterflies over four index bits,
// i.e. a multiplication of each 16-entry row by H_16 = H_2^{(x)4} (the
// recursion of the supplement's FWHT section) -- done as a dense MMA:
//
//   D[m][n] = sum_k A[m][k] H_16[n][k],   H_16[n][k] = (-1)^{popc(n & k)},
//
// with A = the thread rows of the tile in round-0 layout (thread tid owns
// row tid: its 16 entries e = 16 tid + i), real and imaginary parts as
// separate rows (4 M-blocks of 128 rows).  H_16 has exact +-1 entries, so
// the only rounding is in representing A: each FP32 value v is split as
// hi = round(v), lo = round(v - hi) in BF16 (or FP16, after a per-row power
// of two scaling that keeps the row inside FP16's range), and the MMA
// accumulates D = A_hi H + A_lo H in FP32 in tensor memory.
//
// Operands live in shared memory in the canonical no-swizzle K-major layout
// of 8-row x 16-byte core matrices: element (row r, k) at byte
//   (r / 8) * 256 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2,
// so the descriptors use leading (K) byte offset 128 and stride (M/N) byte
// offset 256.  One thread issues the 8 MMAs (M = 128, N = 16, K = 16) of a
// tile and commits them to an mbarrier; every thread waits on it (bounded by
// %globaltimer) and reads its two rows back from TMEM with tcgen05.ld
// (warp w reaches lanes 32 (w % 4) .. + 31).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sre_tile.cuh"

namespace sre {
namespace dev {

enum TcKind { kTcNone = 0, kTcBf16 = 1, kTcFp16 = 2 };

constexpr int kTcCols = 64;        // TMEM columns per CTA: 4 M-blocks x N = 16
constexpr int kTcATileBytes = 4096;  // 128 rows x 16 x 2 bytes
constexpr int kTcABytes = 8 * kTcATileBytes;  // 4 blocks x (hi, lo) = 32 KB
constexpr int kTcBBytes = 512;      // H_16, 16 x 16 x 2 bytes

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (r, k) of a K = 16 operand in the canonical layout
__host__ __device__ constexpr int tc_off(int r, int k) {
    return (r >> 3) * 256 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// tcgen05 shared-memory matrix descriptor, no swizzle, K-major
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);          // start address
    d |= (uint64_t)(128 >> 4) << 16;                  // leading (K) byte offset
    d |= (uint64_t)(256 >> 4) << 32;                  // stride (M/N) byte offset
    d |= (uint64_t)1 << 46;                           // descriptor version
    return d;                                         // base offset 0, no swizzle
}

// instruction descriptor: kind::f16, F32 accumulate, A/B = BF16 or FP16,
// both K-major, M = 128, N = 16
template <int KIND>
__host__ __device__ constexpr uint32_t tc_idesc() {
    return (1u << 4)                                  // D format F32
           | ((KIND == kTcBf16 ? 1u : 0u) << 7)       // A format
           | ((KIND == kTcBf16 ? 1u : 0u) << 10)      // B format
           | ((16u >> 3) << 17)                       // N / 8
           | ((128u >> 4) << 24);                     // M / 16
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// whole warp: allocate kTcCols TMEM columns, address written to *slot
__device__ __forceinline__ void tc_alloc(uint32_t *slot) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_dealloc(uint32_t taddr) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTcCols) : "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity; false on expiry.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity, long long wait_ns) {
    const unsigned long long t0 = globaltimer_ns();
    for (unsigned it = 0; it < (1u << 28); ++it) {
        if (mbar_try_wait(mbar, parity)) return true;
        if ((it & 15) == 15 && (long long)(globaltimer_ns() - t0) > wait_ns) return false;
    }
    return false;
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&r)[16]) {
    uint32_t u[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
          "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]),
          "=r"(u[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) r[i] = __uint_as_float(u[i]);
}

// Split 16 values of one row into hi / lo halves and store them as rows
// `row` of the hi and lo A tiles (canonical layout, two 16-byte chunks each).
template <int KIND>
__device__ __forceinline__ void tc_store_row(const float (&x)[16], unsigned char *a_hi,
                                             unsigned char *a_lo, int row) {
    uint32_t hi[8], lo[8];
#pragma unroll
    for (int k = 0; k < 16; k += 2) {
        if (KIND == kTcBf16) {
            const __nv_bfloat16 h0 = __float2bfloat16_rn(x[k]), h1 = __float2bfloat16_rn(x[k + 1]);
            const __nv_bfloat16 l0 = __float2bfloat16_rn(x[k] - __bfloat162float(h0));
            const __nv_bfloat16 l1 = __float2bfloat16_rn(x[k + 1] - __bfloat162float(h1));
            hi[k >> 1] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            lo[k >> 1] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
        } else {
            const __half h0 = __float2half_rn(x[k]), h1 = __float2half_rn(x[k + 1]);
            const __half l0 = __float2half_rn(x[k] - __half2float(h0));
            const __half l1 = __float2half_rn(x[k + 1] - __half2float(h1));
            hi[k >> 1] = (uint32_t)__half_as_ushort(h0) | ((uint32_t)__half_as_ushort(h1) << 16);
            lo[k >> 1] = (uint32_t)__half_as_ushort(l0) | ((uint32_t)__half_as_ushort(l1) << 16);
        }
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        *reinterpret_cast<uint4 *>(a_hi + tc_off(row, 8 * c)) =
            make_uint4(hi[4 * c], hi[4 * c + 1], hi[4 * c + 2], hi[4 * c + 3]);
        *reinterpret_cast<uint4 *>(a_lo + tc_off(row, 8 * c)) =
            make_uint4(lo[4 * c], lo[4 * c + 1], lo[4 * c + 2], lo[4 * c + 3]);
    }
}

// Per-CTA state of the tensor stage.
struct TcState {
    unsigned char *a;     // kTcABytes of shared memory (A tiles)
    unsigned char *b;     // kTcBBytes of shared memory (H_16)
    uint32_t mbar;        // shared address of the mbarrier
    uint32_t tmem;        // TMEM base address
    uint32_t phase;       // parity of the next completion
};

// Write H_16 into b (all threads cooperate; caller synchronises).
template <int KIND>
__device__ __forceinline__ void tc_init_h16(unsigned char *b, int tid, int nthreads) {
    for (int idx = tid; idx < 256; idx += nthreads) {
        const int n = idx >> 4, k = idx & 15;
        const float h = (__popc(n & k) & 1) ? -1.f : 1.f;
        unsigned short bits;
        if (KIND == kTcBf16)
            bits = __bfloat16_as_ushort(__float2bfloat16_rn(h));
        else
            bits = __half_as_ushort(__float2half_rn(h));
        *reinterpret_cast<unsigned short *>(b + tc_off(n, k)) = bits;
    }
}

// The tensor round: butterflies over tile bits 0-3 of a tile in round-0
// layout (v[i] = entry 16 tid + i), in place.  All 256 threads call it.
// Returns false if the bounded wait expired (v is then unreliable).
template <int KIND>
__device__ __forceinline__ bool tc_round0(cx_t<float> (&v)[16], TcState &tc, int tid, long long wait_ns) {
    const int half_rows = tid >> 7;  // which 128-thread half: M-block 0/1 (re), 2/3 (im)
    const int row = tid & 127;
    float re[16], im[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) Cx<float>::unpack(v[i], re[i], im[i]);
    float sre = 1.f, sim = 1.f;  // FP16: per-row power-of-two scale
    if (KIND == kTcFp16) {
        float mr = 0.f, mi = 0.f;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            mr = fmaxf(mr, fabsf(re[i]));
            mi = fmaxf(mi, fabsf(im[i]));
        }
        // scale so the row maximum lies in [2^10, 2^11): FP16 keeps ~2^-24 of it in hi + lo
        int er = 0, ei = 0;
        frexpf(mr, &er);
        frexpf(mi, &ei);
        sre = mr > 0.f ? ldexpf(1.f, 11 - er) : 1.f;
        sim = mi > 0.f ? ldexpf(1.f, 11 - ei) : 1.f;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            re[i] *= sre;
            im[i] *= sim;
        }
    }
    unsigned char *blk_re = tc.a + (0 + half_rows) * 2 * kTcATileBytes;
    unsigned char *blk_im = tc.a + (2 + half_rows) * 2 * kTcATileBytes;
    tc_store_row<KIND>(re, blk_re, blk_re + kTcATileBytes, row);
    tc_store_row<KIND>(im, blk_im, blk_im + kTcATileBytes, row);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
        tc_fence_after();
        const uint64_t bdesc = tc_desc(smem_u32(tc.b));
        constexpr uint32_t idesc = tc_idesc<KIND>();
#pragma unroll
        for (int blk = 0; blk < 4; ++blk) {
            const uint32_t a_hi = smem_u32(tc.a + blk * 2 * kTcATileBytes);
            const uint32_t d = tc.tmem + blk * 16;
            tc_mma(d, tc_desc(a_hi), bdesc, idesc, 0u);
            tc_mma(d, tc_desc(a_hi + kTcATileBytes), bdesc, idesc, 1u);
        }
        tc_commit(tc.mbar);
    }
    const bool ok = mbar_wait_bounded(tc.mbar, tc.phase, wait_ns);
    tc.phase ^= 1u;
    tc_fence_after();
    const uint32_t lane_base = (uint32_t)(32 * ((tid >> 5) & 3)) << 16;
    float dre[16], dim[16];
    tc_ld16(tc.tmem + lane_base + (uint32_t)((0 + half_rows) * 16), dre);
    tc_ld16(tc.tmem + lane_base + (uint32_t)((2 + half_rows) * 16), dim);
    tc_fence_before();
    const float ire = 1.f / sre, iim = 1.f / sim;
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = Cx<float>::pack(dre[i] * ire, dim[i] * iim);
    return ok;
}

}  // namespace dev
}  // namespace sre
