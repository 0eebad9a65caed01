// sre_tc.cuh -- tcgen05 primitives and the fixed-point hi/lo split of the
// tensor-core Hadamard stages (split-precision modes).
//
// The supplement's FWHT section writes H_{2^N} = H_2^{(x)N} (block recursion),
// so every group of index bits is transformed by an exact +-1 Hadamard
// factor.  A stage over 7 bits is the dense product D = H_128 B, with H_128 in
// tensor memory as the A operand and the data B in shared memory.
//
// Fixed point.  The tensor cores accumulate in FP32 without round-to-nearest;
// sums of integers below 2^24 are nevertheless exact.  So a block of FP32
// values v that shares one power-of-two scale s is split as
//   h  = rn(v s)            an integer with |h| <= 2^P,
//   l  = rn_T(v s - h)      |l| <= 1/2, rounded to the piece type T,
// with P = 8 for BF16 and P = 11 for FP16 (the integers a piece holds
// exactly).  The two pieces form the two 64-column halves of one N = 128
// operand, so the MMA accumulates H h and H l in separate TMEM columns: the
// first sum is an exact integer (|sum| <= 2^(P+7)), the second only feels
// truncation far below the result's own rounding.  The value is represented
// to 2^-(2P+2) of the block maximum (18 bits for BF16, 24 for FP16).  The hi
// piece is stored negated (-h comes out of the rounding for free), so a
// result is lo - hi.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sre_async.cuh"
#include "sre_tile.cuh"

namespace sre {
namespace dev {

enum TcKind { kTcNone = 0, kTcBf16 = 1, kTcFp16 = 2 };

// Integer bits held exactly by one piece (hi in [-2^P, 2^P]).
template <int KIND>
__host__ __device__ constexpr int tc_piece_bits() {
    return KIND == kTcBf16 ? 8 : 11;
}

// ---------------------------------------------------------------- fences

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// ---------------------------------------------------- tensor memory (TMEM)

// Whole warp: allocate ncols (power of two >= 32) columns; address to *slot.
__device__ __forceinline__ void tc_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Whole warp: 8 consecutive 32-bit columns of this warp's 32 lanes.
__device__ __forceinline__ void tc_st8(uint32_t taddr, const uint32_t (&r)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}

__device__ __forceinline__ void tc_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Whole warp: 16 consecutive 32-bit columns of this warp's 32 lanes (lane i
// of the warp gets TMEM lane 32 (warp % 4) + i).  Complete after tc_wait_ld.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&u)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
          "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ------------------------------------------------------------------- MMA

// Shared-memory matrix descriptor (sm_100 format: start, leading and stride
// byte offsets in 16-byte units, version 1, swizzle mode in bits 61-63).
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t swizzle) {
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46) | ((uint64_t)swizzle << 61);
}

// B operand, N-major (N contiguous), no swizzle: core matrices of 8 K-rows x
// 16 bytes; `kgroup` = byte stride between 8-row groups along K (leading
// offset), `ngroup` = byte stride between 8-column groups along N (stride
// offset).  These roles were established on GB300 with integer operands
// (the other assignment gives wrong sums).
__device__ __forceinline__ uint64_t tc_desc_mn(uint32_t saddr, uint32_t kgroup, uint32_t ngroup) {
    return tc_desc(saddr, kgroup, ngroup, 0);
}

// B operand, N-major, 128-byte swizzle (the layout a TMA box of 128-byte rows
// with CU_TENSOR_MAP_SWIZZLE_128B writes): atoms of 8 K-rows x 128 bytes,
// 8-row groups 1024 bytes apart (stride offset), 64-element atom columns
// `atom_col` bytes apart (leading offset).  Start address 1024-aligned.
__device__ __forceinline__ uint64_t tc_desc_mn_sw128(uint32_t saddr, uint32_t atom_col) {
    return tc_desc(saddr, atom_col, 1024, 2);
}

// Instruction descriptor, kind::f16: FP32 accumulate, A and B both BF16 or
// both FP16, A K-major (from TMEM), B N-major, M = 128.
template <int KIND>
__host__ __device__ constexpr uint32_t tc_idesc(int N) {
    return (1u << 4)                                  // D format F32
           | ((KIND == kTcBf16 ? 1u : 0u) << 7)       // A format
           | ((KIND == kTcBf16 ? 1u : 0u) << 10)      // B format
           | (1u << 16)                               // B N-major
           | ((uint32_t)(N >> 3) << 17)               // N / 8
           | ((128u >> 4) << 24);                     // M / 16
}

// D[tmem d] (+)= A[tmem a] * B[smem desc]; issued by one thread.
__device__ __forceinline__ void tc_mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// One Hadamard stage of a tile: eight MMAs (K = 16 each, 128 in all) into
// the accumulator d, A from TMEM columns a0 + 8 s, B from the descriptor
// b0 advanced by bstep (in 16-byte units) per K step; the first MMA
// overwrites d.  One asm block, so that the eight issue back to back.
__device__ __forceinline__ void tc_mma_stage(uint32_t d, uint32_t a0, uint64_t b0, uint32_t bstep, uint32_t idesc) {
    const uint64_t s = bstep;
    asm volatile(
        "{\n\t.reg .pred p0, p1;\n\t"
        "setp.ne.b32 p0, %18, %18;\n\t"
        "setp.eq.b32 p1, %18, %18;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %9, %17, p0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%2], %10, %17, p1;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%3], %11, %17, p1;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%4], %12, %17, p1;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%5], %13, %17, p1;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%6], %14, %17, p1;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%7], %15, %17, p1;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%8], %16, %17, p1;\n\t}\n" ::"r"(d),
        "r"(a0), "r"(a0 + 8u), "r"(a0 + 16u), "r"(a0 + 24u), "r"(a0 + 32u), "r"(a0 + 40u), "r"(a0 + 48u),
        "r"(a0 + 56u), "l"(b0), "l"(b0 + s), "l"(b0 + 2 * s), "l"(b0 + 3 * s), "l"(b0 + 4 * s),
        "l"(b0 + 5 * s), "l"(b0 + 6 * s), "l"(b0 + 7 * s), "r"(idesc), "r"(0)
        : "memory");
}

// Arrive on mbar once every MMA this thread issued before has completed.
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// ------------------------------------------------------ fixed-point split

// Two FP32 values as one word of two pieces, a in the low half.
template <int KIND>
__device__ __forceinline__ uint32_t tc_pack2(float a, float b) {
    uint32_t d;
    if (KIND == kTcBf16)
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
    else
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
    return d;
}

constexpr float kRoundMagic = 12582912.0f;  // 1.5 * 2^23: x + M - M = rn(x) for |x| < 2^22

// Split the packed pair v (re, im) scaled by the packed pair s into the
// negated integer piece (-rn(v s)) and the remainder piece; both words hold
// (re, im) with re in the low half.
template <int KIND>
__device__ __forceinline__ void tc_split(unsigned long long v, unsigned long long s, unsigned long long magic,
                                         uint32_t &hi_neg, uint32_t &lo) {
    unsigned long long t, nh, r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(t) : "l"(v), "l"(s), "l"(magic));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(nh) : "l"(magic), "l"(t));  // -rn(v s), exact
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(v), "l"(s), "l"(nh));  // v s - rn(v s), exact
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(nh));
    hi_neg = tc_pack2<KIND>(a, b);
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
    lo = tc_pack2<KIND>(a, b);
}

// Power of two 2^(P - e) for a block maximum m = f 2^e (f in [1/2, 1)), so
// that m 2^(P - e) < 2^P; 1 for m = 0; kept inside the normal FP32 range.
template <int P>
__device__ __forceinline__ float tc_block_scale(float m) {
    if (!(m > 0.f)) return 1.f;
    int e;
    (void)frexpf(m, &e);
    const int k = max(-126, min(126, P - e));
    return __int_as_float((k + 127) << 23);
}

// Write the 128 x 128 A operand of a stage into TMEM columns [col, col + 64)
// (two pieces per 32-bit column, k even in the low half): the Hadamard
// matrix H_128[m][k] = (-1)^popc(m & k) for G = 7, or the block-diagonal
// I_{2^(7-G)} (x) H_{2^G} for G < 7.  Warps 0-3 call it (warp w writes lanes
// 32 w .. 32 w + 31); complete after tc_wait_st.
template <int KIND>
__device__ __forceinline__ void tc_write_hadamard(uint32_t tmem, int col, int G, int warp, int lane) {
    const int m = 32 * warp + lane;
    const int blk = ~((1 << G) - 1);
    const unsigned short one = KIND == kTcBf16 ? 0x3F80 : 0x3C00;
    const unsigned short neg = KIND == kTcBf16 ? 0xBF80 : 0xBC00;
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 8) {
        uint32_t r[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            uint32_t w = 0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = 2 * (c0 + j) + h;
                const unsigned short v =
                    ((m & blk) != (k & blk)) ? (unsigned short)0 : ((__popc(m & k & ~blk) & 1) ? neg : one);
                w |= (uint32_t)v << (16 * h);
            }
            r[j] = w;
        }
        tc_st8(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(col + c0), r);
    }
}

}  // namespace dev
}  // namespace sre
