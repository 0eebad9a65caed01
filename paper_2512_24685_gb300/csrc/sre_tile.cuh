// sre_tile.cuh -- in-CTA Walsh-Hadamard machinery on a tile of 2^12 complex
// entries held by 256 threads (16 entries each, i.e. 4 "register bits").
//
// The transform is the unnormalised WHT of the supplement's FWHT section:
// stage b maps each pair (a, c) of entries whose indices differ only in bit b
// to (a + c, a - c).  Stages commute, so the 12 bits are done in three rounds
// of four: round k does the butterflies over bits [4k, 4k+4) entirely in
// registers; between rounds the tile is rewritten through shared memory so
// that the next four bits become the register bits.
//
// Round layouts (tid in [0, 256), register slot i in [0, 16)):
//   round 0: e = tid << 4 | i                          (bits 0-3 in registers)
//   round 1: e = (tid >> 4) << 8 | i << 4 | (tid & 15)  (bits 4-7)
//   round 2: e = i << 8 | tid                          (bits 8-11)
// Shared memory is addressed through swz(e), which XORs index bits 4-7 and
// 8-11 into bits 0-3.  Every round's stores and loads, the XOR-shifted
// partner reads (e ^ x) and the strided staging of the second pass are then
// spread over distinct banks for 8- and 16-byte elements.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sre {
namespace dev {

template <typename R> struct V2;
template <> struct V2<float> { using T = float2; };
template <> struct V2<double> { using T = double2; };
template <typename R> using v2_t = typename V2<R>::T;

__device__ __forceinline__ int swz(int e) { return (e & ~15) | ((e ^ (e >> 4) ^ (e >> 8)) & 15); }

template <int K> __device__ __forceinline__ int elem(int tid, int i);
template <> __device__ __forceinline__ int elem<0>(int tid, int i) { return (tid << 4) | i; }
template <> __device__ __forceinline__ int elem<1>(int tid, int i) {
    return ((tid >> 4) << 8) | (i << 4) | (tid & 15);
}
template <> __device__ __forceinline__ int elem<2>(int tid, int i) { return (i << 8) | tid; }

// Butterflies over register bits j in [0, 4) whose tile bit 4K + j < NB.
template <int K, int NB, typename R>
__device__ __forceinline__ void reg_stages(R (&re)[16], R (&im)[16]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (4 * K + j < NB) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                if (!(i & (1 << j))) {
                    const int p = i | (1 << j);
                    const R ar = re[i], ai = im[i], br = re[p], bi = im[p];
                    re[i] = ar + br;
                    im[i] = ai + bi;
                    re[p] = ar - br;
                    im[p] = ai - bi;
                }
            }
        }
    }
}

// Move the tile from round-KA layout to round-KB layout through `buf`.
// Moves between rounds 0 and 1 exchange register bits with thread bits 0-3,
// i.e. data moves only inside groups of 16 threads of one warp and each warp
// touches only its own 512-entry part of the buffer: they are ordered with
// __syncwarp (WARP = true).  Moves between rounds 1 and 2 exchange with
// thread bits 4-7 (across warps) and need a CTA barrier; their buffer must
// not be the one the previous tile's cross-warp move read (callers
// alternate two buffers).
template <int KA, int KB, bool WARP, typename R>
__device__ __forceinline__ void relayout(R (&re)[16], R (&im)[16], v2_t<R> *buf, int tid) {
    if (WARP) __syncwarp();
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        v2_t<R> v;
        v.x = re[i];
        v.y = im[i];
        buf[swz(elem<KA>(tid, i))] = v;
    }
    if (WARP)
        __syncwarp();
    else
        __syncthreads();
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const v2_t<R> v = buf[swz(elem<KB>(tid, i))];
        re[i] = v.x;
        im[i] = v.y;
    }
}

// Transform over tile bits [0, NB), 0 <= NB <= 12, bits 0-3 first.  Input in
// round-0 layout; output in round-(max(NB-1,0)/4) layout.  bufA serves the
// warp-local round 0 -> 1 move (consecutive calls may share it); bufB the
// CTA-wide round 1 -> 2 move (NB > 8): consecutive calls must alternate bufB
// between two buffers.
template <int NB, typename R>
__device__ __forceinline__ void tile_fwht(R (&re)[16], R (&im)[16], v2_t<R> *bufA,
                                          v2_t<R> *bufB, int tid) {
    static_assert(NB >= 0 && NB <= 12, "tile transform covers 0..12 bits");
    reg_stages<0, NB>(re, im);
    if constexpr (NB > 4) {
        relayout<0, 1, true>(re, im, bufA, tid);
        reg_stages<1, NB>(re, im);
    }
    if constexpr (NB > 8) {
        relayout<1, 2, false>(re, im, bufB, tid);
        reg_stages<2, NB>(re, im);
    }
}

// Full 12-bit transform, bits 8-11 first: input in round-2 layout (thread
// tid holds e = i << 8 | tid, so loads of consecutive threads are
// contiguous), output in round-0 layout.  One CTA-wide move (bufB, to be
// alternated between consecutive calls) and one warp-local move (bufA).
template <typename R>
__device__ __forceinline__ void tile_fwht12_rev(R (&re)[16], R (&im)[16], v2_t<R> *bufA,
                                                v2_t<R> *bufB, int tid) {
    reg_stages<2, 12>(re, im);
    relayout<2, 1, false>(re, im, bufB, tid);
    reg_stages<1, 12>(re, im);
    relayout<1, 0, true>(re, im, bufA, tid);
    reg_stages<0, 12>(re, im);
}

template <int NB> struct FinalRound { static constexpr int value = (NB - 1) / 4; };

// sum_i (Re F_i)^4 + (Im F_i)^4 over the thread's 16 entries, in R.
template <typename R>
__device__ __forceinline__ R sum_re4_im4(const R (&re)[16], const R (&im)[16]) {
    R s = R(0);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const R a = re[i] * re[i], b = im[i] * im[i];
        s += a * a + b * b;
    }
    return s;
}

// sum_i |F_i|^4 over the thread's 16 entries, in R.
template <typename R>
__device__ __forceinline__ R sum_abs4(const R (&re)[16], const R (&im)[16]) {
    R s = R(0);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const R m = re[i] * re[i] + im[i] * im[i];
        s += m * m;
    }
    return s;
}

// Load one complex amplitude of input type In (float2 / double2) as R.
template <typename R, typename In>
__device__ __forceinline__ void load_amp(const In *p, uint64_t idx, R &re, R &im) {
    const In v = __ldg(p + idx);
    re = (R)v.x;
    im = (R)v.y;
}

// Deterministic block-wide FP64 sum (fixed tree); result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double *red /* kThreads/32 */) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    }
    return s;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

}  // namespace dev
}  // namespace sre
