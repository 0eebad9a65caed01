// sre_tile.cuh -- in-CTA Walsh-Hadamard machinery on a tile of 2^12 complex
// entries held by 256 threads (16 entries each, i.e. 4 "register bits").
//
// The transform is the unnormalised WHT of the supplement's FWHT section:
// stage b maps each pair (a, c) of entries whose indices differ only in bit b
// to (a + c, a - c).  Stages commute, so the 12 bits are done in three rounds
// of four: a round does the butterflies over four index bits entirely in
// registers; between rounds the tile is rewritten through shared memory so
// that the next four bits become the register bits.
//
// Round layouts (tid in [0, 256), register slot i in [0, 16)):
//   round 0: e = tid << 4 | i                          (bits 0-3 in registers)
//   round 1: e = (tid >> 4) << 8 | i << 4 | (tid & 15)  (bits 4-7)
//   round 2: e = i << 8 | tid                          (bits 8-11)
// Shared memory stores entry e at pad(e) = e + (e >> 4): one spare slot per
// 16 entries.  Every round's stores and loads, and the XOR-shifted partner
// reads of the single-tile kernel, then hit distinct banks for 8- and
// 16-byte elements, and the address of slot i is the thread's base plus a
// compile-time offset.
//
// FP32 complex values live in one 64-bit register pair and are combined with
// the packed add/sub/mul/fma.rn.f32x2 instructions of sm_100+ (two IEEE
// round-to-nearest FP32 operations per instruction: the same results as
// scalar FP32 at half the instruction count).  FP64 values use double2.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sre {
namespace dev {

template <typename R> struct V2;
template <> struct V2<float> { using T = float2; };
template <> struct V2<double> { using T = double2; };
template <typename R> using v2_t = typename V2<R>::T;

constexpr int kTileSlots = 4096 + 256;  // padded shared-memory tile
__host__ __device__ constexpr int pad(int e) { return e + (e >> 4); }

// ------------------------------------------------------------ complex ops
template <typename R> struct Cx;

template <> struct Cx<float> {
    using T = unsigned long long;  // (re, im) packed: re in the low half
    static __device__ __forceinline__ T pack(float re, float im) {
        T d;
        asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(re), "f"(im));
        return d;
    }
    static __device__ __forceinline__ void unpack(T v, float &re, float &im) {
        asm("mov.b64 {%0, %1}, %2;" : "=f"(re), "=f"(im) : "l"(v));
    }
    static __device__ __forceinline__ T add(T a, T b) {
        T d;
        asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
        return d;
    }
    static __device__ __forceinline__ T sub(T a, T b) {
        T d;
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
        return d;
    }
    static __device__ __forceinline__ T mul(T a, T b) {
        T d;
        asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
        return d;
    }
    static __device__ __forceinline__ T fma(T a, T b, T c) {
        T d;
        asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
        return d;
    }
    static __device__ __forceinline__ T zero() { return 0ull; }
    static __device__ __forceinline__ T from(float2 v) { return pack(v.x, v.y); }
    static __device__ __forceinline__ float2 to(T v) {
        float2 r;
        unpack(v, r.x, r.y);
        return r;
    }
};

template <> struct Cx<double> {
    using T = double2;
    static __device__ __forceinline__ T pack(double re, double im) { return make_double2(re, im); }
    static __device__ __forceinline__ void unpack(T v, double &re, double &im) {
        re = v.x;
        im = v.y;
    }
    static __device__ __forceinline__ T add(T a, T b) { return make_double2(a.x + b.x, a.y + b.y); }
    static __device__ __forceinline__ T sub(T a, T b) { return make_double2(a.x - b.x, a.y - b.y); }
    static __device__ __forceinline__ T mul(T a, T b) { return make_double2(a.x * b.x, a.y * b.y); }
    static __device__ __forceinline__ T fma(T a, T b, T c) {
        return make_double2(__fma_rn(a.x, b.x, c.x), __fma_rn(a.y, b.y, c.y));
    }
    static __device__ __forceinline__ T zero() { return make_double2(0.0, 0.0); }
    static __device__ __forceinline__ T from(double2 v) { return v; }
    static __device__ __forceinline__ double2 to(T v) { return v; }
};

template <typename R> using cx_t = typename Cx<R>::T;

// conj(b) * a for scalar factors, packed.
template <typename R>
__device__ __forceinline__ cx_t<R> conj_mul(R br, R bi, R ar, R ai) {
    return Cx<R>::pack(br * ar + bi * ai, br * ai - bi * ar);
}

template <int K> __device__ __forceinline__ int elem(int tid, int i);
template <> __device__ __forceinline__ int elem<0>(int tid, int i) { return (tid << 4) | i; }
template <> __device__ __forceinline__ int elem<1>(int tid, int i) {
    return ((tid >> 4) << 8) | (i << 4) | (tid & 15);
}
template <> __device__ __forceinline__ int elem<2>(int tid, int i) { return (i << 8) | tid; }

// Butterflies over register bits j in [0, 4) whose tile bit 4K + j < NB.
template <int K, int NB, typename R>
__device__ __forceinline__ void reg_stages(cx_t<R> (&v)[16]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (4 * K + j < NB) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                if (!(i & (1 << j))) {
                    const int p = i | (1 << j);
                    const cx_t<R> a = v[i], b = v[p];
                    v[i] = Cx<R>::add(a, b);
                    v[p] = Cx<R>::sub(a, b);
                }
            }
        }
    }
}

// Move the tile from round-KA layout to round-KB layout through `buf`
// (kTileSlots entries).  Moves between rounds 0 and 1 exchange register bits
// with thread bits 0-3, i.e. data moves only inside groups of 16 threads of
// one warp and each warp touches only its own part of the buffer: they are
// ordered with __syncwarp (WARP = true).  Moves between rounds 1 and 2
// exchange with thread bits 4-7 (across warps) and need a CTA barrier; their
// buffer must not be the one the previous tile's cross-warp move read
// (callers alternate two buffers).
template <int KA, int KB, bool WARP, typename R>
__device__ __forceinline__ void relayout(cx_t<R> (&v)[16], v2_t<R> *buf, int tid) {
    if (WARP) __syncwarp();
#pragma unroll
    for (int i = 0; i < 16; ++i) buf[pad(elem<KA>(tid, i))] = Cx<R>::to(v[i]);
    if (WARP)
        __syncwarp();
    else
        __syncthreads();
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = Cx<R>::from(buf[pad(elem<KB>(tid, i))]);
}

// Transform over tile bits [0, NB), 0 <= NB <= 12, bits 0-3 first.  Input in
// round-0 layout; output in round-(max(NB-1,0)/4) layout.  bufA serves the
// warp-local round 0 -> 1 move (consecutive calls may share it); bufB the
// CTA-wide round 1 -> 2 move (NB > 8): consecutive calls must alternate bufB
// between two buffers.
template <int NB, typename R>
__device__ __forceinline__ void tile_fwht(cx_t<R> (&v)[16], v2_t<R> *bufA, v2_t<R> *bufB,
                                          int tid) {
    static_assert(NB >= 0 && NB <= 12, "tile transform covers 0..12 bits");
    reg_stages<0, NB, R>(v);
    if constexpr (NB > 4) {
        relayout<0, 1, true, R>(v, bufA, tid);
        reg_stages<1, NB, R>(v);
    }
    if constexpr (NB > 8) {
        relayout<1, 2, false, R>(v, bufB, tid);
        reg_stages<2, NB, R>(v);
    }
}

// Full 12-bit transform, bits 8-11 first: input in round-2 layout (thread
// tid holds e = i << 8 | tid, so loads of consecutive threads are
// contiguous), output in round-0 layout.  One CTA-wide move (bufB, to be
// alternated between consecutive calls) and one warp-local move (bufA).
template <typename R>
__device__ __forceinline__ void tile_fwht12_rev(cx_t<R> (&v)[16], v2_t<R> *bufA, v2_t<R> *bufB,
                                                int tid) {
    reg_stages<2, 12, R>(v);
    relayout<2, 1, false, R>(v, bufB, tid);
    reg_stages<1, 12, R>(v);
    relayout<1, 0, true, R>(v, bufA, tid);
    reg_stages<0, 12, R>(v);
}

// sum_i |F_i|^4 over the thread's 16 entries, in R.
template <typename R>
__device__ __forceinline__ R sum_abs4(const cx_t<R> (&v)[16]) {
    R s = R(0);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        R re, im;
        Cx<R>::unpack(Cx<R>::mul(v[i], v[i]), re, im);
        const R m = re + im;
        s += m * m;
    }
    return s;
}

// sum_i (Re F_i)^4 + (Im F_i)^4 over the thread's 16 entries, in R.
template <typename R>
__device__ __forceinline__ R sum_re4_im4(const cx_t<R> (&v)[16]) {
    cx_t<R> acc = Cx<R>::zero();
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const cx_t<R> sq = Cx<R>::mul(v[i], v[i]);
        acc = Cx<R>::fma(sq, sq, acc);
    }
    R a, b;
    Cx<R>::unpack(acc, a, b);
    return a + b;
}

// Order alpha of Eq. (sre): sum_i (|F_i|^2)^alpha over the thread's 16
// entries (integer alpha >= 2, a product of alpha factors), in R.
template <typename R>
__device__ __forceinline__ R sum_abs_pow(const cx_t<R> (&v)[16], int alpha) {
    R s = R(0);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        R re, im;
        Cx<R>::unpack(Cx<R>::mul(v[i], v[i]), re, im);
        const R m = re + im;
        R p = m;
        for (int k = 1; k < alpha; ++k) p *= m;
        s += p;
    }
    return s;
}

// Order alpha, halved shifts: sum_i (Re F_i)^(2 alpha) + (Im F_i)^(2 alpha).
template <typename R>
__device__ __forceinline__ R sum_re_im_pow(const cx_t<R> (&v)[16], int alpha) {
    cx_t<R> acc = Cx<R>::zero();
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const cx_t<R> sq = Cx<R>::mul(v[i], v[i]);
        cx_t<R> p = sq;
        for (int k = 1; k < alpha; ++k) p = Cx<R>::mul(p, sq);
        acc = Cx<R>::add(acc, p);
    }
    R a, b;
    Cx<R>::unpack(acc, a, b);
    return a + b;
}

// Orders 3 and 4 with the power unrolled at compile time (same products in
// the same order as the loops above).
template <typename R, int A>
__device__ __forceinline__ R sum_abs_pow_c(const cx_t<R> (&v)[16]) {
    R s = R(0);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        R re, im;
        Cx<R>::unpack(Cx<R>::mul(v[i], v[i]), re, im);
        const R m = re + im;
        R p = m;
#pragma unroll
        for (int k = 1; k < A; ++k) p *= m;
        s += p;
    }
    return s;
}

template <typename R, int A>
__device__ __forceinline__ R sum_re_im_pow_c(const cx_t<R> (&v)[16]) {
    cx_t<R> acc = Cx<R>::zero();
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const cx_t<R> sq = Cx<R>::mul(v[i], v[i]);
        cx_t<R> p = sq;
#pragma unroll
        for (int k = 1; k < A; ++k) p = Cx<R>::mul(p, sq);
        acc = Cx<R>::add(acc, p);
    }
    R a, b;
    Cx<R>::unpack(acc, a, b);
    return a + b;
}

// The thread's share of the order-alpha sum (HALF: the halved-shift form);
// order 2 takes the M2 reductions above unchanged.
template <typename R, bool HALF>
__device__ __forceinline__ R sum_order(const cx_t<R> (&v)[16], int alpha) {
    switch (alpha) {
        case 2: return HALF ? sum_re4_im4<R>(v) : sum_abs4<R>(v);
        case 3: return HALF ? sum_re_im_pow_c<R, 3>(v) : sum_abs_pow_c<R, 3>(v);
        case 4: return HALF ? sum_re_im_pow_c<R, 4>(v) : sum_abs_pow_c<R, 4>(v);
        default: return HALF ? sum_re_im_pow<R>(v, alpha) : sum_abs_pow<R>(v, alpha);
    }
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

// Drop a 128-byte L2 line without writing it back (its contents become
// undefined).  Used on inter-pass scratch once every reader is done with it.
__device__ __forceinline__ void discard_l2_line(const void *p) {
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

}  // namespace dev
}  // namespace sre
