// sre_mid.cu -- single-pass kernel for shifts whose transform spans one,
// two or (FP32) four 4096-entry blocks: the halved shifts (x >= 4096) of
// N = 13, 14 and 15 and the full shifts (x < 4096) of N = 13 and 14.
//
// For such a shift the whole transform stays inside one CTA, so the two-pass
// machinery (scratch ring, lagged work items, inter-CTA waits) is not needed.
// A CTA takes whole shifts, grid-strided over (state, shift): it forms the
// XOR-shifted products of each block, applies the 12-bit tile transform
// (sre_tile.cuh, bits 8-11 first), parks every block but the last in shared
// memory at positions only its own thread reads back (i << 8 | tid, no bank
// conflicts), then applies the butterflies across the blocks (transform bits
// 12 and up).  Four blocks need 168 KB of shared memory: one CTA per SM.  The
// shift's quartic sum (or order-alpha sum; halved shifts with the factor
// 2^(2 alpha)) is summed per thread in R and across the CTA in FP64 in a
// fixed tree: one partial per shift, the same in a single or a batched
// launch.
//
// Halving (x >= 4096, pivot j = highest set bit of x, jh = j - 12): the
// restricted transform runs over t with t_j = 0; block t'_h of it is block
// t_h = t'_h with a zero inserted at bit jh.  For N = 13 there is one block
// (jh = 0, t_h = 0); for N = 14, t'_h = 0, 1; for N = 15, t'_h = 0..3.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "sre_internal.h"
#include "sre_tile.cuh"

namespace sre {
using namespace dev;

namespace {

template <typename R, bool HALF, int NB>
__global__ void __launch_bounds__(kThreads, (sizeof(R) == 4 && NB <= 2) ? 2 : 1)
    k_mid(const v2_t<R> *__restrict__ psi0, const void *const *__restrict__ psis, long long shifts_per_state,
          uint64_t x_begin, long long n, int alpha, double *__restrict__ part, double *__restrict__ per_x) {
    static_assert(NB == 1 || NB == 2 || NB == 4, "one, two or four blocks per shift");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using V = v2_t<R>;
    V *bufA = reinterpret_cast<V *>(smem_raw);  // warp-local moves
    V *bufB = bufA + kTileSlots;                 // CTA-wide moves
    V *park = bufB + kTileSlots;                 // blocks 0 .. NB-2, 4096 entries each
    __shared__ double red[kThreads / 32];
    const int tid = threadIdx.x;
    const double hfac = HALF ? (double)(1ull << (2 * alpha)) : 1.0;

    for (long long g = blockIdx.x; g < n; g += gridDim.x) {
        const long long sidx = psis ? g / shifts_per_state : 0;
        const V *psi = psis ? reinterpret_cast<const V *>(psis[sidx]) : psi0;
        const uint64_t x = x_begin + (uint64_t)(g - sidx * shifts_per_state);
        const uint64_t xh = x >> kTileBits;
        const int xlow = (int)(x & (kTile - 1));
        const int q = xlow >> 8;
        const int jh = HALF ? (63 - __clzll((long long)x)) - kTileBits : 0;
        cx_t<R> v[16];
#pragma unroll
        for (int tp = 0; tp < NB; ++tp) {
            const int th = HALF ? (((tp >> jh) << (jh + 1)) | (tp & ((1 << jh) - 1))) : tp;
            const V *pa = psi + ((uint64_t)th << kTileBits) + tid;
            const V *pb = psi + (((uint64_t)th ^ xh) << kTileBits) + (tid ^ (xlow & 255));
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const V a = __ldg(pa + (i << 8));
                const V b = __ldg(pb + ((i ^ q) << 8));
                v[i] = conj_mul<R>(b.x, b.y, a.x, a.y);  // conj(phi_{t^x}) * phi_t
            }
            // one CTA-wide buffer: the barrier keeps the previous block's (or
            // shift's) readers ahead of this block's writers
            __syncthreads();
            tile_fwht12_rev<R>(v, bufA, bufB, tid);
            if (tp + 1 < NB) {
#pragma unroll
                for (int i = 0; i < 16; ++i) park[(tp << kTileBits) + ((i << 8) | tid)] = Cx<R>::to(v[i]);
            }
        }
        R s;
        if constexpr (NB == 2) {
            cx_t<R> w[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const cx_t<R> a = Cx<R>::from(park[(i << 8) | tid]);
                w[i] = Cx<R>::sub(a, v[i]);
                v[i] = Cx<R>::add(a, v[i]);
            }
            s = sum_order<R, HALF>(v, alpha) + sum_order<R, HALF>(w, alpha);
        } else if constexpr (NB == 4) {
            // 2-bit transform over the block index: pairs (0,1), (2,3), then (0,2), (1,3)
            cx_t<R> c1[16], c2[16], c3[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const cx_t<R> a0 = Cx<R>::from(park[(i << 8) | tid]);
                const cx_t<R> a1 = Cx<R>::from(park[(1 << kTileBits) + ((i << 8) | tid)]);
                const cx_t<R> a2 = Cx<R>::from(park[(2 << kTileBits) + ((i << 8) | tid)]);
                const cx_t<R> b0 = Cx<R>::add(a0, a1), b1 = Cx<R>::sub(a0, a1);
                const cx_t<R> b2 = Cx<R>::add(a2, v[i]), b3 = Cx<R>::sub(a2, v[i]);
                v[i] = Cx<R>::add(b0, b2);
                c2[i] = Cx<R>::sub(b0, b2);
                c1[i] = Cx<R>::add(b1, b3);
                c3[i] = Cx<R>::sub(b1, b3);
            }
            s = sum_order<R, HALF>(v, alpha) + sum_order<R, HALF>(c1, alpha) + sum_order<R, HALF>(c2, alpha) +
                sum_order<R, HALF>(c3, alpha);
        } else {
            s = sum_order<R, HALF>(v, alpha);
        }
        const double tot = block_sum(hfac * (double)s, red);
        if (tid == 0) {
            part[g] = tot;
            if (per_x) per_x[g] = tot;
        }
    }
}

template <typename R, bool HALF, int NB>
cudaError_t launch_mid_t(const void *psi, const void *const *psis, int nstates, long long sps, uint64_t x_begin,
                         int alpha, double *part, double *per_x, const DeviceInfo &dev, cudaStream_t st) {
    const size_t smem = ((size_t)2 * kTileSlots + (size_t)(NB > 1 ? NB - 1 : 0) * kTile) * sizeof(v2_t<R>);
    auto kern = k_mid<R, HALF, NB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long n = sps * (long long)nstates;
    if (n <= 0) return cudaSuccess;
    const int occ = (sizeof(R) == 4 && NB <= 2) ? 2 : 1;
    const int grid = (int)std::min<long long>(n, (long long)dev.sms * occ);
    kern<<<grid, kThreads, smem, st>>>(reinterpret_cast<const v2_t<R> *>(psi), psis, sps, x_begin, n, alpha,
                                       part, per_x);
    return cudaGetLastError();
}

}  // namespace

bool mid_applies(int N, int half, int elem_bytes) {
    const int bits = N - (half ? 1 : 0);
    const int max_bits = elem_bytes == 8 ? kTileBits + 2 : kTileBits + 1;  // four blocks: FP32 only
    return N > kTileBits && bits >= kTileBits && bits <= max_bits;
}

template <typename R>
cudaError_t launch_mid(int N, int half, const void *psi, const void *const *psis, int nstates, long long sps,
                       uint64_t x_begin, int alpha, double *part, double *per_x, const DeviceInfo &dev,
                       cudaStream_t st) {
    const int nb = 1 << (N - (half ? 1 : 0) - kTileBits);
    if (nb == 4) {
        if constexpr (sizeof(R) == 4) {
            return half ? launch_mid_t<R, true, 4>(psi, psis, nstates, sps, x_begin, alpha, part, per_x, dev, st)
                        : launch_mid_t<R, false, 4>(psi, psis, nstates, sps, x_begin, alpha, part, per_x, dev, st);
        }
        return cudaErrorInvalidValue;
    }
    if (half)
        return nb == 1 ? launch_mid_t<R, true, 1>(psi, psis, nstates, sps, x_begin, alpha, part, per_x, dev, st)
                       : launch_mid_t<R, true, 2>(psi, psis, nstates, sps, x_begin, alpha, part, per_x, dev, st);
    return nb == 1 ? launch_mid_t<R, false, 1>(psi, psis, nstates, sps, x_begin, alpha, part, per_x, dev, st)
                   : launch_mid_t<R, false, 2>(psi, psis, nstates, sps, x_begin, alpha, part, per_x, dev, st);
}

template cudaError_t launch_mid<float>(int, int, const void *, const void *const *, int, long long, uint64_t, int,
                                       double *, double *, const DeviceInfo &, cudaStream_t);
template cudaError_t launch_mid<double>(int, int, const void *, const void *const *, int, long long, uint64_t,
                                        int, double *, double *, const DeviceInfo &, cudaStream_t);

}  // namespace sre
