// sre_stage.cuh -- pass-2 tiles of the two-pass kernel staged through the
// Tensor Memory Accelerator (FP32, 5 <= H2 <= 8).
//
// A pass-2 tile of one shift is the 2^H2 x 2^(12 - H2) block of inter-pass
// scratch formed by rows t'_h (the H2 transform bits still to do, one row per
// 4096-entry block) and one z-block of columns.  Its rows lie 32 KB apart, so
// per-thread loads touch one 32-byte sector in each of many L2 lines and the
// warp waits a full L2 round trip per tile.  Here one thread instead issues
// 2^(8 - H2) two-dimensional TMA copies per tile (boxes of 16 columns x 2^H2
// rows, 128-byte rows, 128-byte swizzle) into a shared-memory stage; two
// stages alternate, so the copy of tile g + 2 is in flight while tile g is
// transformed.
//
// Thread layouts over a warp's 512 entries (e9 = 9-bit index: row bits
// r0..r_{H2-1} low, then the low column bits; the warp index supplies the
// three high column bits):
//   layout A (read from the stage): lane bits 0-2 = r0-r2, lane bit 3 = the
//     first column bit, lane bit 4 = the second column bit (r7 for H2 = 8),
//     registers = the remaining four bits in increasing order (r3.. first);
//   layout B (after one warp-local exchange through shared memory):
//     registers = r0, r1, r2 and r7 (H2 = 8) or the top bit (H2 < 8), lanes =
//     the remaining five bits.
// Layout A's register row bits are transformed first, layout B's after the
// exchange: every row bit exactly once, i.e. the 2^H2-point WHT of each
// column.  The 128-byte swizzle stores the 16-byte chunk k of row r at chunk
// k ^ (r mod 8); with lane bits 0-2 = r mod 8 a warp's stage reads, and the
// exchange index q below with one spare slot per 16 entries, give at most
// two lanes per 8-byte bank slot (conflict-free for 8-byte accesses).
// Every per-thread address is a lane term combined with a compile-time
// register term: XOR for the stage (disjoint bit fields; the swizzle XOR acts
// on lane bits only), addition for the padded exchange (disjoint bits of q).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sre_async.cuh"
#include "sre_tile.cuh"

namespace sre {
namespace dev {

constexpr int kStageBytes = 32768;  // one pass-2 tile: 4096 FP32 complex

template <int H2>
struct P2Stage {
    static_assert(H2 >= 5 && H2 <= 8, "staged pass 2 covers 5..8 transform bits");
    static constexpr int kA3 = H2;                    // layout A, lane bit 3
    static constexpr int kA4 = H2 <= 7 ? H2 + 1 : 7;  // layout A, lane bit 4
    static constexpr int kB3 = H2 == 8 ? 7 : 8;       // layout B, register bit 3

    __host__ __device__ static constexpr int laneA(int k) { return k < 3 ? k : (k == 3 ? kA3 : kA4); }
    __host__ __device__ static constexpr int regA(int k) {
        int n = 0;
        for (int b = 3; b < 9; ++b) {
            if (b == kA3 || b == kA4) continue;
            if (n == k) return b;
            ++n;
        }
        return -1;
    }
    __host__ __device__ static constexpr int regB(int k) { return k < 3 ? k : kB3; }
    __host__ __device__ static constexpr int laneB(int k) {
        int n = 0;
        for (int b = 3; b < 9; ++b) {
            if (b == kB3) continue;
            if (n == k) return b;
            ++n;
        }
        return -1;
    }
    // position of e9 bit b in the exchange index q: bits 0-3 = r0, r1, r2 and
    // layout A's lane bit 3; bits 4-7 = layout B's other lane bits in order;
    // bit 8 = layout B's register bit 3
    __host__ __device__ static constexpr int qpos(int b) {
        if (b < 3) return b;
        if (b == kA3) return 3;
        if (b == kB3) return 8;
        int n = 4;
        for (int bb = 3; bb < 9; ++bb) {
            if (bb == kA3 || bb == kB3) continue;
            if (bb == b) return n;
            ++n;
        }
        return -1;
    }
    __host__ __device__ static constexpr int q_of(int e9) {
        int q = 0;
        for (int b = 0; b < 9; ++b)
            if ((e9 >> b) & 1) q |= 1 << qpos(b);
        return q;
    }
    __host__ __device__ static constexpr int e9_laneA(int lane) {
        int e = 0;
        for (int k = 0; k < 5; ++k) e |= ((lane >> k) & 1) << laneA(k);
        return e;
    }
    __host__ __device__ static constexpr int e9_regA(int i) {
        int e = 0;
        for (int k = 0; k < 4; ++k) e |= ((i >> k) & 1) << regA(k);
        return e;
    }
    __host__ __device__ static constexpr int e9_laneB(int lane) {
        int e = 0;
        for (int k = 0; k < 5; ++k) e |= ((lane >> k) & 1) << laneB(k);
        return e;
    }
    __host__ __device__ static constexpr int e9_regB(int i) {
        int e = 0;
        for (int k = 0; k < 4; ++k) e |= ((i >> k) & 1) << regB(k);
        return e;
    }
    // byte offset in the stage of warp w's entry e9 (boxes of 16 columns)
    __host__ __device__ static constexpr uint32_t stage_off(int e9, int w) {
        const int r = e9 & ((1 << H2) - 1);
        const int c = (w << (9 - H2)) | (e9 >> H2);
        const int b = c >> 4, cc = c & 15;
        return (uint32_t)(b * (128 << H2) + r * 128 + ((((cc >> 1) ^ (r & 7))) << 4) + (cc & 1) * 8);
    }
    // register bits whose e9 bit is a row bit: butterflies of layout A / B
    __host__ __device__ static constexpr int maskA() {
        int m = 0;
        for (int k = 0; k < 4; ++k)
            if (regA(k) < H2) m |= 1 << k;
        return m;
    }
    __host__ __device__ static constexpr int maskB() {
        int m = 0;
        for (int k = 0; k < 4; ++k)
            if (regB(k) < H2) m |= 1 << k;
        return m;
    }
};

// Butterflies over the register bits set in MASK.
template <int MASK, typename R>
__device__ __forceinline__ void reg_stages_mask(cx_t<R> (&v)[16]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (MASK & (1 << j)) {
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

// Per-thread lane terms of the stage read and of the exchange (computed once).
struct P2Lane {
    uint32_t stage;  // byte offset, combined by XOR with the register term
    int xa, xb;      // exchange slots (padded), combined by addition
};

template <int H2>
__device__ __forceinline__ P2Lane p2_lane(int lane, int warp) {
    using L = P2Stage<H2>;
    P2Lane p;
    p.stage = L::stage_off(L::e9_laneA(lane), warp);
    p.xa = warp * 544 + pad(L::q_of(L::e9_laneA(lane)));
    p.xb = warp * 544 + pad(L::q_of(L::e9_laneB(lane)));
    return p;
}

// Transform one staged tile and return this thread's share of the quartic
// sum: sum (Re W)^4 + (Im W)^4 (HALF) or sum |W|^4 (exponents 2 alpha in place
// of 4 at Renyi order alpha).  xbuf is the warp-local
// exchange buffer (kTileSlots entries, warp w uses [544 w, 544 w + 544)).
template <int H2, bool HALF>
__device__ __forceinline__ float p2_tile(const unsigned char *stage, float2 *xbuf, const P2Lane &p,
                                         int alpha) {
    using L = P2Stage<H2>;
    using T = cx_t<float>;
    T v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i)
        v[i] = *reinterpret_cast<const T *>(stage + (p.stage ^ L::stage_off(L::e9_regA(i), 0)));
    reg_stages_mask<L::maskA(), float>(v);
    T *xb = reinterpret_cast<T *>(xbuf);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 16; ++i) xb[p.xa + pad(L::q_of(L::e9_regA(i)))] = v[i];
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = xb[p.xb + pad(L::q_of(L::e9_regB(i)))];
    reg_stages_mask<L::maskB(), float>(v);
    return sum_order<float, HALF>(v, alpha);
}

}  // namespace dev
}  // namespace sre
