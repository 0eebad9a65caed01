// sre_large.cuh -- the persistent two-pass CUDA-core kernel of libsre
// (N > 12), and the work-item order and bounded waits it shares with the
// tensor-core kernel of sre_tc.cu.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sre_internal.h"
#include "sre_async.cuh"
#include "sre_stage.cuh"
#include "sre_tile.cuh"

namespace sre {
using namespace dev;

// -------------------------------------------------------- N > 12: k_large

// Work of one evaluation over shifts [x_begin, x_end), N > 12.
//
// Shifts are grouped in chunks of C = 2^C_log consecutive values (aligned, so
// a chunk shares x_h = x >> 12 and, for halved chunks, the pivot bit).  A
// chunk owns one slot of a ring of R scratch slots.  Its work items:
//   pass 1, P1 = 2^(h2 - B1_log) items of 2^B1_log consecutive blocks t'_h,
//           each for every shift of the chunk -- the XOR-shifted products of
//           one 2^12 block of t, the 12 low transform bits, written to
//           scratch[slot][shift][t'_h][z_l];
//   pass 2, P2 items of 2^G2_log tiles: for one shift and a range of z-blocks,
//           the 2^h2 blocks t'_h of each z-block are read back, the h2 high
//           bits are transformed and |A|^4 is reduced, one FP64 partial per
//           warp (item_part[(slot, item, warp)]).
// Completion is counted per warp (P1 * 8 arrivals finish pass 1 of a chunk,
// P2 * 8 pass 2), so no CTA barrier is needed at item boundaries; the warp
// that completes a chunk's pass 2 sums its partials in fixed order, drops
// the chunk's scratch lines from L2 and releases the ring slot.
// Items are claimed from one counter in a lagged order -- step s holds the
// pass-1 items of chunk s and the pass-2 items of chunk s - D -- so pass 2
// rarely waits for pass 1; pass 1 of chunk c waits for slot c % R to be
// released by chunk c - R (D < R keeps this deadlock-free: every item waits
// only on items claimed before it).
//
// Halving (half = 1, shifts x >= 4096).  With pivot j = the highest set bit
// of x, g_x(t ^ x) = conj(g_x(t)) pairs every t with t_j = 1 to one with
// t_j = 0, and sum_z |A_x(z)|^4 = 16 sum_{z'} [(Re W(z'))^4 + (Im W(z'))^4]
// where W is the (N-1)-bit transform of g_x restricted to t_j = 0 (A is
// 2 Re W or 2i Im W, so at Renyi order alpha the exponents are 2 alpha and
// the factor 2^(2 alpha)).  Since
// j >= 12, the restriction removes one high bit: block t'_h maps to
// t_h = t'_h with a zero inserted at bit j - 12, and h2 = N - 13.
//
// FP32 launches with 5 <= h2 <= 8 stage pass-2 tiles through TMA
// (sre_stage.cuh): tmap then describes the scratch ring as a 2-D FP32 array
// of 8192 columns (4096 complex per block t'_h) by R * C * 2^h2 rows.  The
// tensor-core kernel (sre_tc.cu) describes its 16-bit scratch planes there
// instead and reads its per-shift fixed-point scales from tc_e.
struct LargeArgs {
    CUtensorMap tmap;          // pass-2 staging (encode_p2_tmap / tc map), else unused
    const int *tc_e;           // tensor-core kernel: scale exponent per x >> 12
    const void *psi;           // the state (single-state launch)
    const void *const *psis;   // or: states of one batch class (device array)
    long long chunks_per_state;  // chunks of each state (batch class)
    int N, h2;                 // h2: pass-2 transform bits (N - 12, or N - 13 halved)
    int half;
    uint64_t x_begin, x_end;   // evaluated shift range
    uint64_t x0;               // x_begin rounded down to a chunk boundary
    int C_log, R, D, G2_log, B1_log;
    int stage1, stage2;        // staged copy paths enabled (LargeCfg)
    int alpha;                 // Renyi order (2: M2)
    long long n_chunks;
    int P1, P2;                // items per chunk in pass 1 / pass 2
    long long n_items;
    void *scratch;             // R * C * 2^(N - half) complex
    double *item_part;         // R * P2
    double *chunk_sum;         // n_chunks
    unsigned *done1, *done2, *freed;  // n_chunks each
    unsigned long long *work;
    double *per_x;             // optional, indexed by x - x_begin
    int *status;
    long long wait_ns;
};

// Thread 0 waits until *p >= target.  Bounded by wait_ns of %globaltimer and
// by an iteration cap; on expiry it records SRE_ETIMEDOUT and returns false.
// Returns false as well if another CTA already recorded an error.
static __device__ bool wait_counter(const unsigned *p, unsigned target, int *status, long long wait_ns) {
    const unsigned long long t0 = globaltimer_ns();
    for (unsigned it = 0; it < (1u << 30); ++it) {
        if (ld_acquire_u32(p) >= target) return true;
        if (*(volatile int *)status != 0) return false;
        if ((it & 31) == 31 && (long long)(globaltimer_ns() - t0) > wait_ns) break;
        __nanosleep(64);
    }
    atomicCAS(status, 0, (int)SRE_ETIMEDOUT);
    return false;
}

// item -> (chunk, index within its pass, pass) for the lagged order.
__device__ __forceinline__ void decode_item(const LargeArgs &a, long long item, long long &chunk,
                                            int &r, bool &pass1) {
    const long long D = a.D, P1 = a.P1, P2 = a.P2, n = a.n_chunks;
    if (item < D * P1) {
        chunk = item / P1;
        r = (int)(item - chunk * P1);
        pass1 = true;
        return;
    }
    item -= D * P1;
    const long long mid = (n - D) * (P1 + P2);
    if (item < mid) {
        const long long s = item / (P1 + P2);
        const int q = (int)(item - s * (P1 + P2));
        if (q < P1) {
            chunk = D + s;
            r = q;
            pass1 = true;
        } else {
            chunk = s;
            r = q - (int)P1;
            pass1 = false;
        }
        return;
    }
    item -= mid;
    const long long s = item / P2;
    chunk = n - D + s;
    r = (int)(item - s * P2);
    pass1 = false;
}

// Pass 2 of this instantiation stages its tiles through TMA.
template <typename R, int H2>
__host__ __device__ constexpr bool large_uses_tma() {
    return sizeof(R) == 4 && H2 >= 5 && H2 <= 8;
}

// Pass 1 of this instantiation can take its block pairs by bulk copy (FP32
// CUDA-core path; used at run time for one shift per chunk and 16-byte
// aligned states).
template <typename R>
__host__ __device__ constexpr bool large_stages_pass1() {
    return sizeof(R) == 4;
}

// Dynamic shared memory of k_large: three relayout buffers (the first two
// double as the TMA stages of pass 2, hence 1024-byte alignment).
template <typename R, int H2>
__host__ __device__ constexpr size_t large_smem_bytes() {
    return (size_t)3 * kTileSlots * sizeof(v2_t<R>) + (large_uses_tma<R, H2>() ? 1024 : 0);
}

// Host: encode LargeArgs::tmap for the launch's scratch ring.
cudaError_t encode_p2_tmap(LargeArgs &a);

template <typename R, int H2, bool HALF>
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? 2 : 1) k_large(const __grid_constant__ LargeArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using V = v2_t<R>;
    constexpr bool kTma = large_uses_tma<R, H2>();
    constexpr bool kStage1 = large_stages_pass1<R>();
    unsigned char *sbase = smem_raw;
    if constexpr (kTma) sbase += (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
    V *bufB = reinterpret_cast<V *>(sbase);  // round 1 -> 2 moves, alternating with
    V *bufC = bufB + kTileSlots;             //   bufC from tile to tile; pass-2 stages
    V *bufA = bufC + kTileSlots;             // warp-local moves
    __shared__ long long s_next[2];
    __shared__ int s_stop[2];
    // stage barriers: [0], [1] the pass-2 tile stages (kTma), [2] the pass-1
    // block pair (kStage1)
    __shared__ __align__(8) uint64_t s_mbar[3];
    unsigned tcount = 0;  // tiles that used a round 1 -> 2 move (uniform)
    uint32_t sphase = 0;  // parity of the next completion of each barrier
    uint32_t slost = 0;   // barriers whose completion wait expired

    const int tid = threadIdx.x;
    const int lgx = a.N - (HALF ? 1 : 0);        // log2 scratch entries per shift
    const int C = 1 << a.C_log;
    const V *psi0 = reinterpret_cast<const V *>(a.psi);
    V *scratch = reinterpret_cast<V *>(a.scratch);
    constexpr int zsub_bits = kTileBits - H2;     // z entries per block in pass 2
    const int ipx_log = H2 - a.G2_log;            // pass-2 items per shift (log2)
    // halved shifts: sum_z |A|^(2 alpha) = 2^(2 alpha) sum_z' [(Re W)^(2 alpha) +
    // (Im W)^(2 alpha)] (16 at alpha = 2)
    const double hfac = (double)(1ull << (2 * a.alpha));

    const int warp = tid >> 5, lane = tid & 31;
    constexpr int kWarps = kThreads / 32;
    // Item claims are prefetched one item ahead through a two-entry slot;
    // s_stop carries a recorded error so that the whole CTA stops together.
    if (tid == 0) {
        s_next[0] = (long long)atomicAdd(a.work, 1ull);
        s_stop[0] = 0;
        if constexpr (kTma || kStage1) {
            for (int k = 0; k < 3; ++k) mbar_init(smem_u32(&s_mbar[k]), 1);
        }
    }
    __syncthreads();
    for (int par = 0;; par ^= 1) {
        const long long item = s_next[par];
        if (item >= a.n_items || s_stop[par]) break;
        long long next = 0;
        if (tid == 0) next = (long long)atomicAdd(a.work, 1ull);
        long long c;
        int r;
        bool pass1;
        decode_item(a, item, c, r, pass1);
        const int slot = (int)(c % a.R);
        // batch class: chunk c belongs to state c / chunks_per_state
        long long cl = c;
        const V *psi = psi0;
        if (a.psis) {
            const long long sidx = c / a.chunks_per_state;
            cl = c - sidx * a.chunks_per_state;
            psi = reinterpret_cast<const V *>(a.psis[sidx]);
        }
        const uint64_t xc = a.x0 + ((uint64_t)cl << a.C_log);
        V *slot_base = scratch + (size_t)slot * ((size_t)C << lgx);

        if (pass1) {
            // ---------------- pass 1: blocks t'_h in [r 2^B1, (r+1) 2^B1) of
            // every shift in the chunk.  Each warp waits for the ring slot
            // itself (an expired wait records SRE_ETIMEDOUT; the CTA then
            // finishes this item on garbage and stops at the next claim).
            if (c >= a.R) {
                int ok = 1;
                if (lane == 0) ok = wait_counter(a.freed + (c - a.R), 1u, a.status, a.wait_ns);
                __syncwarp();
                (void)ok;
            }
            const uint64_t xh = xc >> kTileBits;
            const int xl0 = (int)(xc & (kTile - 1));
            const int jh = HALF ? (63 - __clzll((long long)xc)) - kTileBits : 0;
            if (kStage1 && a.stage1 && C == 1 && ((uintptr_t)psi & 15) == 0) {
                // One shift per chunk and a 16-byte aligned state: the block
                // t_h and its partner t_h ^ x_h arrive by two 32 KB bulk copies
                // in the two stage buffers.  The products overwrite the own
                // block in place (each thread rewrites only the entries it
                // read) and that buffer serves the CTA-wide move; once it has
                // been read back the next pair's copies are issued, so they
                // overlap the rest of the tile.
                if (xc >= a.x_begin && xc < a.x_end) {
                    const int nb = 1 << a.B1_log;
                    const uint32_t mb = smem_u32(&s_mbar[2]);
                    V *own = bufB;
                    const V *par = bufC;
                    auto issue_pair = [&](int kb) {
                        const int tp = (r << a.B1_log) + kb;
                        const int th = HALF ? (((tp >> jh) << (jh + 1)) | (tp & ((1 << jh) - 1))) : tp;
                        mbar_arrive_expect_tx(mb, 2u * kStageBytes);
                        bulk_load(smem_u32(own), psi + ((uint64_t)th << kTileBits), kStageBytes, mb);
                        bulk_load(smem_u32(par), psi + (((uint64_t)th ^ xh) << kTileBits), kStageBytes, mb);
                    };
                    if (tid == 0) {
                        // the stage's earlier readers (generic loads) before the copies' writes
                        fence_proxy_async_smem();
                        issue_pair(0);
                    }
                    const int xlow = xl0;
                    const int q = xlow >> 8;
                    const int pl = tid ^ (xlow & 255);
                    for (int kb = 0; kb < nb; ++kb) {
                        const int tp = (r << a.B1_log) + kb;
                        if (!mbar_wait_bounded(mb, (sphase >> 2) & 1u, a.wait_ns)) {
                            slost |= 4u;
                            if (lane == 0) atomicCAS(a.status, 0, (int)SRE_ETIMEDOUT);
                        }
                        sphase ^= 4u;
                        cx_t<R> v[16];
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const V b = par[((i ^ q) << 8) | pl];
                            const V va = own[(i << 8) | tid];
                            v[i] = conj_mul<R>(b.x, b.y, va.x, va.y);  // conj(phi_{t^x}) * phi_t
                        }
                        reg_stages<2, 12, R>(v);
#pragma unroll
                        for (int i = 0; i < 16; ++i) own[(i << 8) | tid] = Cx<R>::to(v[i]);
                        __syncthreads();
#pragma unroll
                        for (int i = 0; i < 16; ++i) v[i] = Cx<R>::from(own[elem<1>(tid, i)]);
                        __syncthreads();  // both stage buffers are free
                        if (tid == 0 && kb + 1 < nb) {
                            fence_proxy_async_smem();
                            issue_pair(kb + 1);
                        }
                        reg_stages<1, 12, R>(v);
                        relayout<1, 0, true, R>(v, bufA, tid);
                        reg_stages<0, 12, R>(v);
                        V *o = slot_base + ((size_t)tp << kTileBits) + tid;
#pragma unroll
                        for (int i = 0; i < 16; ++i) __stcg(o + (i << 8), Cx<R>::to(v[i]));
                    }
                }
            } else
            for (int kb = 0; kb < (1 << a.B1_log); ++kb) {
                const int tp = (r << a.B1_log) + kb;
                const int th = HALF ? (((tp >> jh) << (jh + 1)) | (tp & ((1 << jh) - 1))) : tp;
                // Round-2 layout: thread tid holds t_l = i << 8 | tid of block th
                // (own factors phi_t in registers); its partners t ^ x are
                // t_l ^ xlow of block th ^ x_h, read coalesced (each warp load
                // covers one aligned 256-entry run).
                R ar[16], ai[16];
                {
                    const V *pa = psi + ((uint64_t)th << kTileBits) + tid;
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const V va = __ldg(pa + (i << 8));
                        ar[i] = va.x;
                        ai[i] = va.y;
                    }
                }
                const V *pb = psi + (((uint64_t)th ^ xh) << kTileBits);
                for (int xl = 0; xl < C; ++xl) {
                    const uint64_t x = xc + (uint64_t)xl;
                    if (x < a.x_begin || x >= a.x_end) continue;
                    const int xlow = xl0 + xl;
                    const V *pbx = pb + (tid ^ (xlow & 255));
                    const int q = xlow >> 8;
                    cx_t<R> v[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const V b = __ldg(pbx + ((i ^ q) << 8));
                        v[i] = conj_mul<R>(b.x, b.y, ar[i], ai[i]);  // conj(phi_{t^x}) * phi_t
                    }
                    V *bB = (tcount & 1) ? bufC : bufB;
                    ++tcount;
                    tile_fwht12_rev<R>(v, bufA, bB, tid);
                    // output in round-0 layout (z_l = 16 tid + i) stored at the
                    // bit-permuted position i << 8 | tid: coalesced stores; pass 2
                    // only sums over z, so the order of z inside a block is free
                    V *o = slot_base + ((size_t)xl << lgx) + ((size_t)tp << kTileBits) + tid;
#pragma unroll
                    for (int i = 0; i < 16; ++i) __stcg(o + (i << 8), Cx<R>::to(v[i]));
                }
            }
            // per-warp completion: every lane's stores are fenced, then one arrival
            __threadfence();
            __syncwarp();
            if (lane == 0) atomicAdd(a.done1 + c, 1u);
        } else {
            // ---------------- pass 2: 2^G2 z-blocks of one shift; per-warp
            // wait, per-warp partial sums and per-warp completion
            const int j = r;
            const int xl = j >> ipx_log;
            const int zb0 = (j & ((1 << ipx_log) - 1)) << a.G2_log;
            const uint64_t x = xc + (uint64_t)xl;
            double acc = 0.0;
            const bool staged2 = kTma && a.stage2;
            if constexpr (kTma) {
                // One thread waits for the chunk's pass 1 and keeps two TMA
                // tile copies in flight; every thread waits on the stage's
                // mbarrier, reads the tile in layout A and transforms it.
                if (staged2 && x >= a.x_begin && x < a.x_end) {
                    const int ntiles = 1 << a.G2_log;
                    const int y = (int)(((size_t)slot * C + xl) << H2);
                    int ok = 1;
                    auto issue = [&](int g, int st) {
                        const uint32_t mb = smem_u32(&s_mbar[st]);
                        if (!ok) {
                            mbar_arrive(mb);  // no copy: release the waiters on garbage
                            return;
                        }
                        const uint32_t dst = smem_u32(st ? (void *)bufC : (void *)bufB);
                        const int x0 = (zb0 + g) << (kTileBits - H2 + 1);  // FP32 column
                        mbar_arrive_expect_tx(mb, (uint32_t)kStageBytes);
#pragma unroll
                        for (int b = 0; b < (1 << (8 - H2)); ++b)
                            tma_load_2d(dst + (uint32_t)b * (128u << H2), &a.tmap, x0 + 32 * b, y, mb);
                    };
                    if (tid == 0) {
                        ok = wait_counter(a.done1 + c, (unsigned)(a.P1 * kWarps), a.status, a.wait_ns);
                        // pass-1 stores (acquired above) and this CTA's earlier
                        // shared-memory accesses before the async-proxy copies
                        fence_proxy_async();
                        issue(0, 0);
                        if (ntiles > 1) issue(1, 1);
                    }
                    const P2Lane pl = p2_lane<H2>(lane, warp);
                    for (int gb = 0; gb < ntiles; ++gb) {
                        const int st = gb & 1;
                        if (!mbar_wait_bounded(smem_u32(&s_mbar[st]), (sphase >> st) & 1u, a.wait_ns)) {
                            slost |= 1u << st;
                            if (lane == 0) atomicCAS(a.status, 0, (int)SRE_ETIMEDOUT);
                        }
                        sphase ^= 1u << st;
                        {
                            // the tile is in shared memory: drop its 256 scratch
                            // lines (2^H2 rows x 2^(8 - H2) lines) from L2 now,
                            // one per thread, before they can be written back
                            constexpr int kLpr = 1 << (8 - H2);
                            const V *xb = slot_base + ((size_t)xl << lgx);
                            discard_l2_line(xb + ((size_t)(tid / kLpr) << kTileBits) +
                                            ((zb0 + gb) << zsub_bits) + (tid % kLpr) * 16);
                        }
                        const unsigned char *stage = reinterpret_cast<const unsigned char *>(st ? bufC : bufB);
                        const float s = p2_tile<H2, HALF>(stage, reinterpret_cast<float2 *>(bufA), pl, a.alpha);
                        acc += (HALF ? hfac : 1.0) * (double)s;
                        if (gb + 2 < ntiles) {
                            __syncthreads();  // every thread has read stage st
                            if (tid == 0) {
                                // shared-memory WAR only: the scratch rows were
                                // ordered before the copies once per item above
                                fence_proxy_async_smem();
                                issue(gb + 2, st);
                            }
                        }
                    }
                }
            }
            if (!staged2) {
            if (lane == 0) wait_counter(a.done1 + c, (unsigned)(a.P1 * kWarps), a.status, a.wait_ns);
            __syncwarp();
            __threadfence();
            if (x >= a.x_begin && x < a.x_end) {
                const V *xb = slot_base + ((size_t)xl << lgx);
                for (int gb = 0; gb < (1 << a.G2_log); ++gb) {
                    const int zb = zb0 + gb;
                    cx_t<R> v[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int e = elem<0>(tid, i);
                        const int tp = e & ((1 << H2) - 1);
                        const int zs = e >> H2;
                        v[i] = Cx<R>::from(
                            __ldcg(xb + ((size_t)tp << kTileBits) + (zb << zsub_bits) + zs));
                    }
                    V *bB = (tcount & 1) ? bufC : bufB;
                    if (H2 > 8) ++tcount;
                    tile_fwht<H2, R>(v, bufA, bB, tid);
                    acc += (HALF ? hfac : 1.0) * (double)sum_order<R, HALF>(v, a.alpha);
                }
            }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
            // All warps' loads of this item are complete after this barrier:
            // drop the item's scratch lines from L2 without write-back (dead
            // data; the next chunk in this slot rewrites them; the staged path
            // dropped each tile's lines as it arrived).  The drops precede
            // this item's arrivals, hence the slot's release.
            __syncthreads();
            constexpr int kLineElems = 128 / (int)sizeof(V);
            if (((1 << zsub_bits) >= kLineElems) && !staged2 && x >= a.x_begin && x < a.x_end) {
                const V *xb = slot_base + ((size_t)xl << lgx);
                constexpr int lines_per_row = ((1 << zsub_bits) >= kLineElems) ? (1 << zsub_bits) / kLineElems : 1;
                constexpr int lines_per_tile = kTile / kLineElems;
                for (int gb = 0; gb < (1 << a.G2_log); ++gb) {
                    const int zb = zb0 + gb;
                    for (int L = tid; L < lines_per_tile; L += kThreads) {
                        const int row = L / lines_per_row;
                        const int seg = L - row * lines_per_row;
                        discard_l2_line(xb + ((size_t)row << kTileBits) + (zb << zsub_bits) + seg * kLineElems);
                    }
                }
            }
            __syncwarp();
            int last = 0;
            if (lane == 0) {
                a.item_part[(((size_t)slot * a.P2 + j) * kWarps) + warp] = acc;
                __threadfence();
                const unsigned old = atomicAdd(a.done2 + c, 1u);
                last = (old == (unsigned)(a.P2 * kWarps) - 1u);
            }
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last) {
                // last warp of the chunk: per-shift and chunk sums in fixed
                // order, then release the slot
                __threadfence();
                const int per_x_items = (1 << ipx_log) * kWarps;
                double cs = 0.0;
                for (int q = 0; q < C; ++q) {
                    const double *ip = a.item_part + ((size_t)slot * a.P2 + ((size_t)q << ipx_log)) * kWarps;
                    double sx = 0.0;
                    for (int k = lane; k < per_x_items; k += 32) sx += __ldcg(ip + k);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) sx += __shfl_down_sync(0xffffffffu, sx, o);
                    const uint64_t xq = xc + (uint64_t)q;
                    if (lane == 0 && a.per_x && xq >= a.x_begin && xq < a.x_end) a.per_x[xq - a.x_begin] = sx;
                    cs += sx;  // lane 0's value is the one used
                }
                if (lane == 0) {
                    a.chunk_sum[c] = cs;
                    __threadfence();
                    atomicExch(a.freed + c, 1u);
                }
            }
        }
        if (tid == 0) {
            s_next[par ^ 1] = next;
            s_stop[par ^ 1] = (*(volatile int *)a.status != 0);
        }
        __syncthreads();
    }
    if constexpr (kTma || kStage1) {
        // a stage whose completion wait expired may still receive its copy:
        // wait for it once more (bounded) before the CTA's memory is released
        for (int st = 0; st < 3; ++st)
            if (slost & (1u << st)) mbar_wait_bounded(smem_u32(&s_mbar[st]), ((sphase >> st) & 1u) ^ 1u, a.wait_ns);
    }
}


}  // namespace sre
