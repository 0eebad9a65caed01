// sre_tc.cu -- the two-pass kernel of the split-precision modes
// (SRE_MODE_BF16_SPLIT, SRE_MODE_FP16_SPLIT): the Hadamard stages of both
// passes are tcgen05 MMAs against exact +-1 matrices on fixed-point hi/lo
// operands (sre_tc.cuh).  It takes the conjugate-symmetry halved shifts
// (x >= 4096) for 16 <= N <= 20; everything else runs the FP32 path.
//
// One shift's halved transform W (Algorithm 1's FWHT over the N - 1 bits of
// t' = t with the pivot bit removed; the supplement's block recursion
// H_{2^(N-1)} = H_{2^h2} (x) H_2 (x) H_128 (x) H_16 over the bit groups
// [12, N-1), 7, [0, 7), [8, 12)) is computed as:
//
// pass 1, per 4096-entry block t'_h (a "tile", 8192 real values):
//   * products conj(psi[t ^ x]) psi[t] in registers (thread tid holds
//     t_l = i << 8 | tid, i < 16), butterflies over bits 8-11 in registers;
//   * a power-of-two scale: with FP16 pieces (24 bits), from the block
//     pair's bound 16 max|psi| max|psi'| (every value is a signed sum of 16
//     products); with BF16 pieces (18 bits), from the tile's own maximum;
//     the values are split into fixed-point pieces and written
//     as the N-major B operand [K = 128 rows t_l & 127] x [N = 128 columns
//     (piece, t bit 7, i, re/im)];
//   * one MMA stage D = H_128 B over bits 0-6 (8 MMAs, K = 16 each) into
//     TMEM; the thread that reads lane z_l & 127 gets both t bit 7 columns
//     and does the bit-7 butterfly in registers;
//   * the result is split again at the shift's fixed-point scale 2^(P - E)
//     (E from the block-norm bound below) and stored as two 16-bit planes
//     (hi, lo) of scratch rows [slot][shift][plane][t'_h][8192].
// pass 2, per tile of 128 scratch rows x 32 complex columns:
//   * TMA copies the hi and lo planes into the two 64-column atom columns of
//     an N = 128 B operand (128-byte swizzle), through the ring of four
//     copy units that pass 1's block pairs also use;
//   * one MMA stage D = A B over the h2 high bits, A = H_128 (h2 = 7) or the
//     block-diagonal I (x) H_{2^h2} (h2 < 7, the tile then stacks 2^(7-h2)
//     column blocks along K);
//   * F = lo - hi per TMEM column pair, sum F^4 (re and im columns, the
//     halved form), scaled by 16 2^(4 (E - P)).
//
// Per-shift scale.  |A pass-1 output| <= n(b) n(b ^ x_h) by Cauchy-Schwarz
// over the block pair (n = block l2 norm of psi), so E = ceil(log2 of the
// largest such product over the shift's blocks, times 1 + 2^-10) keeps every
// scaled value inside [-2^P, 2^P]: pass 2 contracts over rows that come from
// different blocks and needs one scale along K.  k_tc_scales computes E per
// x >> 12 (per state, for the states of a batch class) before the launch.
//
// Pipelining: warp-specialized roles (below) with two B buffers, three TMEM
// accumulators and a ring of copy units, so that copies, MMAs and CUDA-core
// work of different tiles overlap.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "sre_batched.h"
#include "sre_large.cuh"
#include "sre_tc.cuh"

namespace sre {

namespace {

constexpr int kTcMinH2 = 3, kTcMaxH2 = 7;

// ----------------------------------------------------------- scale table

// l2 norm of every 4096-entry block of psi (FP64); blockIdx.y selects the
// state of a batch class (psis), whose nb = gridDim.x norms follow those of
// the state before.
__global__ void __launch_bounds__(kThreads) k_tc_block_norms(const float2 *__restrict__ psi,
                                                             const void *const *psis,
                                                             double *__restrict__ bn) {
    __shared__ double red[kThreads / 32];
    const float2 *base = psis ? reinterpret_cast<const float2 *>(psis[blockIdx.y]) : psi;
    const float2 *p = base + ((size_t)blockIdx.x << kTileBits);
    double s = 0.0;
    for (int t = threadIdx.x; t < kTile; t += kThreads) {
        const float2 v = p[t];
        s += (double)v.x * v.x + (double)v.y * v.y;
    }
    const double b = block_sum(s, red);
    if (threadIdx.x == 0) bn[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = sqrt(b);
}

// E[x_h] for x_h in [1, nb): ceil(log2(max over blocks b with pivot bit 0 of
// n(b) n(b ^ x_h), times 1 + 2^-10)); -100 where every product is zero.
// blockIdx.y selects the state (nb entries of bn and of E per state).
__global__ void k_tc_scales(const double *__restrict__ bn_all, int nb, int *__restrict__ E_all) {
    const int xh = blockIdx.x * blockDim.x + threadIdx.x;
    if (xh >= nb) return;
    const double *bn = bn_all + (size_t)blockIdx.y * nb;
    int *E = E_all + (size_t)blockIdx.y * nb;
    if (xh == 0) {
        E[0] = 0;
        return;
    }
    const int piv = 31 - __clz(xh);
    double m = 0.0;
    for (int b = 0; b < nb; ++b)
        if (!((b >> piv) & 1)) m = fmax(m, bn[b] * bn[b ^ xh]);
    int e = -100;
    if (m > 0.0) {
        int ex;
        const double f = frexp(m * (1.0 + 1.0 / 1024.0), &ex);  // m' = f 2^ex, f in [1/2, 1)
        e = (f == 0.5) ? ex - 1 : ex;                            // smallest e with m' <= 2^e
        e = max(-100, min(100, e));
    }
    E[xh] = e;
}

__device__ __forceinline__ unsigned long long pack2f(float a, float b) {
    unsigned long long d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(a), "f"(b));
    return d;
}

// lo - hi of 16 accumulator columns (hi stored negated), as 8 packed pairs
// of adjacent columns (re, im).
__device__ __forceinline__ void tc_combine16(const uint32_t (&hv)[16], const uint32_t (&lv)[16],
                                             unsigned long long *F) {
#pragma unroll
    for (int j = 0; j < 8; ++j)
        F[j] = Cx<float>::sub(pack2f(__uint_as_float(lv[2 * j]), __uint_as_float(lv[2 * j + 1])),
                              pack2f(__uint_as_float(hv[2 * j]), __uint_as_float(hv[2 * j + 1])));
}

// ---------------------------------------------------------------- kernel
//
// One CTA per SM, warp-specialized (448 threads):
//   warps 0-7   compute: pass-1 products, bits 8-11, split into the B
//               operand (double-buffered in shared memory) at the block
//               pair's scale;
//   warps 8-11  epilogue: read an accumulator (warp 8 + q reads TMEM lanes
//               32 q .. 32 q + 31, all 128 columns); pass 1: bit-7
//               butterfly, split at the shift's scale, scratch stores; pass
//               2: sum of fourth powers;
//   warp 12     producer: claims work items into a queue of kQueue entries;
//               copies each pass-1 block pair (own and partner block of psi,
//               32 KB each) or each pass-2 tile (hi and lo planes, TMA) into
//               a ring of four 32 KB units;
//   warp 13     MMA: D = A B for every tile into one of three TMEM
//               accumulators (128 columns each).
// Every role walks the same item sequence; the handoffs are mbarriers:
//   queue  q_full (producer -> 13 consumer warps), q_empty (13 arrivals);
//   units  u_full1 / u_full2 (copy bytes of a pass-1 / pass-2 fill),
//          u_empty (pass 1: compute warps after a block pair; pass 2: the
//          MMA's commit);
//   B      b_full (8 compute-warp arrivals), b_empty (MMA commit);
//   D      d_full (MMA commit), d_empty (4 epilogue-warp arrivals).
// A parity wait only tells apart adjacent phases, so every barrier has one
// group of waiters that sees each of its phases in order.  Each role waits
// only on its own upstream for the same or an earlier item, or (pass-1
// epilogue: ring slot; pass-2 producer: pass 1 of the chunk) on items
// claimed earlier, so the lagged item order stays deadlock-free.  All waits
// are bounded and give up at once when an error has been recorded; the
// producer and the MMA warp wait for their last copies and MMAs before the
// CTA exits.

constexpr int kTcThreads = 448;
constexpr int kCompWarps = 8, kEpiWarp0 = 8, kProdWarp = 12, kMmaWarp = 13;
constexpr int kUnits = 4;                 // 32 KB ring units
constexpr uint32_t kUnitBytes = 32768;
constexpr int kQueue = 2;                 // item queue entries (claims run at most this far ahead)
constexpr int kAcc = 3;                   // TMEM accumulators
constexpr uint32_t kTcCols = 512;         // TMEM: H 64 | A2 64 | D0 | D1 | D2 (128 each)
constexpr uint32_t kBOff = kUnits * kUnitBytes;  // two B buffers after the units

static_assert(128 + kAcc * 128 <= (int)kTcCols, "accumulators and factors fit TMEM");
__host__ __device__ constexpr size_t tc_smem_bytes() {
    return (size_t)kUnits * kUnitBytes + 2 * (size_t)kUnitBytes + 1024;
}

// Item geometry shared by all roles.
struct TcItem {
    long long chunk;
    int r, slot;
    int pass1;
    int E;             // scale exponent of the chunk's shifts
    int first, count;  // valid shifts of the chunk: [first, first + count)
    uint64_t xc, xh;
    const float2 *psi;
};

struct __align__(8) TcShared {
    // "full" barriers exist once per consumer, so that every waiter sees
    // each phase of its barrier in order (a parity wait cannot tell a phase
    // from the one two later): u_full1 for pass-1 block pairs (compute
    // warps), u_full2 for pass-2 tiles (MMA warp)
    uint64_t u_full1[kUnits], u_full2[kUnits], u_empty[kUnits];
    uint64_t b_full[2], b_empty[2], d_full[kAcc], d_empty[kAcc];
    uint64_t q_full[kQueue], q_empty[kQueue];
    long long q_item[kQueue];
    TcItem q_dec[kQueue];           // the item decoded once, by the producer
    unsigned long long s1_ring[8];  // pass-1 tile scale: (float bits, tile index + 1)
    uint32_t maxq[kCompWarps], maxp[kCompWarps];  // per block pair: max |psi|^2 of each warp's entries
    uint32_t maxt[2][kCompWarps];                  // BF16: per tile, max |value| of each warp
    double epi_part[2][4];                         // pass-2 item partials of the epilogue warps
    uint32_t tmem;
};

// Bounded wait that gives up at once once an error has been recorded.
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity, const LargeArgs &a) {
    const unsigned long long t0 = globaltimer_ns();
    for (unsigned it = 0; it < (1u << 28); ++it) {
        if (mbar_try_wait(mbar, parity)) return true;
        if ((it & 15) == 15) {
            if (*(volatile int *)a.status != 0) return false;
            if ((long long)(globaltimer_ns() - t0) > a.wait_ns) {
                atomicCAS(a.status, 0, (int)SRE_ETIMEDOUT);
                return false;
            }
        }
    }
    atomicCAS(a.status, 0, (int)SRE_ETIMEDOUT);
    return false;
}

__device__ __forceinline__ void bar_sync_comp() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
__device__ __forceinline__ void bar_sync_epi() { asm volatile("bar.sync 2, 128;" ::: "memory"); }

// Release / acquire at GPU scope by one lane for its warp: after __syncwarp
// the fence also orders the other lanes' earlier accesses (fences are
// cumulative), so one lane does it instead of every lane.
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }


__device__ __forceinline__ TcItem tc_item(const LargeArgs &a, long long item) {
    TcItem t;
    bool p1;
    decode_item(a, item, t.chunk, t.r, p1);
    t.pass1 = p1 ? 1 : 0;
    t.slot = (int)(t.chunk % a.R);
    long long cl = t.chunk;
    t.psi = reinterpret_cast<const float2 *>(a.psi);
    if (a.psis) {
        const long long sidx = t.chunk / a.chunks_per_state;
        cl = t.chunk - sidx * a.chunks_per_state;
        t.psi = reinterpret_cast<const float2 *>(a.psis[sidx]);
    }
    t.xc = a.x0 + ((uint64_t)cl << a.C_log);
    t.xh = t.xc >> kTileBits;
    t.E = a.tc_e[((size_t)(t.chunk / a.chunks_per_state) << (a.N - kTileBits)) + t.xh];
    const int C = 1 << a.C_log;
    int f = 0;
    while (f < C && !(t.xc + (uint64_t)f >= a.x_begin && t.xc + (uint64_t)f < a.x_end)) ++f;
    int n = 0;
    while (f + n < C && t.xc + (uint64_t)(f + n) >= a.x_begin && t.xc + (uint64_t)(f + n) < a.x_end) ++n;
    t.first = f;
    t.count = n;
    return t;
}

__device__ __forceinline__ bool x_valid(const LargeArgs &a, uint64_t x) { return x >= a.x_begin && x < a.x_end; }

// Block t_h of halved block index tp: a zero inserted at the pivot bit jh.
__device__ __forceinline__ int tc_block(int tp, int jh) { return ((tp >> jh) << (jh + 1)) | (tp & ((1 << jh) - 1)); }

template <int H2, int KIND>
__global__ void __launch_bounds__(kTcThreads, 1) k_tc(const __grid_constant__ LargeArgs a) {
    constexpr int P = tc_piece_bits<KIND>();
    constexpr uint32_t idesc = tc_idesc<KIND>(128);
    constexpr int kBlocksPerTile = 1 << (7 - H2);  // column blocks stacked along K in pass 2
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *sbase = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    __shared__ TcShared sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t s0 = smem_u32(sbase);
    const int C = 1 << a.C_log;
    const int ipx_log = H2 - a.G2_log;

    if (warp == kEpiWarp0) tc_alloc(&sh.tmem, kTcCols);
    if (tid == 0) {
        for (int k = 0; k < kUnits; ++k) {
            mbar_init(smem_u32(&sh.u_full1[k]), 1);
            mbar_init(smem_u32(&sh.u_full2[k]), 1);
            mbar_init(smem_u32(&sh.u_empty[k]), 1);
        }
        for (int k = 0; k < 2; ++k) {
            mbar_init(smem_u32(&sh.b_full[k]), kCompWarps);
            mbar_init(smem_u32(&sh.b_empty[k]), 1);
        }
        for (int k = 0; k < kAcc; ++k) {
            mbar_init(smem_u32(&sh.d_full[k]), 1);
            mbar_init(smem_u32(&sh.d_empty[k]), 4);  // the 4 epilogue warps
        }
        for (int k = 0; k < kQueue; ++k) {
            mbar_init(smem_u32(&sh.q_full[k]), 1);
            mbar_init(smem_u32(&sh.q_empty[k]), kCompWarps + 4 + 1);
        }
        for (int k = 0; k < 8; ++k) sh.s1_ring[k] = 0ull;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh.tmem;
    if (warp >= kEpiWarp0 && warp < kEpiWarp0 + 4) {
        tc_write_hadamard<KIND>(tmem, 0, 7, warp - kEpiWarp0, lane);
        if (H2 < 7) tc_write_hadamard<KIND>(tmem, 64, H2, warp - kEpiWarp0, lane);
        tc_wait_st();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tH = tmem, tA2 = H2 == 7 ? tmem : tmem + 64;
    unsigned short *scr = reinterpret_cast<unsigned short *>(a.scratch);
    const unsigned long long magic = pack2f(kRoundMagic, kRoundMagic);

    if (warp == kProdWarp) {
        // ------------------------------------------------------- producer
        if (lane == 0) {
            unsigned long long ucount = 0;  // units filled so far
            uint32_t f1 = 0, f2 = 0;        // units with an odd number of pass-1 / pass-2 fills
            uint32_t p1used = 0, p2used = 0;
            for (long long k = 0;; ++k) {
                const int qs = (int)(k % kQueue);
                if (k >= kQueue) tc_wait(smem_u32(&sh.q_empty[qs]), (uint32_t)((k / kQueue - 1) & 1), a);
                long long item = (long long)atomicAdd(a.work, 1ull);
                if (*(volatile int *)a.status != 0) item = a.n_items;  // stop: everyone drains
                sh.q_item[qs] = item;
                TcItem it{};
                if (item < a.n_items) {
                    it = tc_item(a, item);
                    sh.q_dec[qs] = it;
                }
                mbar_arrive(smem_u32(&sh.q_full[qs]));
                if (item >= a.n_items) break;
                int first = it.first, count = it.count;
                auto take_unit = [&]() {
                    const int u = (int)(ucount % kUnits);
                    const unsigned long long use = ucount / kUnits;
                    if (use > 0) tc_wait(smem_u32(&sh.u_empty[u]), (uint32_t)((use - 1) & 1), a);
                    ++ucount;
                    return u;
                };
                if (it.pass1) {
                    if (count == 0) continue;
                    const int jh = (63 - __clzll((long long)it.xc)) - kTileBits;
                    for (int kb = 0; kb < (1 << a.B1_log); ++kb) {
                        const int th = tc_block((it.r << a.B1_log) + kb, jh);
                        const int uq = take_unit(), up = take_unit();
                        // the units' earlier readers (generic loads of the compute
                        // warps, or MMAs) come before the copies' writes
                        fence_proxy_async_smem();
                        const uint32_t fq = smem_u32(&sh.u_full1[uq]), fp = smem_u32(&sh.u_full1[up]);
                        f1 ^= (1u << uq) | (1u << up);
                        p1used |= (1u << uq) | (1u << up);
                        mbar_arrive_expect_tx(fq, kUnitBytes);
                        bulk_load(s0 + (uint32_t)uq * kUnitBytes, it.psi + ((uint64_t)th << kTileBits), kUnitBytes, fq);
                        mbar_arrive_expect_tx(fp, kUnitBytes);
                        bulk_load(s0 + (uint32_t)up * kUnitBytes, it.psi + (((uint64_t)th ^ it.xh) << kTileBits),
                                  kUnitBytes, fp);
                    }
                } else {
                    const int xl = it.r >> ipx_log;
                    if (!x_valid(a, it.xc + (uint64_t)xl)) continue;
                    const int zb0 = (it.r & ((1 << ipx_log) - 1)) << a.G2_log;
                    const int y_hi = (int)((((size_t)it.slot * C + xl) * 2) << H2);
                    wait_counter(a.done1 + it.chunk, (unsigned)a.P1, a.status, a.wait_ns);
                    // the chunk's scratch rows (generic stores of other CTAs,
                    // acquired above) come before the TMA reads
                    fence_proxy_async();
                    for (int g = 0; g < (1 << a.G2_log); ++g) {
                        const int u = take_unit();
                        fence_proxy_async_smem();
                        const uint32_t f = smem_u32(&sh.u_full2[u]);
                        f2 ^= 1u << u;
                        p2used |= 1u << u;
                        const uint32_t dst = s0 + (uint32_t)u * kUnitBytes;
                        mbar_arrive_expect_tx(f, kUnitBytes);
#pragma unroll
                        for (int b = 0; b < kBlocksPerTile; ++b) {
                            const int col = ((zb0 + g) * kBlocksPerTile + b) * 64;
                            tma_load_2d(dst + (uint32_t)(b << (H2 + 7)), &a.tmap, col, y_hi, f);
                            tma_load_2d(dst + 16384u + (uint32_t)(b << (H2 + 7)), &a.tmap, col, y_hi + (1 << H2), f);
                        }
                    }
                }
            }
            // copies still in flight land before the CTA's memory is released:
            // wait for the latest fill of each kind of every unit (the phase
            // with the parity before the next one)
            for (int u = 0; u < kUnits; ++u) {
                if (p1used & (1u << u))
                    mbar_wait_bounded(smem_u32(&sh.u_full1[u]), ((f1 >> u) & 1u) ^ 1u, a.wait_ns);
                if (p2used & (1u << u))
                    mbar_wait_bounded(smem_u32(&sh.u_full2[u]), ((f2 >> u) & 1u) ^ 1u, a.wait_ns);
            }
        }
        __syncwarp();
    } else {
        // consumers: compute warps, epilogue warps, MMA warp
        const bool is_comp = warp < kCompWarps;
        const bool is_epi = warp >= kEpiWarp0 && warp < kEpiWarp0 + 4;
        const bool is_mma = warp == kMmaWarp;
        unsigned long long ucount = 0;  // ring units consumed
        unsigned long long btile = 0;   // pass-1 tiles (B buffers, scale ring)
        unsigned long long dtile = 0;   // tiles of either pass (accumulators)
        uint32_t par_u = 0;             // parity of the next u_full1 (compute) / u_full2 (MMA) phase, per unit
        uint32_t par_d = 0;             // parity of the next d_full phase, per accumulator
        uint32_t mma_used = 0;          // MMA: accumulators committed to
        unsigned long long p2items = 0;  // epilogue: pass-2 items done
        float2 Q[16];                   // compute: own factors of the block pair
        for (long long k = 0;; ++k) {
            const int qs = (int)(k % kQueue);
            tc_wait(smem_u32(&sh.q_full[qs]), (uint32_t)((k / kQueue) & 1), a);
            const long long item = *(volatile long long *)&sh.q_item[qs];
            TcItem it{};
            if (item < a.n_items) it = sh.q_dec[qs];
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&sh.q_empty[qs]));
            if (item >= a.n_items) break;
            if (it.pass1) {
                const int first = it.first, count = it.count;
                if (count == 0) {
                    if (is_epi) {
                        bar_sync_epi();
                        if (warp == kEpiWarp0 && lane == 0) {
                            fence_acq_rel_gpu();
                            atomicAdd(a.done1 + it.chunk, 1u);
                        }
                    }
                    continue;
                }
                const int jh = (63 - __clzll((long long)it.xc)) - kTileBits;
                const int xl0 = (int)(it.xc & (kTile - 1));
                const int nb = 1 << a.B1_log;
                if (is_comp) {
                    // ------------------------------------------------- compute
                    const int k7 = tid & 127, hb = tid >> 7;
                    const uint32_t brow = (uint32_t)((k7 >> 3) * 2048 + (k7 & 7) * 16);
                    for (int kb = 0; kb < nb; ++kb) {
                        const int uq = (int)(ucount % kUnits), up = (int)((ucount + 1) % kUnits);
                        tc_wait(smem_u32(&sh.u_full1[uq]), (par_u >> uq) & 1u, a);
                        par_u ^= 1u << uq;
                        tc_wait(smem_u32(&sh.u_full1[up]), (par_u >> up) & 1u, a);
                        par_u ^= 1u << up;
                        ucount += 2;
                        const float2 *sq = reinterpret_cast<const float2 *>(sbase + (size_t)uq * kUnitBytes);
                        const float2 *sp = reinterpret_cast<const float2 *>(sbase + (size_t)up * kUnitBytes);
                        // scale of the block pair: every value after the 4 register
                        // butterflies is a signed sum of 16 products, so
                        // |v| <= 16 max|phi_t| max|phi_t'| over the two blocks
                        float mq = 0.f, mp = 0.f;
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            Q[i] = sq[(i << 8) | tid];
                            const float2 pn = sp[(i << 8) | tid];
                            mq = fmaxf(mq, Q[i].x * Q[i].x + Q[i].y * Q[i].y);
                            mp = fmaxf(mp, pn.x * pn.x + pn.y * pn.y);
                        }
                        {
                            const uint32_t wq = __reduce_max_sync(0xffffffffu, __float_as_uint(mq));
                            const uint32_t wp = __reduce_max_sync(0xffffffffu, __float_as_uint(mp));
                            if (lane == 0) {
                                sh.maxq[warp] = wq;
                                sh.maxp[warp] = wp;
                            }
                        }
                        bar_sync_comp();
                        float s1_pair;  // FP16 pieces (24 bits) take the block pair's bound
                        {
                            uint32_t tq = sh.maxq[0], tpp = sh.maxp[0];
#pragma unroll
                            for (int w = 1; w < kCompWarps; ++w) {
                                tq = max(tq, sh.maxq[w]);
                                tpp = max(tpp, sh.maxp[w]);
                            }
                            // 1 + 2^-10 covers the rounding of the FP32 products and sums
                            const float bound = 16.f * sqrtf(__uint_as_float(tq) * __uint_as_float(tpp)) * 1.0009765625f;
                            s1_pair = tc_block_scale<P>(bound);
                        }
                        for (int xl = first; xl < first + count; ++xl) {
                            const int xlow = xl0 + xl;
                            const int q = xlow >> 8, pl = tid ^ (xlow & 255);
                            cx_t<float> v[16];
#pragma unroll
                            for (int i = 0; i < 16; ++i) {
                                const float2 b = sp[((i ^ q) << 8) | pl];
                                v[i] = conj_mul<float>(b.x, b.y, Q[i].x, Q[i].y);  // conj(phi_{t^x}) phi_t
                            }
                            reg_stages<2, 12, float>(v);  // bits 8-11
                            float s1 = s1_pair;
                            if constexpr (KIND == kTcBf16) {
                                // BF16 pieces hold 18 bits: scale by the tile's own
                                // maximum (non-negative floats order like their bits)
                                float m16[16];
#pragma unroll
                                for (int i = 0; i < 16; ++i) {
                                    float re, im;
                                    Cx<float>::unpack(v[i], re, im);
                                    m16[i] = fmaxf(fabsf(re), fabsf(im));
                                }
#pragma unroll
                                for (int w = 8; w > 0; w >>= 1)
#pragma unroll
                                    for (int i = 0; i < w; ++i) m16[i] = fmaxf(m16[i], m16[i + w]);
                                const int par = (int)(btile & 1);
                                const uint32_t wm = __reduce_max_sync(0xffffffffu, __float_as_uint(m16[0]));
                                if (lane == 0) sh.maxt[par][warp] = wm;
                                bar_sync_comp();
                                uint32_t tm = sh.maxt[par][0];
#pragma unroll
                                for (int w = 1; w < kCompWarps; ++w) tm = max(tm, sh.maxt[par][w]);
                                s1 = tc_block_scale<P>(__uint_as_float(tm));
                            }
                            if (tid == 0) {
                                const unsigned long long e =
                                    (unsigned long long)__float_as_uint(s1) | ((btile + 1) << 32);
                                asm volatile("st.volatile.shared.u64 [%0], %1;" ::"r"(smem_u32(&sh.s1_ring[btile & 7])),
                                             "l"(e)
                                             : "memory");
                            }
                            const int bb = (int)(btile & 1);
                            if (btile >= 2) tc_wait(smem_u32(&sh.b_empty[bb]), (uint32_t)((btile / 2 - 1) & 1), a);
                            {
                                const unsigned long long sc = pack2f(s1, s1);
                                const uint32_t bbase = s0 + kBOff + (uint32_t)bb * kUnitBytes + brow;
#pragma unroll
                                for (int j4 = 0; j4 < 4; ++j4) {
                                    uint32_t h[4], l[4];
#pragma unroll
                                    for (int u = 0; u < 4; ++u) tc_split<KIND>(v[4 * j4 + u], sc, magic, h[u], l[u]);
                                    const uint32_t ng = (uint32_t)(hb * 4 + j4);
                                    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(bbase + ng * 128u),
                                                 "r"(h[0]), "r"(h[1]), "r"(h[2]), "r"(h[3])
                                                 : "memory");
                                    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(bbase + (ng + 8u) * 128u),
                                                 "r"(l[0]), "r"(l[1]), "r"(l[2]), "r"(l[3])
                                                 : "memory");
                                }
                            }
                            fence_proxy_async_smem();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(smem_u32(&sh.b_full[bb]));
                            ++btile;
                            ++dtile;
                        }
                        // every compute warp is done with the block pair
                        bar_sync_comp();
                        if (tid == 0) {
                            mbar_arrive(smem_u32(&sh.u_empty[uq]));
                            mbar_arrive(smem_u32(&sh.u_empty[up]));
                        }
                    }
                } else if (is_mma) {
                    // ----------------------------------------------------- MMA
                    for (int kb = 0; kb < nb; ++kb) {
                        ucount += 2;
                        for (int xl = 0; xl < count; ++xl) {
                            const int bb = (int)(btile & 1), dd = (int)(dtile % kAcc);
                            tc_wait(smem_u32(&sh.b_full[bb]), (uint32_t)((btile / 2) & 1), a);
                            if (dtile >= kAcc) tc_wait(smem_u32(&sh.d_empty[dd]), (uint32_t)((dtile / kAcc - 1) & 1), a);
                            tc_fence_after();
                            if (lane == 0) {
                                // K step s: operand rows 16 s .., 4096 bytes further
                                tc_mma_stage(tmem + 128u * (uint32_t)(dd + 1), tH,
                                             tc_desc_mn(s0 + kBOff + (uint32_t)bb * kUnitBytes, 2048u, 128u),
                                             4096u >> 4, idesc);
                                tc_commit(smem_u32(&sh.b_empty[bb]));
                                tc_commit(smem_u32(&sh.d_full[dd]));
                            }
                            __syncwarp();
                            par_d ^= 1u << dd;
                            mma_used |= 1u << dd;
                            ++btile;
                            ++dtile;
                        }
                    }
                } else if (is_epi) {
                    // ------------------------------------------------ epilogue
                    const int qd = warp - kEpiWarp0;
                    const int m = 32 * qd + lane;
                    if (it.chunk >= a.R) {
                        if (lane == 0) wait_counter(a.freed + (it.chunk - a.R), 1u, a.status, a.wait_ns);
                        __syncwarp();
                    }
                    const size_t slot_row = (size_t)it.slot * C * 2;
                    for (int kb = 0; kb < nb; ++kb) {
                        ucount += 2;
                        const int tp = (it.r << a.B1_log) + kb;
                        for (int xl = first; xl < first + count; ++xl) {
                            const int dd = (int)(dtile % kAcc);
                            // this tile's scale (written before its operand)
                            float s1 = 1.f;
                            {
                                const unsigned long long want = btile + 1;
                                const unsigned long long t0 = globaltimer_ns();
                                for (unsigned itn = 0; itn < (1u << 24); ++itn) {
                                    unsigned long long e;
                                    asm volatile("ld.volatile.shared.u64 %0, [%1];" : "=l"(e) : "r"(smem_u32(&sh.s1_ring[btile & 7])) : "memory");
                                    if ((e >> 32) == want) {
                                        s1 = __uint_as_float((uint32_t)e);
                                        break;
                                    }
                                    if ((itn & 15) == 15 && (*(volatile int *)a.status != 0 ||
                                                              (long long)(globaltimer_ns() - t0) > a.wait_ns))
                                        break;
                                }
                            }
                            tc_wait(smem_u32(&sh.d_full[dd]), (par_d >> dd) & 1u, a);
                            par_d ^= 1u << dd;
                            tc_fence_after();
                            const int k12 = P - it.E - ((__float_as_int(s1) >> 23) - 127);
                            const float c12 = __int_as_float((max(-126, min(126, k12)) + 127) << 23);
                            const unsigned long long sc = pack2f(c12, c12);
                            const size_t row_hi = ((slot_row + 2 * (size_t)xl) << H2) + (size_t)tp;
                            const size_t row_lo = row_hi + ((size_t)1 << H2);
                            const uint32_t dcol = tmem + 128u * (uint32_t)(dd + 1) + ((uint32_t)(32 * qd) << 16);
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                // complex i = 8 h + j: hi columns (t bit 7 = b) 32 b + 16 h + 2 j (+1), lo 64 further
                                unsigned long long F0[8], F1[8];
                                {
                                    uint32_t h0[16], l0[16], h1[16], l1[16];
                                    tc_ld16(dcol + 16u * h, h0);
                                    tc_ld16(dcol + 64u + 16u * h, l0);
                                    tc_ld16(dcol + 32u + 16u * h, h1);
                                    tc_ld16(dcol + 96u + 16u * h, l1);
                                    tc_wait_ld();
                                    tc_combine16(h0, l0, F0);
                                    tc_combine16(h1, l1, F1);
                                }
                                if (h == 1) {
                                    // the accumulator has been read: release it
                                    tc_fence_before();
                                    __syncwarp();
                                    if (lane == 0) mbar_arrive(smem_u32(&sh.d_empty[dd]));
                                }
#pragma unroll
                                for (int z7 = 0; z7 < 2; ++z7) {
#pragma unroll
                                    for (int i4 = 0; i4 < 2; ++i4) {
                                        uint32_t hi[4], lo[4];
#pragma unroll
                                        for (int u = 0; u < 4; ++u) {
                                            const int jj = 4 * i4 + u;
                                            const unsigned long long w =
                                                z7 ? Cx<float>::sub(F0[jj], F1[jj]) : Cx<float>::add(F0[jj], F1[jj]);
                                            tc_split<KIND>(w, sc, magic, hi[u], lo[u]);
                                        }
                                        // z = i << 8 | z7 << 7 | m stored at complex position
                                        // (i >> 2) << 10 | z7 << 9 | m << 2 | (i & 3): a warp's
                                        // store covers 512 contiguous bytes (pass 2 sums over
                                        // every z, so the order inside a row is free)
                                        const int i_hi = 2 * h + i4;
                                        const size_t pos = (size_t)((i_hi << 10) | (z7 << 9) | (m << 2)) * 2;
                                        __stcg(reinterpret_cast<uint4 *>(scr + (row_hi << 13) + pos),
                                               make_uint4(hi[0], hi[1], hi[2], hi[3]));
                                        __stcg(reinterpret_cast<uint4 *>(scr + (row_lo << 13) + pos),
                                               make_uint4(lo[0], lo[1], lo[2], lo[3]));
                                    }
                                }
                            }
                            ++btile;
                            ++dtile;
                        }
                    }
                    // the item's stores are complete: after a barrier of the four
                    // epilogue warps one release (fences are cumulative) and
                    // one arrival per item
                    bar_sync_epi();
                    if (warp == kEpiWarp0 && lane == 0) {
                        fence_acq_rel_gpu();
                        atomicAdd(a.done1 + it.chunk, 1u);
                    }
                } else {
                    // other lanes of the producer warp never get here; the
                    // count keeps the ring position of idle roles consistent
                    ucount += 2 * nb;
                    btile += (unsigned long long)nb * count;
                    dtile += (unsigned long long)nb * count;
                }
            } else {
                // ------------------------------------------------------ pass 2
                const int j = it.r;
                const int xl = j >> ipx_log;
                const bool valid = x_valid(a, it.xc + (uint64_t)xl);
                const int ntiles = valid ? 1 << a.G2_log : 0;
                if (is_mma) {
                    for (int g = 0; g < ntiles; ++g) {
                        const int u = (int)(ucount % kUnits), dd = (int)(dtile % kAcc);
                        tc_wait(smem_u32(&sh.u_full2[u]), (par_u >> u) & 1u, a);
                        par_u ^= 1u << u;
                        if (dtile >= kAcc) tc_wait(smem_u32(&sh.d_empty[dd]), (uint32_t)((dtile / kAcc - 1) & 1), a);
                        tc_fence_after();
                        if (lane == 0) {
                            // K step s: 16 swizzled rows, 2048 bytes further
                            tc_mma_stage(tmem + 128u * (uint32_t)(dd + 1), tA2,
                                         tc_desc_mn_sw128(s0 + (uint32_t)u * kUnitBytes, 16384u), 2048u >> 4, idesc);
                            tc_commit(smem_u32(&sh.u_empty[u]));
                            tc_commit(smem_u32(&sh.d_full[dd]));
                        }
                        __syncwarp();
                        par_d ^= 1u << dd;
                        mma_used |= 1u << dd;
                        ++ucount;
                        ++dtile;
                    }
                } else if (is_epi) {
                    // pass-2 epilogue: warp 8 + q reads TMEM lanes 32 q .., all
                    // 128 columns (hi 0-63, lo 64-127) in two halves
                    const int qd = warp - kEpiWarp0;
                    float part = 0.f;
                    for (int g = 0; g < ntiles; ++g) {
                        const int dd = (int)(dtile % kAcc);
                        tc_wait(smem_u32(&sh.d_full[dd]), (par_d >> dd) & 1u, a);
                        par_d ^= 1u << dd;
                        tc_fence_after();
                        const uint32_t dcol = tmem + 128u * (uint32_t)(dd + 1) + ((uint32_t)(32 * qd) << 16);
                        unsigned long long s4 = 0ull;
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            unsigned long long F[16];
                            {
                                uint32_t h0[16], h1[16], l0[16], l1[16];
                                tc_ld16(dcol + 32u * h, h0);
                                tc_ld16(dcol + 32u * h + 16u, h1);
                                tc_ld16(dcol + 64u + 32u * h, l0);
                                tc_ld16(dcol + 64u + 32u * h + 16u, l1);
                                tc_wait_ld();
                                tc_combine16(h0, l0, F);
                                tc_combine16(h1, l1, F + 8);
                            }
                            if (h == 1) {
                                // the accumulator has been read: release it
                                tc_fence_before();
                                __syncwarp();
                                if (lane == 0) mbar_arrive(smem_u32(&sh.d_empty[dd]));
                            }
#pragma unroll
                            for (int uu = 0; uu < 16; ++uu) {
                                const unsigned long long sq = Cx<float>::mul(F[uu], F[uu]);
                                s4 = Cx<float>::fma(sq, sq, s4);
                            }
                        }
                        float sa, sb;
                        Cx<float>::unpack(s4, sa, sb);
                        part += sa + sb;
                        ++ucount;
                        ++dtile;
                    }
                    {
                        // drop the item's scratch lines from L2 (dead data; the
                        // next chunk in this slot rewrites them)
                        if (valid) {
                            const int zb0 = (j & ((1 << ipx_log) - 1)) << a.G2_log;
                            const size_t y_hi = (((size_t)it.slot * C + xl) * 2) << H2;
                            const int lines = (1 << a.G2_log) * 256;
                            for (int L = tid - kEpiWarp0 * 32; L < lines; L += 128) {
                                const int g = L >> 8, w = L & 255;
                                const int plane = w >> 7, b = (w & 127) >> H2, row = w & ((1 << H2) - 1);
                                const int col = ((zb0 + g) * kBlocksPerTile + b) * 64;
                                discard_l2_line(scr + ((y_hi + ((size_t)plane << H2) + row) << 13) + col);
                            }
                        }
                    }
                    // halved form: 16 sum (Re W)^4 + (Im W)^4, W = F 2^(E - P)
                    double acc = valid ? ldexp((double)part, 4 + 4 * (it.E - P)) : 0.0;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
                    // the four warps' partials, added in warp order by warp 8,
                    // which releases the item with one arrival (the buffers
                    // alternate between pass-2 items: warp 8 reads one before
                    // it reaches the next item's barrier)
                    const int pb = (int)(p2items & 1);
                    ++p2items;
                    if (lane == 0) sh.epi_part[pb][qd] = acc;
                    bar_sync_epi();  // also orders every warp's discards before the arrival
                    if (warp != kEpiWarp0) continue;
                    int last = 0;
                    if (lane == 0) {
                        const double v = ((sh.epi_part[pb][0] + sh.epi_part[pb][1]) + sh.epi_part[pb][2]) +
                                         sh.epi_part[pb][3];
                        a.item_part[(size_t)it.slot * a.P2 + j] = v;
                        fence_acq_rel_gpu();
                        const unsigned old = atomicAdd(a.done2 + it.chunk, 1u);
                        last = (old == (unsigned)a.P2 - 1u);
                    }
                    last = __shfl_sync(0xffffffffu, last, 0);
                    if (last) {
                        // last item of the chunk: per-shift and chunk sums in
                        // fixed order, then release the slot
                        fence_acq_rel_gpu();
                        const int per_x_items = 1 << ipx_log;
                        double cs = 0.0;
                        for (int qq = 0; qq < C; ++qq) {
                            const double *ip = a.item_part + ((size_t)it.slot * a.P2 + ((size_t)qq << ipx_log));
                            double sx = 0.0;
                            for (int kk = lane; kk < per_x_items; kk += 32) sx += __ldcg(ip + kk);
#pragma unroll
                            for (int o = 16; o > 0; o >>= 1) sx += __shfl_down_sync(0xffffffffu, sx, o);
                            const uint64_t xq = it.xc + (uint64_t)qq;
                            if (lane == 0 && a.per_x && x_valid(a, xq)) a.per_x[xq - a.x_begin] = sx;
                            cs += sx;
                        }
                        if (lane == 0) {
                            a.chunk_sum[it.chunk] = cs;
                            fence_acq_rel_gpu();
                            atomicExch(a.freed + it.chunk, 1u);
                        }
                    }
                } else {
                    ucount += ntiles;
                    dtile += ntiles;
                }
            }
        }
        // the MMA warp: its last accumulators of either kind are complete
        // before exit (the latest phase of each used barrier)
        if (is_mma) {
            for (int d = 0; d < kAcc; ++d) {
                if (mma_used & (1u << d))
                    mbar_wait_bounded(smem_u32(&sh.d_full[d]), ((par_d >> d) & 1u) ^ 1u, a.wait_ns);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kEpiWarp0) tc_dealloc(tmem, kTcCols);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point.
PFN_cuTensorMapEncodeTiled_v12000 tc_tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// The 16-bit scratch planes as a 2-D array: 8192 pieces (16 KB) per row,
// R * C * 2 * 2^h2 rows; boxes of 64 pieces (128 bytes, the swizzle span) by
// 2^h2 rows.
cudaError_t encode_tc_tmap(LargeArgs &a) {
    auto enc = tc_tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    if (((uintptr_t)a.scratch & 15)) return cudaErrorInvalidValue;
    const cuuint64_t rows = ((cuuint64_t)a.R << (a.C_log + 1)) << a.h2;
    if (rows > 0xFFFFFFFFull) return cudaErrorInvalidValue;
    const cuuint64_t dims[2] = {2ull * kTile, rows};
    const cuuint64_t strides[1] = {(cuuint64_t)kTile * 4};
    const cuuint32_t box[2] = {64u, 1u << a.h2};
    const cuuint32_t estr[2] = {1u, 1u};
    const CUresult r = enc(&a.tmap, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, a.scratch, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int H2, int KIND>
cudaError_t launch_tc_h(const LargeArgs &a, int grid, cudaStream_t st) {
    const size_t smem = tc_smem_bytes();
    auto kern = k_tc<H2, KIND>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    LargeArgs b = a;
    if ((e = encode_tc_tmap(b)) != cudaSuccess) return e;
    kern<<<grid, kTcThreads, smem, st>>>(b);
    return cudaGetLastError();
}

template <int KIND>
cudaError_t launch_tc(const LargeArgs &a, int grid, cudaStream_t st) {
    switch (a.h2) {
#define SRE_CASE(n) \
    case n: return launch_tc_h<n, KIND>(a, grid, st);
        SRE_CASE(3) SRE_CASE(4) SRE_CASE(5) SRE_CASE(6) SRE_CASE(7)
#undef SRE_CASE
        default: return cudaErrorNotSupported;
    }
}

}  // namespace

bool tc_applies(int N, int half, int alpha, const void *psi) {
    const int h2 = N - kTileBits - 1;
    return half && alpha == 2 && h2 >= kTcMinH2 && h2 <= kTcMaxH2 && ((uintptr_t)psi & 15) == 0;
}

cudaError_t launch_large_tc(const LargeArgs &a, const Workspace &ws, const DeviceInfo &dev, int grid,
                            cudaStream_t st, int tc_kind, int *e_buf, double *bn_buf, size_t buf_cap) {
    if (!a.half || a.alpha != 2) return cudaErrorInvalidValue;
    const int nb = 1 << (a.N - kTileBits);
    // states of the launch: one, or the states of a batch class
    const long long S = a.psis ? a.n_chunks / a.chunks_per_state : 1;
    if (S < 1 || S > 65535 || (a.psis && S * a.chunks_per_state != a.n_chunks)) return cudaErrorInvalidValue;
    int *tc_e = e_buf ? e_buf : ws.tc_e;
    double *tc_bn = e_buf ? bn_buf : ws.tc_bn;
    const size_t cap = e_buf ? buf_cap : (size_t)ws.tc_cap;
    if (!tc_e || !tc_bn || (size_t)S * nb > cap) return cudaErrorInvalidValue;
    k_tc_block_norms<<<dim3(nb, (unsigned)S), kThreads, 0, st>>>(reinterpret_cast<const float2 *>(a.psi), a.psis,
                                                                 tc_bn);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_tc_scales<<<dim3((nb + 127) / 128, (unsigned)S), 128, 0, st>>>(tc_bn, nb, tc_e);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ws.launches += 2;
    LargeArgs b = a;
    b.tc_e = tc_e;
    if (!b.psis) b.chunks_per_state = b.n_chunks;  // one state: every chunk is state 0
    grid = std::max(1, std::min(grid, dev.sms));  // one CTA per SM (all of TMEM)
    if (tc_kind != kTcBf16 && tc_kind != kTcFp16) return cudaErrorInvalidValue;
    // the profiling events bracket the tensor-core kernel alone
    if (ws.ev_begin && (e = cudaEventRecord(ws.ev_begin, st)) != cudaSuccess) return e;
    e = tc_kind == kTcBf16 ? launch_tc<kTcBf16>(b, grid, st) : launch_tc<kTcFp16>(b, grid, st);
    if (e != cudaSuccess) return e;
    if (ws.ev_end && (e = cudaEventRecord(ws.ev_end, st)) != cudaSuccess) return e;
    ws.main_kernel = tc_kind == kTcBf16 ? "k_tc<bf16>" : "k_tc<fp16>";
    return cudaSuccess;
}

bool tc_mode_available(sre_mode_t mode) {
    return mode == SRE_MODE_BF16_SPLIT || mode == SRE_MODE_FP16_SPLIT;
}

cudaError_t tc_enqueue_m2(const Workspace &ws, const DeviceInfo &dev, const void *d_state,
                          sre_dtype_t dtype, int N, uint64_t x_begin, uint64_t x_end,
                          sre_mode_t mode, cudaStream_t stream, double *d_m2, double *d_per_x,
                          long long wait_ns, LargeCfg *cfg_half, int alpha) {
    return enqueue_m2(ws, dev, d_state, dtype, N, x_begin, x_end, mode, stream, d_m2, d_per_x, wait_ns,
                      cfg_half, alpha);
}

}  // namespace sre
