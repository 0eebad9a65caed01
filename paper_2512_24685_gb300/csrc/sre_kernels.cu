// sre_kernels.cu -- CUDA-core XOR-FWHT path of libsre (FP32 and FP64).
//
// Algorithm 1 of the paper: for every shift x, form the XOR-shifted product
// g_x(t) = conj(phi_{t^x}) phi_t, transform it with the unnormalised FWHT over
// t (A_x(z) = <psi|X^x Z^z|psi>, Eq. (Pauli_expect)) and accumulate
// sum_z |A_x(z)|^4; M2 = -log2(S / (d n2^4)) (Eq. (final1), base 2).
//
// Kernels
//   k_convert   element-type conversion of the state (complex128 <-> complex64)
//   k_norm      n2 = <psi|psi> in FP64 + NaN/Inf detection (fixed grid)
//   k_small     N <= 12: one 2^12-entry tile holds 2^(12-N) whole shifts; the
//               state sits in shared memory; static tile->CTA assignment
//   k_large     N  > 12: persistent two-pass kernel.  Pass 1 (one work item
//               per chunk of C shifts and high index block t_h) forms the
//               products of a 2^12 block, transforms its 12 low bits and
//               writes the block to an L2-sized ring of scratch; pass 2 (work
//               items of whole-z-block tiles) gathers the 2^(N-12) blocks of
//               a z-range, transforms the high bits and reduces |A|^4.  Items
//               are claimed in order from one counter; pass 2 of a chunk waits
//               (bounded, %globaltimer) for its pass-1 items, and pass 1 of a
//               chunk waits for the ring slot to be released.
//   k_finalize  fixed-order FP64 sums of the partials, M2 and the status.
// Every reduction has a fixed order, so results are bitwise reproducible and
// do not depend on what else runs on the device.
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "sre_internal.h"
#include "sre_large.cuh"
#include "sre_tile.cuh"

namespace sre {
using namespace dev;

// ---------------------------------------------------------------- helpers

template <typename Out, typename In>
__global__ void k_convert(const In *__restrict__ src, Out *__restrict__ dst, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const In v = src[i];
        Out o;
        o.x = (decltype(o.x))v.x;
        o.y = (decltype(o.y))v.y;
        dst[i] = o;
    }
}

// n2 = sum_t |phi_t|^2 (FP64), per-block partials in a fixed grid.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_norm(const v2_t<R> *__restrict__ psi, uint64_t d,
                                                   double *__restrict__ npart,
                                                   int *__restrict__ flags) {
    __shared__ double red[kThreads / 32];
    double s = 0.0;
    int bad = 0;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < d;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const v2_t<R> v = psi[t];
        const double re = (double)v.x, im = (double)v.y;
        if (!isfinite(re) || !isfinite(im)) bad = 1;
        s += re * re + im * im;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, kFlagNonFinite);
    const double b = block_sum(s, red);
    if (threadIdx.x == 0) npart[blockIdx.x] = b;
}

// ------------------------------------------------------- N <= 12: k_small

// Tile g covers flat indices [g*4096, (g+1)*4096) of the (x - x_begin, t)
// space: x = x_begin + (flat >> N), t = flat & (d - 1).  The transform runs
// over the low NB = N bits of the tile index.
template <typename R, int NB>
__global__ void __launch_bounds__(kThreads) k_small(const v2_t<R> *__restrict__ psi,
                                                    const void *const *__restrict__ psis,
                                                    long long tiles_per_state,
                                                    uint64_t x_begin, uint64_t x_end,
                                                    long long ntiles,
                                                    double *__restrict__ part, int alpha) {
    // Single state: psis == nullptr.  Several states of the same N: psis[s] is
    // state s and tiles are numbered state-major.  Tile g's sum goes to
    // part[g] (fixed-order tree inside the tile), so a state's partials do not
    // depend on the grid or on the other states of a batch.
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using V = v2_t<R>;
    V *psi_s = reinterpret_cast<V *>(smem_raw);
    V *bufA = psi_s + kTileSlots;
    V *bufB = bufA + kTileSlots;
    __shared__ double red[kThreads / 32];
    constexpr int N = NB;
    constexpr int d = 1 << N;
    const int tid = threadIdx.x;

    long long cur = -1;
    for (long long g = blockIdx.x; g < ntiles; g += gridDim.x) {
        const long long sidx = psis ? g / tiles_per_state : 0;
        const long long gl = g - sidx * tiles_per_state;
        if (sidx != cur) {
            const V *src = psis ? reinterpret_cast<const V *>(psis[sidx]) : psi;
            __syncthreads();
            for (int t = tid; t < d; t += kThreads) psi_s[pad(t)] = src[t];
            __syncthreads();
            cur = sidx;
        }
        cx_t<R> v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const uint64_t flat = ((uint64_t)gl << kTileBits) | (uint64_t)elem<0>(tid, i);
            const uint64_t x = x_begin + (flat >> N);
            const int t = (int)(flat & (d - 1));
            if (x < x_end) {
                const V a = psi_s[pad(t)];
                const V b = psi_s[pad(t ^ (int)x)];
                v[i] = conj_mul<R>(b.x, b.y, a.x, a.y);  // conj(phi_{t^x}) * phi_t
            } else {
                v[i] = Cx<R>::zero();
            }
        }
        tile_fwht<NB, R>(v, bufA, bufB, tid);
        // block_sum's barriers also protect bufB before the next tile
        const double s = block_sum((double)sum_order<R, false>(v, alpha), red);
        if (tid == 0) part[g] = s;
    }
}

// ------------------------------------------------------------- finalize

// Fixed-order FP64 sum of two segments of partials by one warp: lane l adds
// entries l, l+32, ... of each segment in order, then a fixed shuffle tree.
// Shared by the single-state and the batch finalize, so a state's M2 is
// bitwise the same in either.
__device__ __forceinline__ double warp_sum_segments(const double *p, long long o1, long long n1,
                                                    long long o2, long long n2) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (long long k = lane; k < n1; k += 32) s += p[o1 + k];
    for (long long k = lane; k < n2; k += 32) s += p[o2 + k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    return s;  // valid in lane 0
}

__device__ __forceinline__ double m2_from(double S, double n2, int N, bool bad) {
    // M2 = -log2(S / (d n2^4)), in logs so tiny norms do not underflow
    return bad ? __longlong_as_double(0x7ff8000000000000ll)
               : -(log2(S) - (double)N - 4.0 * log2(n2));
}

// Eq. (sre) at integer order alpha: M_alpha = log2(S / (d n2^(2 alpha))) /
// (1 - alpha); order 2 is m2_from.
__device__ __forceinline__ double malpha_from(double S, double n2, int N, int alpha, bool bad) {
    if (alpha == 2) return m2_from(S, n2, N, bad);
    return bad ? __longlong_as_double(0x7ff8000000000000ll)
               : (log2(S) - (double)N - 2.0 * alpha * log2(n2)) / (1.0 - alpha);
}

// One warp: S from the partial segments [o1, o1+n1) and [o2, o2+n2), n2 from
// the norm partials, M2 and the status.
__global__ void k_finalize(const double *__restrict__ parts, long long o1, long long n1, long long o2,
                           long long n2c, const double *__restrict__ npart, int nn, int N,
                           const int *flags, const int *status, Result *res, double *d_m2,
                           int alpha) {
    const double S = warp_sum_segments(parts, o1, n1, o2, n2c);
    const double n2 = warp_sum_segments(npart, 0, nn, 0, 0);
    if (threadIdx.x == 0) {
        int st = *status;
        if (st == 0 && (*flags & kFlagNonFinite)) st = SRE_ENONFINITE;
        if (st == 0 && !(n2 > 0.0)) st = SRE_EZERO;
        const double m2 = malpha_from(S, n2, N, alpha, st != 0);
        res->m2 = m2;
        res->S = S;
        res->n2 = n2;
        res->status = st;
        if (d_m2) *d_m2 = m2;
    }
}

// M_alpha from a reduced sum and a norm (sums of shards added elsewhere).
__global__ void k_malpha_from_sums(const double *S, const double *n2, int N, int alpha, double *out) {
    const double s = *S, n = *n2;
    const bool bad = !(s > 0.0) || !(n > 0.0) || !isfinite(s) || !isfinite(n);
    *out = malpha_from(s, n, N, alpha, bad);
}

__global__ void k_copy_sums(const Result *res, double *out2) {
    out2[0] = res->S;
    out2[1] = res->n2;
}

// ------------------------------------------------------------ host side

cudaError_t query_device(DeviceInfo *info) {
    cudaError_t e = cudaGetDevice(&info->device);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&info->sms, cudaDevAttrMultiProcessorCount, info->device);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&info->l2_bytes, cudaDevAttrL2CacheSize, info->device);
    if (e != cudaSuccess) return e;
    return cudaDeviceGetAttribute(&info->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                  info->device);
}

static size_t tile_smem_bytes(int elem_bytes) { return (size_t)3 * kTileSlots * elem_bytes; }

// deterministic pseudo-random amplitudes for timing runs (values irrelevant)
template <typename V>
__global__ void k_fill_synthetic(V *p, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t h = (i + 1) * 0x9E3779B97F4A7C15ull;
        h ^= h >> 31;
        h *= 0xBF58476D1CE4E5B9ull;
        h ^= h >> 29;
        V v;
        v.x = (decltype(v.x))((double)(h & 0xFFFFFF) / 16777216.0 - 0.5);
        v.y = (decltype(v.y))((double)((h >> 24) & 0xFFFFFF) / 16777216.0 - 0.5);
        p[i] = v;
    }
}

cudaError_t enqueue_fill_synthetic(void *buf, int N, sre_dtype_t dtype, cudaStream_t st) {
    const uint64_t d = 1ull << N;
    const int grid = (int)std::min<uint64_t>((d + 255) / 256, 4096);
    if (dtype == SRE_C128)
        k_fill_synthetic<double2><<<grid, 256, 0, st>>>(reinterpret_cast<double2 *>(buf), d);
    else
        k_fill_synthetic<float2><<<grid, 256, 0, st>>>(reinterpret_cast<float2 *>(buf), d);
    return cudaGetLastError();
}

bool large_cfg_fits(const Workspace &ws, const LargeCfg &c, int N, int half) {
    if (c.C_log < 0 || c.C_log > 3 || c.R < 2 || c.R > kMaxRing || c.D < 1 || c.D >= c.R) return false;
    const int h2 = N - kTileBits - half;
    if (c.G2_log < 0 || c.G2_log > h2 || c.B1_log < 0 || c.B1_log > h2) return false;
    const size_t ring = (size_t)c.R * ((size_t)1 << c.C_log) * ((size_t)ws.elem_bytes << (N - half));
    const size_t P2 = ((size_t)1 << c.C_log) << (h2 - c.G2_log);
    return ring <= ws.scratch_bytes && (size_t)c.R * P2 * 8 <= ws.item_part_cap;
}

// Ring / chunk configuration for the two-pass kernel.  About grid / P1
// chunks are in pass 1 at any time (P1 = 2^h2 items per chunk), so pass 2
// lags D = that + 1 chunks behind and the ring holds R = 2 D + 1 chunks:
// pass-2 items then find their chunk finished and pass-1 items find their
// slot free.  The chunk size C (shifts sharing one pass-1 partner block) is
// the largest power of two up to 8 whose ring R * C * elem * 2^(N - half)
// stays within 60% of L2, so the inter-pass traffic stays on chip.
LargeCfg choose_large_cfg(const DeviceInfo &dev, int N, int elem_bytes, int half) {
    LargeCfg c;
    const int h2 = N - kTileBits - half;
    const double per_x = (double)elem_bytes * (double)(1ull << (N - half));
    const double budget = std::max(24.0 * (1 << 20), 0.6 * (double)dev.l2_bytes);
    const int occ = elem_bytes == 8 ? 2 : 1;
    c.grid = std::max(1, dev.sms * occ);
    const int P1 = 1 << h2;
    const int inflight = (c.grid + P1 - 1) / P1;
    c.D = std::min(inflight + 1, kMaxRing / 2 - 1);
    c.R = 2 * c.D + 1;
    int C_log = 3;
    while (C_log > 0 && (double)c.R * (double)(1 << C_log) * per_x > budget) --C_log;
    c.C_log = C_log;
    c.G2_log = std::min(C_log, h2);
    // pass 2 staged through TMA (FP32, 5 <= h2 <= 8) overlaps the copy of
    // tile g + 2 with tile g: give each item four tiles or more
    c.stage1 = 1;
    c.stage2 = 1;
    if (elem_bytes == 8 && h2 >= 5 && h2 <= 8) c.G2_log = std::min(C_log + 2, h2);
    c.B1_log = 0;
    return c;
}

size_t workspace_scratch_bytes(const DeviceInfo &dev, int N_max, int elem_bytes, sre_mode_t mode) {
    (void)mode;
    if (N_max <= kTileBits) return 0;
    size_t b = 0;
    for (int half = 0; half <= 1; ++half) {
        const LargeCfg c = choose_large_cfg(dev, N_max, elem_bytes, half);
        b = std::max(b, (size_t)c.R * ((size_t)1 << c.C_log) * ((size_t)elem_bytes << (N_max - half)));
    }
    return b;
}

void workspace_free(Workspace *ws) {
    if (ws->ev_begin) cudaEventDestroy(ws->ev_begin);
    if (ws->ev_end) cudaEventDestroy(ws->ev_end);
    cudaFree(ws->npart);
    cudaFree(ws->flags);
    cudaFree(ws->part);
    cudaFree(ws->scratch);
    cudaFree(ws->item_part);
    cudaFree(ws->chunk_sum);
    cudaFree(ws->counters);
    cudaFree(ws->work);
    cudaFree(ws->status);
    cudaFree(ws->result);
    cudaFree(ws->conv);
    cudaFree(ws->tc_e);
    cudaFree(ws->tc_bn);
    *ws = Workspace();
}

cudaError_t workspace_alloc(Workspace *ws, const DeviceInfo &dev, int N_max, int elem_bytes,
                            sre_mode_t mode, size_t scratch_floor) {
    (void)mode;
    *ws = Workspace();
    ws->N_max = N_max;
    ws->elem_bytes = elem_bytes;
    cudaError_t e;
#define SRE_TRY(x)                  \
    do {                            \
        e = (x);                    \
        if (e != cudaSuccess) {     \
            workspace_free(ws);     \
            return e;               \
        }                           \
    } while (0)
    SRE_TRY(cudaMalloc(&ws->npart, sizeof(double) * kNormBlocks));
    SRE_TRY(cudaMalloc(&ws->flags, sizeof(int)));
    ws->part_cap = kTile;  // one partial per tile of an N <= 12 state
    SRE_TRY(cudaMalloc(&ws->part, sizeof(double) * ws->part_cap));
    SRE_TRY(cudaMalloc(&ws->work, sizeof(unsigned long long) * 2));
    SRE_TRY(cudaMalloc(&ws->status, sizeof(int)));
    SRE_TRY(cudaMalloc(&ws->result, sizeof(Result)));
    if (N_max > kTileBits) {
        // sizes for every N up to N_max and both halves of the shift range,
        // with room for tuned configurations: chunks of a single shift, up to
        // kMaxRing ring slots, a scratch ring of at least scratch_floor bytes
        size_t scratch = scratch_floor, item_cap = 0, chunk_cap = 0;
        for (int n = kTileBits + 1; n <= N_max; ++n) {
            for (int half = 0; half <= 1; ++half) {
                const LargeCfg c = choose_large_cfg(dev, n, elem_bytes, half);
                const int h2 = n - kTileBits - half;
                scratch = std::max(scratch, (size_t)c.R * ((size_t)1 << c.C_log) *
                                                ((size_t)elem_bytes << (n - half)));
                // R * P2 per-warp partials (8 warps, P2 <= 8 * 2^h2)
                item_cap = std::max(item_cap, (size_t)std::max(c.R, kMaxRing) * ((size_t)8 << h2) * 8);
            }
            chunk_cap = std::max(chunk_cap, ((size_t)1 << n) + 4);
        }
        ws->scratch_bytes = scratch;
        ws->item_part_cap = item_cap;
        ws->chunk_cap = chunk_cap;
        SRE_TRY(cudaMalloc(&ws->scratch, scratch));
        SRE_TRY(cudaMalloc(&ws->item_part, sizeof(double) * item_cap));
        SRE_TRY(cudaMalloc(&ws->chunk_sum, sizeof(double) * chunk_cap));
        SRE_TRY(cudaMalloc(&ws->counters, sizeof(unsigned) * 3 * chunk_cap));
        ws->tc_cap = 1 << (N_max - kTileBits);
        SRE_TRY(cudaMalloc(&ws->tc_e, sizeof(int) * ws->tc_cap));
        SRE_TRY(cudaMalloc(&ws->tc_bn, sizeof(double) * ws->tc_cap));
    }
#undef SRE_TRY
    return cudaSuccess;
}

template <typename R, int NB>
static cudaError_t launch_small_nb(const void *psi, const void *const *psis, int nstates,
                                   uint64_t x_begin, uint64_t x_end, double *part, int part_cap,
                                   const DeviceInfo &dev, cudaStream_t st, int *nparts,
                                   int forced_grid = 0, int alpha = 2) {
    const size_t smem = tile_smem_bytes(sizeof(v2_t<R>));
    auto kern = k_small<R, NB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const uint64_t flat = (x_end - x_begin) << NB;
    const long long tps = (long long)((flat + kTile - 1) >> kTileBits);
    const long long ntiles = tps * nstates;
    if (ntiles > part_cap) return cudaErrorInvalidValue;
    const int occ = sizeof(R) == 4 ? 2 : 1;
    const int grid = forced_grid > 0 ? forced_grid
                                     : (int)std::min<long long>(ntiles, (long long)dev.sms * occ);
    if (grid < 1) return cudaErrorInvalidValue;
    kern<<<grid, kThreads, smem, st>>>(reinterpret_cast<const v2_t<R> *>(psi), psis, tps, x_begin,
                                       x_end, ntiles, part, alpha);
    *nparts = (int)ntiles;
    return cudaGetLastError();
}

template <typename R>
static cudaError_t launch_small(int N, const void *psi, const void *const *psis, int nstates,
                                uint64_t xb, uint64_t xe, double *part, int part_cap,
                                const DeviceInfo &dev, cudaStream_t st, int *nparts,
                                int forced_grid = 0, int alpha = 2) {
    switch (N) {
#define SRE_CASE(n) \
    case n: return launch_small_nb<R, n>(psi, psis, nstates, xb, xe, part, part_cap, dev, st, nparts, forced_grid, alpha);
        SRE_CASE(1) SRE_CASE(2) SRE_CASE(3) SRE_CASE(4) SRE_CASE(5) SRE_CASE(6)
        SRE_CASE(7) SRE_CASE(8) SRE_CASE(9) SRE_CASE(10) SRE_CASE(11) SRE_CASE(12)
#undef SRE_CASE
        default: return cudaErrorInvalidValue;
    }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// dependency on the driver library).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
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

// The scratch ring of a launch as a 2-D FP32 array: 8192 columns (the 4096
// complex entries of one block t'_h) by R * C * 2^h2 rows, 32 KB apart; boxes
// of 32 FP32 columns (128 bytes, the swizzle span) by 2^h2 rows.
cudaError_t encode_p2_tmap(LargeArgs &a) {
    auto enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    if (a.h2 < 5 || a.h2 > 8 || ((uintptr_t)a.scratch & 15)) return cudaErrorInvalidValue;
    const cuuint64_t rows = (cuuint64_t)a.R << (a.C_log + a.h2);
    if (rows > 0xFFFFFFFFull) return cudaErrorInvalidValue;
    const cuuint64_t dims[2] = {2ull * kTile, rows};
    const cuuint64_t strides[1] = {(cuuint64_t)kTile * sizeof(float2)};
    const cuuint32_t box[2] = {32u, 1u << a.h2};
    const cuuint32_t estr[2] = {1u, 1u};
    const CUresult r = enc(&a.tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, a.scratch, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <typename R, int H2, bool HALF>
static cudaError_t launch_large_h(const LargeArgs &a, int grid, cudaStream_t st) {
    const size_t smem = large_smem_bytes<R, H2>();
    auto kern = k_large<R, H2, HALF>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if constexpr (large_uses_tma<R, H2>()) {
        LargeArgs b = a;
        if ((e = encode_p2_tmap(b)) != cudaSuccess) return e;
        kern<<<grid, kThreads, smem, st>>>(b);
    } else {
        kern<<<grid, kThreads, smem, st>>>(a);
    }
    return cudaGetLastError();
}

template <typename R, bool HALF>
static cudaError_t launch_large(const LargeArgs &a, int grid, cudaStream_t st) {
    switch (a.h2) {
#define SRE_CASE(n) \
    case n: return launch_large_h<R, n, HALF>(a, grid, st);
        SRE_CASE(0) SRE_CASE(1) SRE_CASE(2) SRE_CASE(3) SRE_CASE(4) SRE_CASE(5) SRE_CASE(6)
        SRE_CASE(7) SRE_CASE(8) SRE_CASE(9) SRE_CASE(10) SRE_CASE(11) SRE_CASE(12)
#undef SRE_CASE
        default: return cudaErrorInvalidValue;
    }
}

// Fill LargeArgs for the shift range [xb, xe) (all of it halved or not).
static cudaError_t make_large_args(LargeArgs *a, const Workspace &ws, const DeviceInfo &dev,
                                   const void *psi, int N, uint64_t xb, uint64_t xe, int half,
                                   int elem_bytes, size_t chunk_off, double *per_x,
                                   long long wait_ns, const LargeCfg *ovr, int *grid) {
    const LargeCfg c = ovr ? *ovr : choose_large_cfg(dev, N, elem_bytes, half);
    LargeArgs &A = *a;
    A.psi = psi;
    A.psis = nullptr;
    A.chunks_per_state = 0;
    A.N = N;
    A.half = half;
    A.h2 = N - kTileBits - half;
    A.x_begin = xb;
    A.x_end = xe;
    A.C_log = c.C_log;
    A.R = c.R;
    A.G2_log = std::min(c.G2_log, A.h2);
    A.x0 = xb & ~((1ull << c.C_log) - 1);
    A.n_chunks = (long long)((xe - A.x0 + (1ull << c.C_log) - 1) >> c.C_log);
    A.D = (int)std::max<long long>(1, std::min<long long>(std::min(c.D, c.R - 1), A.n_chunks));
    if (A.R < 2) return cudaErrorInvalidValue;
    A.B1_log = std::max(0, std::min(c.B1_log, A.h2));
    A.stage1 = c.stage1;
    A.stage2 = c.stage2;
    A.alpha = 2;
    A.P1 = 1 << (A.h2 - A.B1_log);
    A.P2 = (1 << c.C_log) << (A.h2 - A.G2_log);
    A.n_items = A.n_chunks * (long long)(A.P1 + A.P2);
    const size_t need_scratch = (size_t)c.R * ((size_t)1 << c.C_log) * ((size_t)elem_bytes << (N - half));
    if (need_scratch > ws.scratch_bytes || chunk_off + (size_t)A.n_chunks > ws.chunk_cap ||
        (size_t)c.R * A.P2 * 8 > ws.item_part_cap)
        return cudaErrorInvalidValue;
    A.scratch = ws.scratch;
    A.item_part = ws.item_part;
    A.chunk_sum = ws.chunk_sum + chunk_off;
    A.done1 = ws.counters + chunk_off;
    A.done2 = ws.counters + ws.chunk_cap + chunk_off;
    A.freed = ws.counters + 2 * ws.chunk_cap + chunk_off;
    A.work = ws.work + (half ? 1 : 0);
    A.per_x = per_x;
    A.status = ws.status;
    A.wait_ns = wait_ns;
    *grid = (int)std::max<long long>(1, std::min<long long>(c.grid, A.n_items));
    return cudaSuccess;
}

cudaError_t enqueue_copy_sums(const Workspace &ws, double *d_out2, cudaStream_t stream) {
    k_copy_sums<<<1, 1, 0, stream>>>(ws.result, d_out2);
    return cudaGetLastError();
}

template <typename R>
static cudaError_t enqueue_m2_t(const Workspace &ws, const DeviceInfo &dev, const void *psi, int N,
                                uint64_t x_begin, uint64_t x_end, cudaStream_t st, double *d_m2,
                                double *d_per_x, long long wait_ns, LargeCfg *cfg_override,
                                int tc_kind, int alpha) {
    cudaError_t e;
    const uint64_t d = 1ull << N;
    if ((e = cudaMemsetAsync(ws.flags, 0, sizeof(int), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ws.status, 0, sizeof(int), st)) != cudaSuccess) return e;
    k_norm<R><<<kNormBlocks, kThreads, 0, st>>>(reinterpret_cast<const v2_t<R> *>(psi), d, ws.npart,
                                                ws.flags);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ws.launches += 2;  // k_norm + k_finalize
    const double *parts = nullptr;
    long long nparts = 0, seg1 = 0;  // large path: [0, seg1) full shifts, [seg1, nparts) halved
    if (N <= kTileBits) {
        int np = 0;
        if (ws.ev_begin && (e = cudaEventRecord(ws.ev_begin, st)) != cudaSuccess) return e;
        if ((e = launch_small<R>(N, psi, nullptr, 1, x_begin, x_end, ws.part, ws.part_cap, dev, st,
                                 &np, 0, alpha)) != cudaSuccess)
            return e;
        if (ws.ev_end && (e = cudaEventRecord(ws.ev_end, st)) != cudaSuccess) return e;
        ws.main_kernel = "k_small";
        ws.launches += 1;
        parts = ws.part;
        nparts = np;
        seg1 = np;
    } else {
        // shifts below 4096 (pivot bit inside the 12-bit block): full
        // transform; shifts from 4096 up: conjugate-symmetry halving
        const int eb = (int)sizeof(v2_t<R>);
        const uint64_t split = std::min<uint64_t>(std::max<uint64_t>(x_begin, kTile), x_end);
        if ((e = cudaMemsetAsync(ws.counters, 0, sizeof(unsigned) * 3 * ws.chunk_cap, st)) != cudaSuccess)
            return e;
        if ((e = cudaMemsetAsync(ws.work, 0, sizeof(unsigned long long) * 2, st)) != cudaSuccess) return e;
        size_t chunks = 0;
        for (int half = 0; half <= 1; ++half) {
            const uint64_t xb = half ? split : x_begin;
            const uint64_t xe = half ? x_end : split;
            if (xb >= xe) continue;
            const bool tc_here = tc_kind && tc_applies(N, half, alpha, psi);
            // the profiling events bracket the dominant launch: the halved
            // shifts, or the full-transform range when there are none
            const bool timed = half == 1 || split >= x_end;
            if (timed && !tc_here && ws.ev_begin && (e = cudaEventRecord(ws.ev_begin, st)) != cudaSuccess)
                return e;
            if (!tc_here && mid_applies(N, half, eb)) {
                // one or two blocks per shift: single pass, one partial per shift
                const long long ns = (long long)(xe - xb);
                if (chunks + (size_t)ns > ws.chunk_cap) return cudaErrorInvalidValue;
                if ((e = launch_mid<R>(N, half, psi, nullptr, 1, ns, xb, alpha, ws.chunk_sum + chunks,
                                       d_per_x ? d_per_x + (xb - x_begin) : nullptr, dev, st)) != cudaSuccess)
                    return e;
                if (timed && ws.ev_end && (e = cudaEventRecord(ws.ev_end, st)) != cudaSuccess) return e;
                if (timed) ws.main_kernel = "k_mid";
                ws.launches += 1;
                chunks += (size_t)ns;
                if (!half) seg1 = (long long)chunks;
                continue;
            }
            LargeArgs a;
            int grid = 0;
            if ((e = make_large_args(&a, ws, dev, psi, N, xb, xe, half, eb, chunks,
                                     d_per_x ? d_per_x + (xb - x_begin) : nullptr, wait_ns,
                                     cfg_override && half ? cfg_override : nullptr, &grid)) != cudaSuccess)
                return e;
            a.alpha = alpha;
            if (tc_here)
                e = launch_large_tc(a, ws, dev, grid, st, tc_kind);
            else if (half)
                e = launch_large<R, true>(a, grid, st);
            else
                e = launch_large<R, false>(a, grid, st);
            if (e != cudaSuccess) return e;
            if (timed && !tc_here) {
                if (ws.ev_end && (e = cudaEventRecord(ws.ev_end, st)) != cudaSuccess) return e;
                ws.main_kernel = "k_large";
            }
            ws.launches += 1;
            chunks += (size_t)a.n_chunks;
            if (!half) seg1 = (long long)chunks;
        }
        parts = ws.chunk_sum;
        nparts = (long long)chunks;
    }
    k_finalize<<<1, 32, 0, st>>>(parts, 0, seg1, seg1, nparts - seg1, ws.npart, kNormBlocks, N,
                                 ws.flags, ws.status, ws.result, d_m2, alpha);
    return cudaGetLastError();
}

// M2 of one complex64 state in FP32 with fixed two-pass configurations for
// both shift ranges (no allocation, no autotuning): used by callers that
// hand in preassigned scratch.  It shares the norm and finalize kernels
// with the single-state path and, like it, takes the single-pass kernel for
// the shift ranges of N = 13..15; larger N run the two-pass kernel with the
// given fixed configuration (no autotuned plan).
cudaError_t enqueue_m2_fixed(const Workspace &ws, const DeviceInfo &dev, const void *psi, int N,
                             const LargeCfg &cfg_full, const LargeCfg &cfg_half, cudaStream_t st,
                             double *d_m2, long long wait_ns) {
    using R = float;
    cudaError_t e;
    const uint64_t d = 1ull << N;
    if ((e = cudaMemsetAsync(ws.flags, 0, sizeof(int), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ws.status, 0, sizeof(int), st)) != cudaSuccess) return e;
    k_norm<R><<<kNormBlocks, kThreads, 0, st>>>(reinterpret_cast<const v2_t<R> *>(psi), d, ws.npart,
                                                ws.flags);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    long long nparts = 0, seg1 = 0;
    const double *parts = nullptr;
    if (N <= kTileBits) {
        int np = 0;
        if ((e = launch_small<R>(N, psi, nullptr, 1, 0, d, ws.part, ws.part_cap, dev, st, &np)) != cudaSuccess)
            return e;
        parts = ws.part;
        nparts = seg1 = np;
    } else {
        if ((e = cudaMemsetAsync(ws.counters, 0, sizeof(unsigned) * 3 * ws.chunk_cap, st)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(ws.work, 0, sizeof(unsigned long long) * 2, st)) != cudaSuccess) return e;
        size_t chunks = 0;
        for (int half = 0; half <= 1; ++half) {
            const uint64_t xb = half ? (uint64_t)kTile : 0, xe = half ? d : (uint64_t)kTile;
            if (mid_applies(N, half, 8)) {
                // one, two or four blocks per shift: the single-pass kernel,
                // one partial per shift, no ring and no waits
                const long long ns = (long long)(xe - xb);
                if (chunks + (size_t)ns > ws.chunk_cap) return cudaErrorInvalidValue;
                if ((e = launch_mid<R>(N, half, psi, nullptr, 1, ns, xb, 2, ws.chunk_sum + chunks, nullptr, dev,
                                       st)) != cudaSuccess)
                    return e;
                chunks += (size_t)ns;
                if (!half) seg1 = (long long)chunks;
                continue;
            }
            LargeArgs a;
            int grid = 0;
            if ((e = make_large_args(&a, ws, dev, psi, N, xb, xe, half, 8, chunks, nullptr, wait_ns,
                                     half ? &cfg_half : &cfg_full, &grid)) != cudaSuccess)
                return e;
            e = half ? launch_large<R, true>(a, grid, st) : launch_large<R, false>(a, grid, st);
            if (e != cudaSuccess) return e;
            chunks += (size_t)a.n_chunks;
            if (!half) seg1 = (long long)chunks;
        }
        parts = ws.chunk_sum;
        nparts = (long long)chunks;
    }
    k_finalize<<<1, 32, 0, st>>>(parts, 0, seg1, seg1, nparts - seg1, ws.npart, kNormBlocks, N, ws.flags,
                                 ws.status, ws.result, d_m2, 2);
    return cudaGetLastError();
}

cudaError_t enqueue_m2(const Workspace &ws, const DeviceInfo &dev, const void *d_state,
                       sre_dtype_t dtype, int N, uint64_t x_begin, uint64_t x_end,
                       sre_mode_t mode, cudaStream_t stream, double *d_m2, double *d_per_x,
                       long long wait_ns, LargeCfg *cfg_override, int alpha) {
    const bool fp64 = (mode == SRE_MODE_FP64);
    const int want = fp64 ? SRE_C128 : SRE_C64;
    const void *psi = d_state;
    const uint64_t d = 1ull << N;
    if ((int)dtype != want) {
        const size_t need = (size_t)d * (fp64 ? 16 : 8);
        if (!ws.conv || ws.conv_bytes < need) return cudaErrorInvalidValue;
        const int grid = (int)std::min<uint64_t>((d + kThreads - 1) / kThreads, 4096);
        if (fp64)
            k_convert<double2, float2><<<grid, kThreads, 0, stream>>>(
                reinterpret_cast<const float2 *>(d_state), reinterpret_cast<double2 *>(ws.conv), d);
        else
            k_convert<float2, double2><<<grid, kThreads, 0, stream>>>(
                reinterpret_cast<const double2 *>(d_state), reinterpret_cast<float2 *>(ws.conv), d);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        ws.launches += 1;
        psi = ws.conv;
    }
    const int tc_kind = mode == SRE_MODE_BF16_SPLIT ? 1 : mode == SRE_MODE_FP16_SPLIT ? 2 : 0;
    if (fp64)
        return enqueue_m2_t<double>(ws, dev, psi, N, x_begin, x_end, stream, d_m2, d_per_x, wait_ns,
                                    cfg_override, 0, alpha);
    return enqueue_m2_t<float>(ws, dev, psi, N, x_begin, x_end, stream, d_m2, d_per_x, wait_ns,
                               cfg_override, tc_kind, alpha);
}

// --------------------------------------------------------- wait self test

// One thread waits on a counter nothing increments; records the outcome.
__global__ void k_wait_selftest(const unsigned *counter, int *status, long long wait_ns) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        if (wait_counter(counter, 1u, status, wait_ns)) atomicCAS(status, 0, -1);
    }
}

cudaError_t run_wait_selftest(long long wait_ns, cudaStream_t st, int *status_out) {
    unsigned *counter = nullptr;
    int *status = nullptr;
    cudaError_t e = cudaMalloc(&counter, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        k_wait_selftest<<<1, 32, 0, st>>>(counter, status, wait_ns);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(status_out, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(counter);
    cudaFree(status);
    return e;
}

// ------------------------------------------------------------------ batch

// n2 of several states (state s = blockIdx.y, its size from Ns[s]);
// partials in npart[s * kNormBlocks + b], flags[s] |= non-finite.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_norm_batch(const void *const *__restrict__ psis,
                                                         const int *__restrict__ Ns,
                                                         double *__restrict__ npart,
                                                         int *__restrict__ flags) {
    __shared__ double red[kThreads / 32];
    const int sidx = blockIdx.y;
    const v2_t<R> *psi = reinterpret_cast<const v2_t<R> *>(psis[sidx]);
    const uint64_t d = 1ull << Ns[sidx];
    double s = 0.0;
    int bad = 0;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < d;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const v2_t<R> v = psi[t];
        const double re = (double)v.x, im = (double)v.y;
        if (!isfinite(re) || !isfinite(im)) bad = 1;
        s += re * re + im * im;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags + sidx, kFlagNonFinite);
    const double b = block_sum(s, red);
    if (threadIdx.x == 0) npart[(size_t)sidx * gridDim.x + blockIdx.x] = b;
}

// M2 of every state of a batch: one warp per state, the same fixed-order
// segment sums as the single-state finalize (seg = {off1, n1, off2, n2}).
// status_out (may be null) receives each state's status with the same
// precedence as k_finalize: the batch's device-wait status first, then a
// non-finite amplitude, then a zero norm.
__global__ void k_finalize_batch(const longlong4 *__restrict__ seg, const double *__restrict__ parts,
                                 const double *__restrict__ npart, int nnorm,
                                 const int *__restrict__ flags, const int *__restrict__ Ns,
                                 const int *__restrict__ out_index, int count, const int *status,
                                 double *__restrict__ m2_out, int *__restrict__ status_out) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= count) return;
    const longlong4 g = seg[w];
    const double S = warp_sum_segments(parts, g.x, g.y, g.z, g.w);
    const double n = warp_sum_segments(npart, (long long)w * nnorm, nnorm, 0, 0);
    if ((threadIdx.x & 31) == 0) {
        int st = *status;
        if (st == 0 && (flags[w] & kFlagNonFinite)) st = SRE_ENONFINITE;
        if (st == 0 && !(n > 0.0)) st = SRE_EZERO;
        m2_out[out_index[w]] = m2_from(S, n, Ns[w], st != 0);
        if (status_out) status_out[out_index[w]] = st;
    }
}

template <typename R>
static size_t small_grid_for(const DeviceInfo &dev, int N, int S) {
    const uint64_t flat = (1ull << N) << N;
    const long long tps = (long long)((flat + kTile - 1) >> kTileBits);
    const int occ = sizeof(R) == 4 ? 2 : 1;
    return (size_t)std::min<long long>(tps * S, (long long)dev.sms * occ);
}

BatchClass batch_class_layout(const DeviceInfo &dev, const Workspace &ws, int N, int S,
                              sre_mode_t mode, const LargeCfg *tuned_half) {
    BatchClass L;
    L.N = N;
    L.S = S;
    const int eb = mode == SRE_MODE_FP64 ? 16 : 8;
    if (N <= kTileBits) {
        L.small_grid = (int)(eb == 8 ? small_grid_for<float>(dev, N, S) : small_grid_for<double>(dev, N, S));
        const long long tps = (long long)((((1ull << N) << N) + kTile - 1) >> kTileBits);
        L.cps_full = tps;  // tiles (= partials) per state
        L.parts_n = (size_t)S * (size_t)tps;
        return L;
    }
    L.cfg_full = choose_large_cfg(dev, N, eb, 0);
    L.cfg_half = tuned_half ? *tuned_half : choose_large_cfg(dev, N, eb, 1);
    // ranges taken by the single-pass kernel have one partial per shift
    if (mid_applies(N, 0, eb)) L.cfg_full.C_log = 0;
    if (mid_applies(N, 1, eb)) L.cfg_half.C_log = 0;
    L.cps_full = (long long)(((uint64_t)kTile + (1ull << L.cfg_full.C_log) - 1) >> L.cfg_full.C_log);
    const uint64_t span = (1ull << N) - kTile;
    L.cps_half = (long long)((span + (1ull << L.cfg_half.C_log) - 1) >> L.cfg_half.C_log);
    L.parts_n = (size_t)S * (size_t)(L.cps_full + L.cps_half);
    L.chunks_max = (size_t)S * (size_t)std::max(L.cps_full, L.cps_half);
    (void)ws;
    return L;
}

template <typename R>
static cudaError_t enqueue_batch_class_t(const Workspace &ws, const DeviceInfo &dev,
                                         const BatchClass &L, const void *const *d_ptrs,
                                         double *parts, unsigned *counters, size_t chunk_cap,
                                         cudaStream_t st, long long wait_ns, int *tc_e, double *tc_bn,
                                         size_t tc_cap) {
    cudaError_t e;
    const int N = L.N;
    if (N <= kTileBits) {
        int np = 0;
        e = launch_small<R>(N, nullptr, d_ptrs, L.S, 0, 1ull << N, parts + L.parts_off,
                            (int)L.parts_n, dev, st, &np, L.small_grid);
        ws.launches += 1;
        return e;
    }
    size_t off = L.parts_off;
    for (int half = 0; half <= 1; ++half) {
        const LargeCfg &c = half ? L.cfg_half : L.cfg_full;
        const long long cps = half ? L.cps_half : L.cps_full;
        const uint64_t xb = half ? (uint64_t)kTile : 0, xe = half ? (1ull << N) : (uint64_t)kTile;
        if (mid_applies(N, half, (int)sizeof(v2_t<R>))) {
            // cps = shifts per state (the layout gave this range one chunk per shift)
            if ((e = launch_mid<R>(N, half, nullptr, d_ptrs, L.S, cps, xb, 2, parts + off, nullptr, dev, st)) !=
                cudaSuccess)
                return e;
            ws.launches += 1;
            off += (size_t)cps * L.S;
            continue;
        }
        if (!large_cfg_fits(ws, c, N, half)) return cudaErrorInvalidValue;
        LargeArgs A;
        A.psi = nullptr;
        A.psis = d_ptrs;
        A.chunks_per_state = cps;
        A.N = N;
        A.half = half;
        A.h2 = N - kTileBits - half;
        A.x_begin = xb;
        A.x_end = xe;
        A.x0 = xb;  // kTile and 0 are chunk-aligned
        A.C_log = c.C_log;
        A.R = c.R;
        A.G2_log = std::min(c.G2_log, A.h2);
        A.B1_log = std::max(0, std::min(c.B1_log, A.h2));
        A.stage1 = c.stage1;
        A.stage2 = c.stage2;
        A.alpha = 2;
        A.n_chunks = cps * L.S;
        A.D = (int)std::max<long long>(1, std::min<long long>(std::min(c.D, c.R - 1), A.n_chunks));
        A.P1 = 1 << (A.h2 - A.B1_log);
        A.P2 = (1 << c.C_log) << (A.h2 - A.G2_log);
        A.n_items = A.n_chunks * (long long)(A.P1 + A.P2);
        if ((size_t)A.n_chunks > chunk_cap || (size_t)A.R * A.P2 * 8 > ws.item_part_cap)
            return cudaErrorInvalidValue;
        A.scratch = ws.scratch;
        A.item_part = ws.item_part;
        A.chunk_sum = parts + off;
        A.done1 = counters;
        A.done2 = counters + chunk_cap;
        A.freed = counters + 2 * chunk_cap;
        A.work = ws.work;
        A.per_x = nullptr;
        A.status = ws.status;
        A.wait_ns = wait_ns;
        if ((e = cudaMemsetAsync(counters, 0, sizeof(unsigned) * 3 * chunk_cap, st)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(ws.work, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
        const int grid = (int)std::max<long long>(1, std::min<long long>(c.grid, A.n_items));
        if (half && L.tc_kind)
            e = launch_large_tc(A, ws, dev, grid, st, L.tc_kind, tc_e, tc_bn, tc_cap);
        else
            e = half ? launch_large<R, true>(A, grid, st) : launch_large<R, false>(A, grid, st);
        if (e != cudaSuccess) return e;
        ws.launches += 1;
        off += (size_t)A.n_chunks;
    }
    return cudaSuccess;
}

cudaError_t enqueue_batch_class(const Workspace &ws, const DeviceInfo &dev, const BatchClass &L,
                                const void *const *d_ptrs, double *parts, unsigned *counters,
                                size_t chunk_cap, sre_mode_t mode, cudaStream_t st,
                                long long wait_ns, int *tc_e, double *tc_bn, size_t tc_cap) {
    if (mode == SRE_MODE_FP64)
        return enqueue_batch_class_t<double>(ws, dev, L, d_ptrs, parts, counters, chunk_cap, st, wait_ns, nullptr,
                                             nullptr, 0);
    return enqueue_batch_class_t<float>(ws, dev, L, d_ptrs, parts, counters, chunk_cap, st, wait_ns, tc_e, tc_bn,
                                        tc_cap);
}

cudaError_t enqueue_batch_norm(const Workspace &ws, const void *const *d_ptrs, const int *d_Ns,
                               int count, double *npart, int *flags, sre_mode_t mode,
                               cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(flags, 0, sizeof(int) * count, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ws.status, 0, sizeof(int), st)) != cudaSuccess) return e;
    const dim3 grid(kNormBlocks, count);
    if (mode == SRE_MODE_FP64)
        k_norm_batch<double><<<grid, kThreads, 0, st>>>(d_ptrs, d_Ns, npart, flags);
    else
        k_norm_batch<float><<<grid, kThreads, 0, st>>>(d_ptrs, d_Ns, npart, flags);
    ws.launches += 1;
    return cudaGetLastError();
}

cudaError_t enqueue_batch_finalize(const Workspace &ws, const void *seg, const double *parts,
                                   const double *npart, const int *flags, const int *d_Ns,
                                   const int *d_out_index, int count, double *m2_out,
                                   int *status_out, cudaStream_t st) {
    const int threads = 256;
    const int blocks = (count * 32 + threads - 1) / threads;
    k_finalize_batch<<<blocks, threads, 0, st>>>(reinterpret_cast<const longlong4 *>(seg), parts, npart,
                                                 kNormBlocks, flags, d_Ns, d_out_index, count,
                                                 ws.status, m2_out, status_out);
    ws.launches += 1;
    return cudaGetLastError();
}

cudaError_t enqueue_malpha_from_sums(const double *S, const double *n2, int N, int alpha, double *out,
                                     cudaStream_t st) {
    k_malpha_from_sums<<<1, 1, 0, st>>>(S, n2, N, alpha, out);
    return cudaGetLastError();
}

cudaError_t enqueue_convert(const void *src, sre_dtype_t from, void *dst, int N, cudaStream_t st) {
    const uint64_t d = 1ull << N;
    const int grid = (int)std::min<uint64_t>((d + kThreads - 1) / kThreads, 4096);
    if (from == SRE_C64)
        k_convert<double2, float2><<<grid, kThreads, 0, st>>>(reinterpret_cast<const float2 *>(src),
                                                              reinterpret_cast<double2 *>(dst), d);
    else
        k_convert<float2, double2><<<grid, kThreads, 0, st>>>(reinterpret_cast<const double2 *>(src),
                                                              reinterpret_cast<float2 *>(dst), d);
    return cudaGetLastError();
}

}  // namespace sre
