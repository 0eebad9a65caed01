// sre_noalloc.cu -- sre_m2_noalloc: M2 without any device or host allocation.
//
// Some callers cannot allocate memory at the point where they need M2: code
// running inside a region where cudaMalloc is forbidden or unsafe (a CUDA
// stream capture in global mode, a real-time or signal-sensitive loop, a
// host process whose memory manager owns the whole device), or an embedder
// that has a fixed memory budget and wants no hidden allocations.  For them
// this file provides one entry point that takes the caller's input state and
// output pointer and uses, as its only scratch, one file-scope device array
// of fixed size: a ring of inter-pass scratch, the partial sums and the wait
// counters of the two-pass kernel, and the norm / status words.
//
// The array belongs to the module: every GPU that loads the library holds
// its kNoAllocBytes until the process exits, and every call on a device uses
// the same array.  The words that must start at zero (counters, status,
// flags) are cleared on the stream by each call; the rest is overwritten
// before it is read.  Two calls whose work overlaps on the GPU (different
// streams, or host threads racing on one stream) therefore race on the
// array; calls that are ordered on the GPU are safe.
//
// In host code the name g_noalloc_scratch stands for the device symbol, not
// for a device address: the address is looked up with cudaGetSymbolAddress
// on every call made while its stream is not being captured (a
// cudaDeviceReset unloads the module, and the array may come back
// elsewhere); a call during a capture uses the address found before, so the
// first call with a given device current must not be made during a capture.
#include <cuda_runtime.h>

#include <mutex>

#include "sre.h"
#include "sre_internal.h"

namespace {

constexpr int kNoAllocMaxN = SRE_NOALLOC_MAX_QUBITS;  // 16

// Fixed two-pass configuration (N = 16; N = 13..15 take the single-pass
// kernel): one shift per chunk, 8 ring slots, lag 3.
constexpr int kRingSlots = 8;
constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Capacities for N <= kNoAllocMaxN.
constexpr size_t kRingBytes = (size_t)kRingSlots * 8 * ((size_t)1 << kNoAllocMaxN);  // full part, N = 16
constexpr size_t kChunkCap = ((size_t)1 << kNoAllocMaxN) + 8;                     // chunks of C = 1
constexpr size_t kItemCap = 1024;                                                  // >= R * P2
constexpr size_t kPartCap = sre::kTile;                                            // N <= 12 tiles

constexpr size_t kOffRing = 0;
constexpr size_t kOffChunk = align_up(kOffRing + kRingBytes);
constexpr size_t kOffCount = align_up(kOffChunk + sizeof(double) * kChunkCap);
constexpr size_t kOffItem = align_up(kOffCount + sizeof(unsigned) * 3 * kChunkCap);
constexpr size_t kOffPart = align_up(kOffItem + sizeof(double) * kItemCap);
constexpr size_t kOffNorm = align_up(kOffPart + sizeof(double) * kPartCap);
constexpr size_t kOffWork = align_up(kOffNorm + sizeof(double) * sre::kNormBlocks);
constexpr size_t kOffStatus = align_up(kOffWork + 2 * sizeof(unsigned long long));
constexpr size_t kOffFlags = align_up(kOffStatus + sizeof(int));
constexpr size_t kOffResult = align_up(kOffFlags + sizeof(int));
constexpr size_t kNoAllocBytes = align_up(kOffResult + sizeof(sre::Result));  // about 5.4 MB

}  // namespace

// The scratch of sre_m2_noalloc (see the file comment).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
bool g_ready[kMaxDevices];
unsigned char *g_base[kMaxDevices];
sre::DeviceInfo g_info[kMaxDevices];

// With the device current: the device address of the array and the device
// properties.  The address is looked up again on every call made while
// `stream` is not being captured (a cudaDeviceReset unloads the module, and
// the array may come back elsewhere); during a capture the address found
// before is used, and a capture before any lookup on the device fails.
sre_status_t setup(int dev, cudaStream_t stream) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) {
        cudaGetLastError();
        cs = cudaStreamCaptureStatusActive;  // unknown: do not look anything up
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (cs != cudaStreamCaptureStatusNone) return g_ready[dev] ? SRE_OK : SRE_ECUDA;
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
        cudaGetLastError();
        return SRE_ECUDA;
    }
    if (!g_ready[dev] && sre::query_device(&g_info[dev]) != cudaSuccess) {
        cudaGetLastError();
        return SRE_ECUDA;
    }
    g_base[dev] = static_cast<unsigned char *>(ptr);
    g_ready[dev] = true;
    return SRE_OK;
}

}  // namespace

extern "C" sre_status_t sre_m2_noalloc(const void *d_state, int N, sre_stream_t stream, double *d_m2) {
    if (!d_state || !d_m2) return SRE_EINVAL;
    if (N < 1 || N > kNoAllocMaxN) return SRE_EINVAL;  // beyond the fixed scratch
    if (((uintptr_t)d_state) % 8 || ((uintptr_t)d_m2) % 8) return SRE_EALIGN;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return SRE_ECUDA;
    }
    const sre_status_t s = setup(dev, (cudaStream_t)stream);
    if (s != SRE_OK) return s;
    unsigned char *base = g_base[dev];

    sre::Workspace ws;  // views into the static array; nothing is allocated
    ws.N_max = kNoAllocMaxN;
    ws.elem_bytes = 8;
    ws.scratch = base + kOffRing;
    ws.scratch_bytes = kRingBytes;
    ws.chunk_sum = reinterpret_cast<double *>(base + kOffChunk);
    ws.chunk_cap = kChunkCap;
    ws.counters = reinterpret_cast<unsigned *>(base + kOffCount);
    ws.item_part = reinterpret_cast<double *>(base + kOffItem);
    ws.item_part_cap = kItemCap;
    ws.part = reinterpret_cast<double *>(base + kOffPart);
    ws.part_cap = (int)kPartCap;
    ws.npart = reinterpret_cast<double *>(base + kOffNorm);
    ws.work = reinterpret_cast<unsigned long long *>(base + kOffWork);
    ws.status = reinterpret_cast<int *>(base + kOffStatus);
    ws.flags = reinterpret_cast<int *>(base + kOffFlags);
    ws.result = reinterpret_cast<sre::Result *>(base + kOffResult);

    sre::LargeCfg c;
    c.C_log = 0;
    c.R = kRingSlots;
    c.D = 3;
    c.G2_log = 0;
    c.B1_log = 0;
    c.grid = 2 * g_info[dev].sms;
    const cudaError_t e =
        sre::enqueue_m2_fixed(ws, g_info[dev], d_state, N, c, c, (cudaStream_t)stream, d_m2, 5000000000ll);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorInvalidValue ? SRE_EINVAL : SRE_ECUDA;
    }
    return SRE_OK;
}
