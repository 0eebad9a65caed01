// sre_tc.cu -- tensor-core (tcgen05) instantiations of the two-pass kernel:
// the split-precision modes SRE_MODE_BF16_SPLIT and SRE_MODE_FP16_SPLIT run
// the last round of every pass-1 tile (tile bits 0-3) as an MMA with the
// exact +-1 matrix H_16 on hi/lo-split operands (see sre_tc.cuh); all other
// stages, the reductions and the shifts below 4096 are the FP32 path.
#include <cuda_runtime.h>

#include "sre_batched.h"
#include "sre_large.cuh"

namespace sre {

size_t tc_extra_smem_bytes() { return (size_t)kTcBBytes + 16; }

template <int H2, int TC>
static cudaError_t launch_tc_h(const LargeArgs &a, int grid, cudaStream_t st) {
    const size_t smem = large_smem_bytes<float, H2>(tc_extra_smem_bytes());
    auto kern = k_large<float, H2, true, TC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if constexpr (large_uses_tma<float, H2>()) {
        LargeArgs b = a;
        if ((e = encode_p2_tmap(b)) != cudaSuccess) return e;
        kern<<<grid, kThreads, smem, st>>>(b);
    } else {
        kern<<<grid, kThreads, smem, st>>>(a);
    }
    return cudaGetLastError();
}

template <int TC>
static cudaError_t launch_tc(const LargeArgs &a, int grid, cudaStream_t st) {
    switch (a.h2) {
#define SRE_CASE(n) \
    case n: return launch_tc_h<n, TC>(a, grid, st);
        SRE_CASE(0) SRE_CASE(1) SRE_CASE(2) SRE_CASE(3) SRE_CASE(4) SRE_CASE(5) SRE_CASE(6)
        SRE_CASE(7) SRE_CASE(8)
#undef SRE_CASE
        default: return cudaErrorNotSupported;  // N > 21 has no tensor-core instantiation
    }
}

cudaError_t launch_large_tc(const LargeArgs &a, int grid, cudaStream_t st, int tc_kind) {
    if (tc_kind == kTcBf16) return launch_tc<kTcBf16>(a, grid, st);
    if (tc_kind == kTcFp16) return launch_tc<kTcFp16>(a, grid, st);
    return cudaErrorInvalidValue;
}

bool tc_mode_available(sre_mode_t mode) {
    return mode == SRE_MODE_BF16_SPLIT || mode == SRE_MODE_FP16_SPLIT;
}

cudaError_t tc_enqueue_m2(const Workspace &ws, const DeviceInfo &dev, const void *d_state,
                          sre_dtype_t dtype, int N, uint64_t x_begin, uint64_t x_end,
                          sre_mode_t mode, cudaStream_t stream, double *d_m2, double *d_per_x,
                          long long wait_ns, LargeCfg *cfg_half, int alpha) {
    if (N > kTileBits + 9) return cudaErrorNotSupported;
    return enqueue_m2(ws, dev, d_state, dtype, N, x_begin, x_end, mode, stream, d_m2, d_per_x, wait_ns,
                      cfg_half, alpha);
}

}  // namespace sre
