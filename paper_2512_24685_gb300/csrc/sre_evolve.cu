// sre_evolve.cu -- brickwork random-circuit dynamics on the device (the
// paper's Example 2): S independent realizations of an N-qubit open chain,
// each started in |0...0>, evolved step by step; one step applies a
// two-qubit gate to every even bond (0,1), (2,3), ... and then to every odd
// bond (1,2), (3,4), ...  The states are complex128 and the gates are
// applied in FP64, so the evolution adds no rounding beyond FP64's; M2 of
// each step is then taken by the batched path.
//
// Gate layout (caller-owned device memory): for step t, realization s and
// bond index b (b < N/2: bond q = 2b; else q = 2(b - N/2) + 1), the 4x4
// complex128 matrix U at gates[((t * S + s) * (N - 1) + b) * 16], row-major,
// acting on the pair index k = 2 b_{q+1} + b_q of qubits q (low) and q+1.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sre_internal.h"

namespace sre {

namespace {

// all S states := |0...0>
__global__ void k_basis0(double2 *states, uint64_t d, uint64_t total) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x)
        states[i] = make_double2((i & (d - 1)) == 0 ? 1.0 : 0.0, 0.0);
}

// One gate per realization on bond (q, q+1): thread g of state s owns the
// four amplitudes whose bits q, q+1 run over 00, 01, 10, 11.
__global__ void k_apply_2q(double2 *states, int N, int S, int q, const double2 *gates, long long gate_stride,
                           long long gate_first) {
    const uint64_t groups = 1ull << (N - 2);
    const uint64_t total = groups * (uint64_t)S;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t s = i >> (N - 2);
        const uint64_t g = i & (groups - 1);
        const uint64_t lo = g & ((1ull << q) - 1);
        const uint64_t i00 = ((g >> q) << (q + 2)) | lo;  // zeros at bits q, q+1
        double2 *psi = states + (s << N);
        const uint64_t idx[4] = {i00, i00 | (1ull << q), i00 | (2ull << q), i00 | (3ull << q)};
        double2 a[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] = psi[idx[k]];
        const double2 *U = gates + gate_first + (long long)s * gate_stride;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            double re = 0.0, im = 0.0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const double2 u = __ldg(U + 4 * r + k);
                re = fma(u.x, a[k].x, re);
                re = fma(-u.y, a[k].y, re);
                im = fma(u.x, a[k].y, im);
                im = fma(u.y, a[k].x, im);
            }
            psi[idx[r]] = make_double2(re, im);
        }
    }
}

int grid_for(uint64_t work, const DeviceInfo &dev) {
    const uint64_t blocks = (work + 255) / 256;
    const uint64_t cap = (uint64_t)dev.sms * 16;
    return (int)(blocks < cap ? blocks : cap);
}

}  // namespace

cudaError_t evolve_init(void *d_states, int N, int S, const DeviceInfo &dev, cudaStream_t st) {
    const uint64_t d = 1ull << N, total = d * (uint64_t)S;
    k_basis0<<<grid_for(total, dev), 256, 0, st>>>(reinterpret_cast<double2 *>(d_states), d, total);
    return cudaGetLastError();
}

cudaError_t evolve_brickwork_step(void *d_states, int N, int S, int t, const void *d_gates,
                                  const DeviceInfo &dev, cudaStream_t st) {
    const int nb = N - 1, n_even = N / 2;
    const long long per_real = (long long)nb * 16;  // complex entries per realization and step
    const uint64_t work = (1ull << (N - 2)) * (uint64_t)S;
    for (int b = 0; b < nb; ++b) {
        const int q = b < n_even ? 2 * b : 2 * (b - n_even) + 1;
        const long long first = (long long)t * S * per_real + (long long)b * 16;
        k_apply_2q<<<grid_for(work, dev), 256, 0, st>>>(reinterpret_cast<double2 *>(d_states), N, S, q,
                                                        reinterpret_cast<const double2 *>(d_gates), per_real,
                                                        first);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace sre
