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

#include <cmath>
#include <vector>

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

// TFIM with longitudinal field (Example 1, open chain), scaled by 1/a:
// (H v)[t] = diag(t) v[t] - hx sum_i v[t ^ 2^i], with
// diag(t) = -J sum_{i<N-1} s_i s_{i+1} - hz sum_i s_i and s_i = 1 - 2 t_i.
// One Chebyshev term per launch (w = H v_k / a):
//   first: out = w, acc = c0 v_k + c w
//   else:  out = 2 w - out (out holds v_{k-1} on entry), acc += c out.
struct ChebArgs {
    int N, S;
    double J, hx, hz, inv_a;
    double2 c, c0;
    int first;
};

__global__ void k_tfim_cheb(const double2 *__restrict__ vk, double2 *out, double2 *acc, ChebArgs p) {
    const int N = p.N;
    const uint64_t d = 1ull << N;
    const uint64_t total = d * (uint64_t)p.S;
    const uint64_t bond_mask = (N > 1) ? ((1ull << (N - 1)) - 1) : 0ull;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t t = i & (d - 1);
        const double2 *v = vk + (i - t);
        const int anti = __popcll((t ^ (t >> 1)) & bond_mask);   // bonds with s_i s_{i+1} = -1
        const int ones = __popcll(t);
        const double zz = (double)((N - 1) - 2 * anti);
        const double z = (double)(N - 2 * ones);
        const double dg = -p.J * zz - p.hz * z;
        const double2 vt = v[t];
        double xr = 0.0, xi = 0.0;
        for (int b = 0; b < N; ++b) {
            const double2 u = v[t ^ (1ull << b)];
            xr += u.x;
            xi += u.y;
        }
        double wr = (dg * vt.x - p.hx * xr) * p.inv_a;
        double wi = (dg * vt.y - p.hx * xi) * p.inv_a;
        double2 a;
        if (p.first) {
            out[i] = make_double2(wr, wi);
            a.x = p.c0.x * vt.x - p.c0.y * vt.y + p.c.x * wr - p.c.y * wi;
            a.y = p.c0.x * vt.y + p.c0.y * vt.x + p.c.x * wi + p.c.y * wr;
        } else {
            const double2 prev = out[i];
            wr = 2.0 * wr - prev.x;
            wi = 2.0 * wi - prev.y;
            out[i] = make_double2(wr, wi);
            a = acc[i];
            a.x += p.c.x * wr - p.c.y * wi;
            a.y += p.c.x * wi + p.c.y * wr;
        }
        acc[i] = a;
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

// exp(-i H dt) by the Chebyshev expansion exp(-i z x) = sum_k (2 - [k = 0])
// (-i)^k J_k(z) T_k(x) with x = H / a, z = a dt and a = J (N - 1) +
// (|hx| + |hz|) N >= ||H||, truncated where |J_k(z)| < 1e-17 beyond k > z.
// T_k(x) v follows the three-term recurrence T_{k+1} = 2 x T_k - T_{k-1}.
// buf and acc hold S * 2^N complex128 each; the states are overwritten by
// the evolved states.
cudaError_t evolve_tfim_step(void *d_states, void *d_buf, void *d_acc, int N, int S, double dt, double J,
                             double hx, double hz, const DeviceInfo &dev, cudaStream_t st) {
    const double a = std::fabs(J) * (N - 1) + (std::fabs(hx) + std::fabs(hz)) * N + 1e-12;
    const double z = a * dt;
    std::vector<double> jk;
    for (int k = 0; k < 100000; ++k) {
        const double v = std::cyl_bessel_j((double)k, z);
        jk.push_back(v);
        if (k > z + 4 && std::fabs(v) < 1e-17 && std::fabs(jk[k - 1]) < 1e-17) break;
    }
    auto coeff = [&](int k) {
        const double m = (k == 0 ? 1.0 : 2.0) * jk[k];
        switch (k & 3) {  // (-i)^k
            case 0: return make_double2(m, 0.0);
            case 1: return make_double2(0.0, -m);
            case 2: return make_double2(-m, 0.0);
            default: return make_double2(0.0, m);
        }
    };
    ChebArgs p;
    p.N = N;
    p.S = S;
    p.J = J;
    p.hx = hx;
    p.hz = hz;
    p.inv_a = 1.0 / a;
    double2 *bufs[2] = {reinterpret_cast<double2 *>(d_states), reinterpret_cast<double2 *>(d_buf)};
    double2 *acc = reinterpret_cast<double2 *>(d_acc);
    const uint64_t total = (1ull << N) * (uint64_t)S;
    const int grid = grid_for(total, dev);
    // term 1 (with term 0 folded in): v1 = x v0 into buf; then v_{k+1}
    // overwrites v_{k-1}: the two buffers alternate
    for (int k = 1; k < (int)jk.size(); ++k) {
        p.first = (k == 1);
        p.c = coeff(k);
        p.c0 = coeff(0);
        const double2 *vk = bufs[(k - 1) & 1];
        double2 *out = bufs[k & 1];
        k_tfim_cheb<<<grid, 256, 0, st>>>(vk, out, acc, p);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaMemcpyAsync(d_states, d_acc, total * sizeof(double2), cudaMemcpyDeviceToDevice, st);
}

}  // namespace sre
