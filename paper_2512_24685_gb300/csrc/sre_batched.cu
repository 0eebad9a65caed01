// sre_batched.cu -- batched evaluation of many states of uneven N.
#include <cuda_runtime.h>

#include <new>

#include "sre_batched.h"

namespace sre {

struct BatchedContext {
    DeviceInfo dev;
};

BatchedContext *batched_create(const DeviceInfo &dev) {
    BatchedContext *c = new (std::nothrow) BatchedContext();
    if (c) c->dev = dev;
    return c;
}

void batched_destroy(BatchedContext *ctx) { delete ctx; }

cudaError_t batched_run(BatchedContext *ctx, const Workspace &ws, const DeviceInfo &dev,
                        const void *const *d_states, const int *Ns, int count, sre_dtype_t dtype,
                        sre_mode_t mode, cudaStream_t stream, double *d_m2_out, long long wait_ns) {
    (void)ctx;
    for (int i = 0; i < count; ++i) {
        cudaError_t e = enqueue_m2(ws, dev, d_states[i], dtype, Ns[i], 0, 1ull << Ns[i], mode,
                                   stream, d_m2_out + i, nullptr, wait_ns, nullptr);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

bool tc_mode_available(sre_mode_t mode) {
    (void)mode;
    return false;
}

cudaError_t tc_enqueue_m2(const Workspace &, const DeviceInfo &, const void *, sre_dtype_t, int,
                          uint64_t, uint64_t, sre_mode_t, cudaStream_t, double *, double *,
                          long long) {
    return cudaErrorNotSupported;
}

}  // namespace sre
