// sre_batched.h -- batched (uneven N) execution and the tensor-core modes of
// libsre; internal declarations.
#pragma once
#include <cuda_runtime.h>

#include "sre_internal.h"

namespace sre {

struct BatchedContext;

BatchedContext *batched_create(const DeviceInfo &dev);
void batched_destroy(BatchedContext *ctx);

// M2 of `count` states (device pointers, uneven N) into d_m2_out[count].
// tuned_half[N] (may be null, or hold nulls) gives autotuned two-pass
// configurations of the halved shifts per N.  d_status_out (device, may be
// null) receives each state's sre_status_t (SRE_ETIMEDOUT for every state
// of a batch in which a device wait expired).
cudaError_t batched_run(BatchedContext *ctx, const Workspace &ws, const DeviceInfo &dev,
                        const void *const *d_states, const int *Ns, int count, sre_dtype_t dtype,
                        sre_mode_t mode, cudaStream_t stream, double *d_m2_out, long long wait_ns,
                        const LargeCfg *const *tuned_half, bool capture = true,
                        int *d_status_out = nullptr);

// Tensor-core split-precision modes (BF16 / FP16 hi-lo fixed-point Hadamard stages).
bool tc_mode_available(sre_mode_t mode);
cudaError_t tc_enqueue_m2(const Workspace &ws, const DeviceInfo &dev, const void *d_state,
                          sre_dtype_t dtype, int N, uint64_t x_begin, uint64_t x_end,
                          sre_mode_t mode, cudaStream_t stream, double *d_m2, double *d_per_x,
                          long long wait_ns, LargeCfg *cfg_half, int alpha = 2);

}  // namespace sre
