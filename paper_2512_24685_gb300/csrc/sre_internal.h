// sre_internal.h -- host-side declarations shared by the libsre translation
// units (kernels, plan / C ABI, batched path, server).  Not installed.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sre.h"

namespace sre {

constexpr int kTileBits = 12;              // one CTA tile: 2^12 complex entries
constexpr int kTile = 1 << kTileBits;
constexpr int kThreads = 256;              // threads per tile CTA
constexpr int kPerThread = kTile / kThreads;  // 16 entries per thread (4 register bits)
constexpr int kNormBlocks = 264;           // fixed grid of the norm reduction
constexpr int kFinalThreads = 256;
constexpr int kMaxRing = 64;                      // ring slots a tuned configuration may use
constexpr size_t kTuneScratch = (size_t)192 << 20;  // scratch floor for N > 12 plans (tuned rings)
constexpr size_t kSlotScratch = (size_t)96 << 20;   // scratch floor for server slots (default rings)

// Device-side result block of one evaluation (written by the finalize kernel).
struct Result {
    double m2;     // -log2(S / (d n2^4)), NaN on a zero / non-finite state
    double S;      // sum_{x,z} |A_x(z)|^4 over the evaluated shift range
    double n2;     // <psi|psi>
    int status;    // sre_status_t of the data checks and device waits
    int pad;
};

// Error word bits written by kernels.
constexpr int kFlagNonFinite = 1;

// Launch configuration of the two-pass (N > 12) persistent kernel.
struct LargeCfg {
    int C_log;   // log2 shifts per chunk (shared partner tile in pass 1)
    int R;       // ring slots of inter-pass scratch
    int D;       // lag (in chunks) of pass 2 behind pass 1, D < R
    int G2_log;  // log2 tiles per pass-2 work item
    int B1_log;  // log2 consecutive blocks per pass-1 work item
    int grid;    // persistent CTAs
    int stage1 = 1;  // pass 1 by bulk copy where available (C = 1, FP32, aligned)
    int stage2 = 1;  // pass 2 by TMA tile copies where available (FP32, 5 <= h2 <= 8)
};

// Everything one evaluation needs on the device (owned by a plan or a
// batched / server context).
struct Workspace {
    int N_max = 0;
    int elem_bytes = 8;            // 8 (FP32 complex) or 16 (FP64 complex)
    double *npart = nullptr;       // kNormBlocks
    int *flags = nullptr;          // 1 int: data flags (non-finite)
    double *part = nullptr;        // per-CTA partials of the single-tile path
    int part_cap = 0;
    void *scratch = nullptr;       // ring of inter-pass scratch
    size_t scratch_bytes = 0;
    double *item_part = nullptr;   // ring of pass-2 item partials
    size_t item_part_cap = 0;
    double *chunk_sum = nullptr;   // per-chunk sums
    size_t chunk_cap = 0;
    unsigned *counters = nullptr;  // done1 | done2 | freed, chunk_cap each
    unsigned long long *work = nullptr;  // work-queue counters (full, halved)
    int *status = nullptr;         // device status word
    Result *result = nullptr;      // device result block
    void *conv = nullptr;          // state converted to the compute type (lazy)
    size_t conv_bytes = 0;
    int *tc_e = nullptr;           // tensor-core path: scale exponent per x >> 12
    double *tc_bn = nullptr;       // tensor-core path: l2 norm per 4096-entry block
    int tc_cap = 0;                // entries of tc_e / tc_bn
    // profiling: events recorded around the main transform kernel when set
    cudaEvent_t ev_begin = nullptr, ev_end = nullptr;
    mutable const char *main_kernel = "";
    mutable unsigned long long launches = 0;  // kernels launched through this workspace
};

struct DeviceInfo {
    int device = 0;
    int sms = 0;
    int l2_bytes = 0;
    int max_smem_optin = 0;
};

cudaError_t query_device(DeviceInfo *info);

// Pick the two-pass configuration for N > 12 (half: conjugate-symmetry halved
// shifts, x >= 4096).
LargeCfg choose_large_cfg(const DeviceInfo &dev, int N, int elem_bytes, int half);

// Tensor-core two-pass kernel (sre_tc.cu) for the halved shifts of one
// state: tc_kind 1 = BF16 hi/lo pieces, 2 = FP16 hi/lo pieces.  tc_applies
// says whether it covers (N, half, Renyi order, state alignment); the launch
// first computes the per-shift fixed-point scales of the state into
// ws.tc_bn / ws.tc_e.
struct LargeArgs;
bool tc_applies(int N, int half, int alpha, const void *psi);
// Tensor-core launch of the halved shifts of one state (a.psi) or of the
// states of a batch class (a.psis, a.chunks_per_state); the per-state scale
// tables go to e_buf / bn_buf (buf_cap entries) when given, else to ws.
cudaError_t launch_large_tc(const LargeArgs &a, const Workspace &ws, const DeviceInfo &dev, int grid,
                            cudaStream_t st, int tc_kind, int *e_buf = nullptr, double *bn_buf = nullptr,
                            size_t buf_cap = 0);

// Does a (possibly tuned) configuration fit the workspace allocation?
bool large_cfg_fits(const Workspace &ws, const LargeCfg &c, int N, int half);

// Fill a state buffer with deterministic pseudo-random amplitudes (timing).
cudaError_t enqueue_fill_synthetic(void *buf, int N, sre_dtype_t dtype, cudaStream_t st);

// Bytes of workspace needed for states up to N_max with element size.
size_t workspace_scratch_bytes(const DeviceInfo &dev, int N_max, int elem_bytes, sre_mode_t mode);

cudaError_t workspace_alloc(Workspace *ws, const DeviceInfo &dev, int N_max, int elem_bytes,
                            sre_mode_t mode, size_t scratch_floor = kTuneScratch);
void workspace_free(Workspace *ws);

// Enqueue the sum over shifts [x_begin, x_end) and the norm of one state.
// The result block (m2, S, n2, status) lands in ws->result; if d_m2 is not
// null M2 is also written there; if d_per_x is not null and N > 12 each
// shift's sum is written there.  mode: SRE_MODE_FP32 or SRE_MODE_FP64.
// alpha: Renyi order (2: M2; larger integers: M_alpha, S the order-alpha sum).
cudaError_t enqueue_m2(const Workspace &ws, const DeviceInfo &dev, const void *d_state,
                       sre_dtype_t dtype, int N, uint64_t x_begin, uint64_t x_end,
                       sre_mode_t mode, cudaStream_t stream, double *d_m2, double *d_per_x,
                       long long wait_ns, LargeCfg *cfg_override, int alpha = 2);

// ---- batched evaluation: states grouped in classes of equal N.
struct BatchClass {
    int N = 0, S = 0;         // size and number of states of the class
    int small_grid = 0;       // N <= 12: CTAs of the single-tile launch
    LargeCfg cfg_full{}, cfg_half{};  // N > 12: shifts < 4096 / halved shifts
    long long cps_full = 0, cps_half = 0;  // chunks per state of each part
    size_t parts_off = 0, parts_n = 0;     // partials of the class
    size_t chunks_max = 0;                 // counters needed by one launch
    int tc_kind = 0;                       // split modes: the halved shifts on the tensor cores
};

BatchClass batch_class_layout(const DeviceInfo &dev, const Workspace &ws, int N, int S,
                              sre_mode_t mode, const LargeCfg *tuned_half);
cudaError_t enqueue_batch_class(const Workspace &ws, const DeviceInfo &dev, const BatchClass &L,
                                const void *const *d_ptrs, double *parts, unsigned *counters,
                                size_t chunk_cap, sre_mode_t mode, cudaStream_t st,
                                long long wait_ns, int *tc_e = nullptr, double *tc_bn = nullptr,
                                size_t tc_cap = 0);
cudaError_t enqueue_batch_norm(const Workspace &ws, const void *const *d_ptrs, const int *d_Ns,
                               int count, double *npart, int *flags, sre_mode_t mode,
                               cudaStream_t st);
cudaError_t enqueue_batch_finalize(const Workspace &ws, const void *seg, const double *parts,
                                   const double *npart, const int *flags, const int *d_Ns,
                                   const int *d_out_index, int count, double *m2_out,
                                   int *status_out, cudaStream_t st);
cudaError_t enqueue_convert(const void *src, sre_dtype_t from, void *dst, int N, cudaStream_t st);
// out = M_alpha from device scalars S and n2 (NaN unless both are finite and > 0).
cudaError_t enqueue_malpha_from_sums(const double *S, const double *n2, int N, int alpha, double *out,
                                     cudaStream_t st);

// Single-pass kernel (sre_mid.cu) for shift ranges whose transform spans one,
// two or (FP32, elem_bytes 8) four 4096-entry blocks: one FP64 partial per
// shift in part[state * sps + shift index], also in per_x if given (single
// state).
bool mid_applies(int N, int half, int elem_bytes);
template <typename R>
cudaError_t launch_mid(int N, int half, const void *psi, const void *const *psis, int nstates, long long sps,
                       uint64_t x_begin, int alpha, double *part, double *per_x, const DeviceInfo &dev,
                       cudaStream_t st);

// Brickwork circuit dynamics (sre_evolve.cu): S complex128 states of N
// qubits set to |0...0>; one step t of even-bond then odd-bond gates.
cudaError_t evolve_init(void *d_states, int N, int S, const DeviceInfo &dev, cudaStream_t st);
cudaError_t evolve_brickwork_step(void *d_states, int N, int S, int t, const void *d_gates,
                                  const DeviceInfo &dev, cudaStream_t st);
// TFIM + longitudinal field: states <- exp(-i H dt) states (Chebyshev, FP64);
// buf and acc are two more buffers of S * 2^N complex128.
cudaError_t evolve_tfim_step(void *d_states, void *d_buf, void *d_acc, int N, int S, double dt, double J,
                             double hx, double hz, const DeviceInfo &dev, cudaStream_t st);

// Bounded-wait self test (see sre_selftest_wait_timeout).
cudaError_t run_wait_selftest(long long wait_ns, cudaStream_t st, int *status_out);

// FP32 M2 of a complex64 state with given two-pass configurations for the
// shifts below 4096 and the halved shifts; allocates nothing (the workspace
// pointers may point into preassigned memory).
cudaError_t enqueue_m2_fixed(const Workspace &ws, const DeviceInfo &dev, const void *psi, int N,
                             const LargeCfg &cfg_full, const LargeCfg &cfg_half, cudaStream_t st,
                             double *d_m2, long long wait_ns);

// Copy the result block to d_out2 = {S, n2} (for the range API).
cudaError_t enqueue_copy_sums(const Workspace &ws, double *d_out2, cudaStream_t stream);

}  // namespace sre
