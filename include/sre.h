/*
 * sre.h -- C ABI of libsre: the second-order stabilizer Renyi entropy M2 of
 * an N-qubit pure state by the exact XOR-FWHT method, on one NVIDIA GB300
 * (sm_103a).
 *
 * What is computed (paper, "Algebraic Reformulation" and Algorithm 1).
 * The state |psi> = sum_t phi_t |t>, t in {0,1}^N, is a vector of d = 2^N
 * complex amplitudes; qubit j is bit j of the index t.  For every X-mask x
 * and Z-mask z, Eq. (Pauli_expect) gives
 *     A_x(z) = <psi| X^x Z^z |psi> = sum_t (-1)^{popc(z & t)} conj(phi_{t^x}) phi_t,
 * i.e. the unnormalised Walsh-Hadamard transform over t of the XOR-shifted
 * product g_x(t) = conj(phi_{t^x}) phi_t.  Eq. (final1) / Algorithm 1:
 *     S  = sum_{x,z} |A_x(z)|^4,      M2 = -log2( S / d ),
 * for a normalised state.  The library does not rescale the caller's
 * amplitudes: it computes n2 = <psi|psi> in FP64 and returns
 *     M2 = -log2( S / (d * n2^4) ),
 * which is the same quantity for the normalised state (S scales as n2^4).
 * The logarithm is base 2 (Algorithm 1, last step).
 *
 * Conventions for every entry point:
 *  - Device pointers are CUDA device (or managed) addresses on the current
 *    device; host pointers are ordinary host addresses.
 *  - State buffers are interleaved complex: (re, im) float pairs for
 *    SRE_C64, (re, im) double pairs for SRE_C128, d = 2^N entries, 8- or
 *    16-byte aligned respectively, contiguous.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on it; entry points marked "synchronous"
 *    wait for that stream before returning.
 *  - The caller owns every buffer it passes and keeps it valid until the
 *    work that reads or writes it has completed on `stream`.
 *  - A plan owns its device scratch; one plan must not be used from two
 *    host threads, or on two streams, at the same time.
 *  - Every function returns an sre_status_t; on error nothing is written to
 *    the caller's outputs unless stated otherwise.
 */
#ifndef SRE_H_
#define SRE_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define SRE_API __attribute__((visibility("default")))
#else
#define SRE_API
#endif

#define SRE_MAX_QUBITS 24 /* largest N a plan accepts */
#define SRE_MAX_ORDER 16  /* largest Renyi order alpha of sre_m_alpha */

typedef enum {
    SRE_OK = 0,
    SRE_EINVAL = 1,       /* bad N, null pointer, bad dtype / mode / range */
    SRE_EALIGN = 2,       /* misaligned pointer */
    SRE_EZERO = 3,        /* the state has zero norm */
    SRE_ENONFINITE = 4,   /* a NaN or Inf amplitude */
    SRE_ENOMEM = 5,       /* device or host allocation failed */
    SRE_EBUSY = 6,        /* server admission rejected (HBM budget / queue full) */
    SRE_ETIMEDOUT = 7,    /* a bounded device-side wait expired */
    SRE_ECUDA = 8,        /* a CUDA runtime call failed (see sre_last_cuda_error) */
    SRE_ENOTFOUND = 9,    /* unknown server ticket */
    SRE_EUNSUPPORTED = 10 /* mode not available for this N / dtype */
} sre_status_t;

typedef enum {
    SRE_C64 = 0,  /* interleaved float32 (re, im) */
    SRE_C128 = 1  /* interleaved float64 (re, im) */
} sre_dtype_t;

/* Arithmetic used for the product, the transform and the per-element
 * |A|^4; the cross-shift accumulation, the norm and the final log are FP64
 * in every mode.  The split modes apply to complex64 states and take the
 * halved shifts (x >= 4096) of 16-byte aligned states with 16 <= N <= 20
 * (other sizes run wholly in FP32) through two
 * tensor-core Hadamard stages of 128 x 128: each operand is scaled by a
 * power of two and split into an integer high piece (|hi| <= 2^8 for bf16,
 * 2^11 for fp16) and the remainder rounded to the 16-bit type as the low
 * piece.  The Hadamard matrix is +-1, so the high piece's sums are exact in
 * the FP32 accumulator and the low piece adds the next 8 (bf16) or 11
 * (fp16) significant bits; the remaining shifts run in FP32.  Value 3 is unused (a tf32 split would need the same two
 * pieces at half the bf16 tensor rate and twice the operand bytes). */
typedef enum {
    SRE_MODE_FP32 = 0,       /* CUDA-core FP32 butterflies */
    SRE_MODE_BF16_SPLIT = 1, /* tensor-core Hadamard stages, bf16 hi/lo fixed-point split */
    SRE_MODE_FP16_SPLIT = 2, /* tensor-core Hadamard stages, fp16 hi/lo fixed-point split */
    SRE_MODE_FP64 = 4,       /* CUDA-core FP64 everywhere */
    SRE_MODE_AUTO = -1       /* the plan's tuned default */
} sre_mode_t;

typedef struct sre_plan_s *sre_plan_t;
typedef void *sre_stream_t; /* cudaStream_t */

/* Human-readable message for a status (static storage, never NULL). */
SRE_API const char *sre_status_str(sre_status_t status);

/* Text of the last CUDA error seen by this host thread ("" if none). */
SRE_API const char *sre_last_cuda_error(void);

/* Library version, major*10000 + minor*100 + patch. */
SRE_API int sre_version(void);

/*
 * Create a plan for states of up to N qubits (1 <= N <= SRE_MAX_QUBITS) of
 * element type `dtype` on the current CUDA device.  The plan allocates its
 * device scratch here (reduction partials, status words, and for N > 12 the
 * ring of inter-pass scratch, sized from N and the device's L2).  *out is
 * set only on SRE_OK.  Errors: SRE_EINVAL (N or dtype out of range, out
 * NULL), SRE_ENOMEM, SRE_ECUDA.
 */
SRE_API sre_status_t sre_plan_create(int N, sre_dtype_t dtype, sre_plan_t *out);

/* Select the arithmetic mode (default SRE_MODE_FP32 for SRE_C64 plans,
 * SRE_MODE_FP64 for SRE_C128 plans).  SRE_EUNSUPPORTED if the mode is not
 * built for this plan. */
SRE_API sre_status_t sre_plan_set_mode(sre_plan_t plan, sre_mode_t mode);
SRE_API sre_status_t sre_plan_get_mode(sre_plan_t plan, sre_mode_t *mode);

/*
 * Tuning of the two-pass kernel used for N > 12 (one pass transforms the
 * low 12 bits of t per block into an L2-resident ring of scratch, the other
 * the remaining bits).  x_batch_log: log2 of the shifts that share one
 * pass-1 partner block (0..3); ring_slots: chunks held in the ring (>= 2);
 * lag: how many chunks pass 2 trails pass 1 (1 <= lag < ring_slots);
 * pass2_tiles_log: log2 of the 2^12-entry tiles per pass-2 work item;
 * pass1_blocks_log: log2 of the consecutive 2^12-entry blocks of t per
 * pass-1 work item;
 * pass1_staged (0/1): pass 1 takes each block and its partner block by bulk
 * copy into shared memory (FP32 CUDA-core path, x_batch_log = 0 and a
 * 16-byte aligned state; otherwise, or with 0, per-thread loads);
 * pass2_staged (0/1): pass 2 takes its tiles by 2-D tensor-memory-accelerator
 * copies into shared memory (FP32, 17 <= N <= 21; otherwise, or with 0,
 * per-thread loads).
 * A value of -1 keeps the library's choice for that field; all -1 restores
 * the defaults.  The scratch ring must fit the plan's allocation
 * (SRE_EINVAL otherwise).  Applies to the halved shifts (x >= 4096).
 */
typedef struct {
    int x_batch_log;
    int ring_slots;
    int lag;
    int pass2_tiles_log;
    int pass1_blocks_log;
    int pass1_staged;
    int pass2_staged;
} sre_tuning_t;
SRE_API sre_status_t sre_plan_set_tuning(sre_plan_t plan, const sre_tuning_t *tuning);
SRE_API sre_status_t sre_plan_get_tuning(sre_plan_t plan, int N, sre_tuning_t *tuning);

/*
 * Autotuner: for the plan's mode and the given N (> 12), time a fixed set of
 * candidate tunings on a bounded slice of shifts of a synthetic state held in
 * the plan, keep the fastest and make it the plan's tuning for that N.
 * SYNCHRONOUS (uses `stream`).  *best receives the chosen tuning and *ms its
 * time on the slice (either may be NULL).  N <= 12 has nothing to tune
 * (SRE_OK, tuning left unchanged).
 */
SRE_API sre_status_t sre_plan_autotune(sre_plan_t plan, int N, sre_stream_t stream,
                                       sre_tuning_t *best, double *ms);

/* Profiling support.  When enabled (enable != 0), the plan records two CUDA
 * events on the stream around the main transform launch of each
 * evaluation: for N > 12 the launch of the conjugate-symmetry halved
 * shifts x >= 4096 (k_large, k_mid or k_tc; 99.6 % of the shifts at
 * N = 20), else the single-tile kernel.  sre_plan_last_kernel_ms waits for
 * the second event and returns the elapsed milliseconds of the last
 * evaluation's main launch and its kernel's name (static string).  sre_plan_launch_count returns the number of kernels
 * the plan has launched since it was created (its own kernels only). */
SRE_API sre_status_t sre_plan_set_profiling(sre_plan_t plan, int enable);
SRE_API sre_status_t sre_plan_last_kernel_ms(sre_plan_t plan, double *ms, const char **name);
SRE_API sre_status_t sre_plan_launch_count(sre_plan_t plan, uint64_t *count);

/* Release the plan and its device memory.  Waits for the plan's work on the
 * device to finish first.  NULL is accepted. */
SRE_API sre_status_t sre_plan_destroy(sre_plan_t plan);

/*
 * M2 of one state (Algorithm 1 over all d shifts), SYNCHRONOUS.
 * d_state: device buffer of 2^N elements of the plan's dtype, N <= plan N.
 * m2_host: host double receiving M2.  Waits for `stream`.
 * Errors: SRE_EINVAL, SRE_EALIGN, SRE_EZERO (n2 == 0), SRE_ENONFINITE
 * (a NaN/Inf amplitude), SRE_ETIMEDOUT, SRE_ECUDA.
 */
SRE_API sre_status_t sre_m2(sre_plan_t plan, const void *d_state, int N, sre_stream_t stream,
                    double *m2_host);

/*
 * Asynchronous M2: enqueue the whole computation on `stream` and write M2
 * to the device double d_m2 (NaN when the state has zero norm or a
 * non-finite amplitude).  Returns after enqueueing; argument errors are
 * reported immediately, data errors only through the NaN.
 */
SRE_API sre_status_t sre_m2_async(sre_plan_t plan, const void *d_state, int N, sre_stream_t stream,
                          double *d_m2);

/*
 * End-to-end M2 from a HOST buffer: copies the 2^N amplitudes host->device
 * on `stream` (pinned host memory gives an asynchronous copy), computes,
 * and reads M2 back.  SYNCHRONOUS.  Same errors as sre_m2.
 */
SRE_API sre_status_t sre_m2_host(sre_plan_t plan, const void *h_state, int N, sre_stream_t stream,
                         double *m2_host);

/*
 * Partial sum over a range of X-masks (the paper's shift k; shifts are
 * independent, so a state's work splits by shift range):
 *     d_out[0] = sum_{x in [x_begin, x_end)} sum_z |A_x(z)|^4      (FP64)
 *     d_out[1] = n2 = <psi|psi>                                    (FP64)
 * d_out is a device buffer of 2 doubles.  If d_per_x is not NULL it is a
 * device buffer of (x_end - x_begin) doubles receiving each shift's
 * sum_z |A_x(z)|^4 (available for N >= 13; SRE_EUNSUPPORTED below).
 * Asynchronous.  Shards over ranges add up to the full S; M2 follows as
 * -log2(S / (d n2^4)).  SRE_EINVAL unless 0 <= x_begin < x_end <= 2^N.
 */
SRE_API sre_status_t sre_sum4_range(sre_plan_t plan, const void *d_state, int N, uint64_t x_begin,
                            uint64_t x_end, sre_stream_t stream, double *d_out,
                            double *d_per_x);

/*
 * Stabilizer Renyi entropy of integer order alpha, Eq. (sre):
 *     M_alpha = 1/(1 - alpha) * log2( (1/d) sum_P |<psi|P|psi>|^{2 alpha} )
 * for the normalised state, i.e. log2(S_alpha / (d n2^{2 alpha})) / (1 - alpha)
 * with S_alpha = sum_{x,z} |A_x(z)|^{2 alpha} of the stored state.  The same
 * XOR-FWHT pass as M2 (Algorithm 1) with the exponent 2 alpha in place of 4;
 * for x >= 4096 the conjugate symmetry gives sum_z |A_x(z)|^{2 alpha} =
 * 2^{2 alpha} sum_{z'} [(Re W)^{2 alpha} + (Im W)^{2 alpha}].  alpha = 2 is M2
 * (bitwise the same as sre_m2).  2 <= alpha <= SRE_MAX_ORDER, else
 * SRE_EINVAL.  SYNCHRONOUS; result in *m_host; other arguments and errors as
 * sre_m2.  FP32 modes: terms below the FP32 range (|A|^{2 alpha} < ~1e-45)
 * count as zero; for a normalised state they are far below the result's
 * rounding.
 */
SRE_API sre_status_t sre_m_alpha(sre_plan_t plan, const void *d_state, int N, int alpha,
                                 sre_stream_t stream, double *m_host);

/*
 * Random-circuit quench dynamics (the paper's Example 2), evolved on the
 * device: S independent realizations of an N-qubit open chain start in
 * |0...0>; step t applies a two-qubit gate to every even bond (0,1), (2,3),
 * ... and then to every odd bond (1,2), (3,4), ...; after every step M2 of
 * every realization is evaluated (the batched path, in the plan's mode).
 *   d_gates  device, T * S * (N - 1) gates of 16 complex128 (re, im) each:
 *            gate (t, s, b) at offset ((t S + s)(N - 1) + b) * 16, row-major,
 *            acting on the index 2 b_{q+1} + b_q of bond (q, q+1); b < N/2 is
 *            the even bond q = 2b, larger b the odd bond q = 2(b - N/2) + 1.
 *            For Example 2 every gate is Haar-random on U(4).
 *   d_states device, S * 2^N complex128, caller-owned scratch; holds the
 *            final states on return.
 *   d_m2_out device, T * S doubles: M2 of realization s after step t at
 *            t * S + s.
 * The plan's dtype must be SRE_C128 and 2 <= N <= its N, 1 <= S <= 65535,
 * T >= 1 (SRE_EINVAL otherwise; SRE_EALIGN for pointers not 16-byte aligned,
 * d_m2_out 8-byte).  Gates are applied in FP64.  Asynchronous on `stream`.
 */
SRE_API sre_status_t sre_brickwork_m2_series(sre_plan_t plan, int N, int S, int T, const void *d_gates,
                                             void *d_states, sre_stream_t stream, double *d_m2_out);

/*
 * Hamiltonian quench dynamics (the paper's Example 1), evolved on the device:
 * the transverse-field Ising chain with a longitudinal field, Eq.
 * (TFIM_LF_OBC) on an open chain,
 *     H = -J sum_{i=0}^{N-2} Z_i Z_{i+1} - hx sum_i X_i - hz sum_i Z_i
 * (qubit i = bit i, Z|0> = |0>; the paper takes J = 1, hx = hz = 1.5).
 * d_states (device, S * 2^N complex128, caller-owned) holds S initial states
 * on entry; each of T steps applies exp(-i H dt) to every state (Chebyshev
 * expansion to |J_k| < 1e-17, FP64) and then evaluates M2 of every state
 * (batched path, in the plan's mode) into d_m2_out[t * S + s] (device, T * S
 * doubles).  On return d_states holds the states at time T dt.  The plan's
 * dtype must be SRE_C128; 1 <= N <= its N, 1 <= S <= 65535, T >= 1, dt >= 0
 * and ||H|| dt <= 1000 with ||H|| <= |J|(N-1) + (|hx|+|hz|) N (SRE_EINVAL
 * otherwise; SRE_EALIGN for misaligned pointers).  The plan keeps two
 * evolution buffers of the states' size.  Asynchronous on `stream`.
 */
SRE_API sre_status_t sre_tfim_m2_series(sre_plan_t plan, int N, int S, int T, double dt, double J, double hx,
                                        double hz, void *d_states, sre_stream_t stream, double *d_m2_out);

/*
 * sre_sum4_range at Renyi order alpha: d_out[0] = sum over shifts
 * [x_begin, x_end) of sum_z |A_x(z)|^{2 alpha}, d_out[1] = n2; d_per_x as
 * there.  Asynchronous; shards add up to S_alpha.  SRE_EINVAL for alpha
 * outside [2, SRE_MAX_ORDER] or a bad range.
 */
SRE_API sre_status_t sre_sum_pow_range(sre_plan_t plan, const void *d_state, int N, int alpha,
                                       uint64_t x_begin, uint64_t x_end, sre_stream_t stream,
                                       double *d_out, double *d_per_x);

/*
 * The last step of Algorithm 1 for sums reduced elsewhere (for example the
 * all-reduce of sre_sum4_range / sre_sum_pow_range partials over shards of
 * the shifts): Eq. (final1) at order 2 and Eq. (sre) at integer order alpha,
 *     *d_m = log2(S / (d n2^(2 alpha))) / (1 - alpha),   d = 2^N,
 * so M2 = -log2(S / (d n2^4)).  d_S and d_n2: device doubles holding the
 * total sum S_alpha and n2 = <psi|psi>; d_m: device double receiving the
 * result (NaN unless S and n2 are finite and > 0).  All three are owned by
 * the caller and must be 8-byte aligned (SRE_EALIGN).  SRE_EINVAL for a
 * null pointer, N outside [1, SRE_MAX_QUBITS] or alpha outside
 * [2, SRE_MAX_ORDER].  Asynchronous on `stream`; needs no plan.
 */
SRE_API sre_status_t sre_m_alpha_from_sums(const double *d_S, const double *d_n2, int N, int alpha,
                                           sre_stream_t stream, double *d_m);

/*
 * M2 of `count` states of uneven size in one submission (states may have
 * different N, each <= the plan's N): Algorithm 1 with Eq. (final1) per
 * state, the paper's loop over states of one experiment (the realizations
 * and time steps of its Examples 1 and 2) folded into one launch sequence.
 * d_states: host array of `count`
 * device pointers; Ns: host array of the N_i; d_m2_out: device array of
 * `count` doubles (NaN for a zero / non-finite state, and for every state
 * of a submission in which a device wait expired).  In the split modes the
 * states with 16 <= N <= 20 (all of a size class 16-byte aligned) take the
 * tensor-core kernel for their halved shifts, each with its own scale
 * table; every result equals the state's sre_m2 in the plan's mode bit for
 * bit.  The batch is
 * executed by persistent kernels walking one work list, and is replayed
 * from a captured CUDA graph when the same (pointers, Ns) batch is
 * submitted again.  Asynchronous.  Errors: SRE_EINVAL, SRE_EALIGN,
 * SRE_ENOMEM, SRE_ECUDA.
 */
SRE_API sre_status_t sre_m2_batched(sre_plan_t plan, const void *const *d_states, const int *Ns,
                            int count, sre_stream_t stream, double *d_m2_out);

/*
 * M2 of one complex64 state (FP32 arithmetic, device output) WITHOUT ANY
 * ALLOCATION -- for callers that cannot allocate device or host memory at
 * the point of the call (inside a region where cudaMalloc is unsafe or
 * forbidden, under a fixed memory budget, ...).  The paper has no
 * counterpart; this is an interface variant of sre_m2_async.
 *   d_state: device buffer of 2^N interleaved (re, im) float pairs, 8-byte
 *            aligned, 1 <= N <= SRE_NOALLOC_MAX_QUBITS (16); larger N is
 *            rejected with SRE_EINVAL before anything is launched.
 *   d_m2:    device double receiving M2; NaN for a zero / non-finite state,
 *            and NaN as well when a device wait of the two-pass kernel
 *            expires (fixed limit of 5 s): the status the kernel records
 *            stays in the library's own array, out of the caller's reach.
 * Asynchronous on `stream`.  Its only scratch is one fixed module array of
 * about 5.4 MB that every GPU loading the library holds until exit; a call
 * made while `stream` is not being captured looks up that array's address
 * (so a call after cudaDeviceReset finds the reloaded array), a call during
 * a capture reuses the address found before, so the first call with a
 * device current must not be made during a stream capture.  Every call shares the array, so
 * calls whose work overlaps on the GPU race; calls ordered on the GPU are
 * safe.  Returns SRE_EINVAL, SRE_EALIGN or SRE_ECUDA on error.
 */
#define SRE_NOALLOC_MAX_QUBITS 16
SRE_API sre_status_t sre_m2_noalloc(const void *d_state, int N, sre_stream_t stream, double *d_m2);

/*
 * Failure-detection self test: launch one CTA that waits, with the same
 * bounded wait the two-pass kernel uses, on a device counter that nothing
 * increments.  The wait gives up after wait_ns of GPU time and the call
 * returns the status the kernel recorded (SRE_ETIMEDOUT when the bound
 * works).  SYNCHRONOUS on `stream`; the device context stays usable.
 */
SRE_API sre_status_t sre_selftest_wait_timeout(uint64_t wait_ns, sre_stream_t stream);

/* ----------------------------------------------------------------------- */
/* Serving: continuous batching of M2 requests of mixed N.                  */
/* The paper has no serving layer; each request is Algorithm 1 with         */
/* Eq. (final1), evaluated by the single-state path (N > 16) or merged with */
/* other small requests into one sre_m2_batched-style submission.           */
/* ----------------------------------------------------------------------- */

typedef struct sre_server_s *sre_server_t;

typedef struct {
    uint64_t hbm_budget_bytes; /* admission limit on resident request bytes */
    int max_inflight;          /* slots: units of work on the device at once */
    int max_queue;             /* waiting requests before SRE_EBUSY */
    int max_N;                 /* largest N accepted */
    sre_mode_t mode;           /* arithmetic for every request: FP32, FP64 or a split mode
                                  (split modes: requests with 16 <= N <= 20 run their halved
                                  shifts on the tensor cores, merged small requests in FP32) */
    uint64_t wait_limit_ns;    /* bound on every device-side wait */
    int device;                /* CUDA device ordinal */
    uint64_t slot_scratch_bytes; /* scratch ring of each slot; 0: 96 MiB (room for the
                                    library's default rings); tuned rings may need more */
    uint64_t chunk_terms;      /* 0: every request is one unit.  Otherwise a request with
                                  N > 16 and more than chunk_terms Pauli terms runs as 2^k
                                  shift ranges of at most chunk_terms terms (at least 4096
                                  shifts each); the ranges of one request take turns with
                                  the other queued work, and their partial sums are added
                                  in range order before the final log */
} sre_server_cfg_t;

typedef struct {
    uint64_t submitted, admitted, completed, rejected, failed;
    uint64_t inflight, queued;
    double p50_latency_ms, p99_latency_ms, mean_latency_ms;
    double states_per_s, pauli_terms_per_s; /* since the first submission */
    uint64_t resident_bytes, peak_resident_bytes;
} sre_server_stats_t;

/* Fill cfg with defaults (HBM budget 8 GiB, 4 slots, 4096 queued,
 * max_N 20, FP32, 5 s wait limit, device 0, default slot scratch, no
 * chunking). */
SRE_API void sre_server_cfg_default(sre_server_cfg_t *cfg);

/* Start a server: a host scheduler thread plus device streams.  *out set
 * on SRE_OK.  Errors: SRE_EINVAL, SRE_ENOMEM, SRE_ECUDA. */
SRE_API sre_status_t sre_server_create(const sre_server_cfg_t *cfg, sre_server_t *out);

/*
 * Tuning of the two-pass kernel for requests of N qubits (13 <= N <= the
 * server's max_N; fields as sre_tuning_t for sre_plan_set_tuning, -1 keeps
 * the library's choice), applied to the halved shifts of every later unit
 * of that N.  The ring must fit each slot's scratch (SRE_EINVAL otherwise;
 * see slot_scratch_bytes).  Thread-safe.
 */
SRE_API sre_status_t sre_server_set_tuning(sre_server_t srv, int N, const sre_tuning_t *tuning);

/*
 * Submit one request.  state: interleaved amplitudes of `dtype`, 2^N of
 * them, in host memory if on_device == 0 or device memory if 1.  The
 * server copies the state into memory it owns before returning, so the
 * caller may reuse its buffer at once.  *ticket identifies the request.
 * on_device must say where `state` lives (it selects the copy's
 * direction; the pointer is not inspected).  Errors: SRE_EINVAL, SRE_EBUSY
 * (queue full, or the request does not fit the HBM budget next to what is
 * resident), SRE_ENOMEM, SRE_ECUDA (the copy failed).
 */
SRE_API sre_status_t sre_server_submit(sre_server_t srv, const void *state, int on_device, int N,
                               sre_dtype_t dtype, uint64_t *ticket);

/* Non-blocking poll: *done = 1 and *m2 set once the request finished
 * (M2 is NaN for a zero / non-finite state); *done = 0 otherwise.  A
 * finished ticket is forgotten after it has been polled done once.
 * SRE_ENOTFOUND for an unknown ticket; SRE_ETIMEDOUT (with *done = 1 and
 * M2 NaN) if a device wait of the launch that evaluated it expired -- for
 * a request merged with others, a wait anywhere in that launch; SRE_ECUDA
 * if that launch failed. */
SRE_API sre_status_t sre_server_poll(sre_server_t srv, uint64_t ticket, int *done, double *m2);

/* Block until `ticket` is done or timeout_ms elapses (SRE_ETIMEDOUT, the
 * ticket stays valid); a finished request returns as sre_server_poll. */
SRE_API sre_status_t sre_server_wait(sre_server_t srv, uint64_t ticket, double timeout_ms, double *m2);

SRE_API sre_status_t sre_server_stats(sre_server_t srv, sre_server_stats_t *stats);

/* Stop the scheduler, drain in-flight work, free everything.  NULL ok. */
SRE_API sre_status_t sre_server_destroy(sre_server_t srv);

#ifdef __cplusplus
}
#endif
#endif /* SRE_H_ */
