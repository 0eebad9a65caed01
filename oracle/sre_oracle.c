/*
 * sre_oracle.c -- plain, slow, obviously correct FP64 CPU oracle for the
 * second-order stabilizer Renyi entropy M2 of an N-qubit pure state.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path (the CUDA library
 * and its Python binding) may include, link, load or call this file.  Only
 * the tests, the package's smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code, header, table or helper with the
 * CUDA path.
 *
 * Notation (paper, "Algebraic Reformulation"): the state is
 * |psi> = sum_t phi_t |t>, t in Z_2^N, qubit j <-> bit j of t.  A Pauli string
 * with its global phase dropped is X^x Z^z with x, z in Z_2^N.  X^x|t> = |t^x>,
 * Z^z|t> = (-1)^{popc(z&t)} |t>.
 *
 * Every routine evaluates the *exact stored state*: nothing is normalised in
 * place.  With n2 = <psi|psi>, the sum of fourth powers scales as n2^4, so
 *     M2 = -log2( S / (d * n2^4) ),   S = sum_{x,z} |<psi|X^x Z^z|psi>|^4,
 * which equals Eq. (sre) at alpha = 2 for the normalised state (the paper
 * requires a normalised input in Algorithm 1; dividing by n2^4 is the same
 * thing without rounding the input).  The logarithm is base 2, as in
 * Algorithm 1 and the Haar formula of Fig. 1(b).
 *
 * Two independent evaluations of S:
 *   O1  sre_oracle_sum4_direct   -- the definition: each Pauli expectation
 *       summed directly from Eq. (Pauli_expect), then |.|^4 summed over all
 *       (x, z).  Cost 8^N; meant for N <= 10.
 *   O2  sre_oracle_sum4_xorfwht  -- Algorithm 1 ("XOR-FWHT"): for each shift
 *       form the XOR-shifted product, apply the unnormalised fast
 *       Walsh-Hadamard transform (supplement, FWHT section: butterflies
 *       (a,b) -> (a+b, a-b) over N stages), sum |.|^4.  Cost N 4^N.
 *
 * Sums over many terms use Neumaier compensated summation; the cross-shift
 * sum runs in a fixed order after a parallel loop, so results do not depend
 * on the number of OpenMP threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- compensated summation (Neumaier) -------------------------------- */
typedef struct { double s, c; } ksum_t;

static inline void ksum_add(ksum_t *k, double v) {
    double t = k->s + v;
    if (fabs(k->s) >= fabs(v)) k->c += (k->s - t) + v;
    else                       k->c += (v - t) + k->s;
    k->s = t;
}
static inline double ksum_get(const ksum_t *k) { return k->s + k->c; }

static inline int parity64(uint64_t v) { return __builtin_parityll(v); }

int sre_oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void sre_oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* <psi|psi> = sum_t |phi_t|^2.  psi is interleaved (re, im) doubles. */
double sre_oracle_norm2(const double *psi, int N) {
    const uint64_t d = (uint64_t)1 << N;
    ksum_t k = {0.0, 0.0};
    for (uint64_t t = 0; t < d; ++t)
        ksum_add(&k, psi[2 * t] * psi[2 * t] + psi[2 * t + 1] * psi[2 * t + 1]);
    return ksum_get(&k);
}

/*
 * One Pauli expectation, Eq. (Pauli_expect):
 *   <psi| X^x Z^z |psi> = sum_t (-1)^{z.t} conj(phi_{t^x}) phi_t.
 * Exact for the operator X^x Z^z (no i^{x.z} phase is attached).
 */
void sre_oracle_pauli_expectation(const double *psi, int N, uint64_t x, uint64_t z,
                                  double *out_re, double *out_im) {
    const uint64_t d = (uint64_t)1 << N;
    ksum_t kr = {0.0, 0.0}, ki = {0.0, 0.0};
    for (uint64_t t = 0; t < d; ++t) {
        const double ar = psi[2 * (t ^ x)], ai = -psi[2 * (t ^ x) + 1]; /* conj(phi_{t^x}) */
        const double br = psi[2 * t], bi = psi[2 * t + 1];             /* phi_t */
        double pr = ar * br - ai * bi, pi = ar * bi + ai * br;
        if (parity64(z & t)) { pr = -pr; pi = -pi; }
        ksum_add(&kr, pr);
        ksum_add(&ki, pi);
    }
    *out_re = ksum_get(&kr);
    *out_im = ksum_get(&ki);
}

/* Full table A_x(z) = <psi|X^x Z^z|psi> by the direct sum; out has 2*4^N
 * doubles, entry (x, z) at index x*d + z.  Small N only (tests). */
void sre_oracle_pauli_table_direct(const double *psi, int N, double *out) {
    const uint64_t d = (uint64_t)1 << N;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t x = 0; x < (int64_t)d; ++x)
        for (uint64_t z = 0; z < d; ++z)
            sre_oracle_pauli_expectation(psi, N, (uint64_t)x, z,
                                         &out[2 * ((uint64_t)x * d + z)],
                                         &out[2 * ((uint64_t)x * d + z) + 1]);
}

/*
 * O1: S by the definition, sum over all 4^N Pauli strings X^x Z^z of
 * |<psi|X^x Z^z|psi>|^4, each expectation from Eq. (Pauli_expect).
 * per_x (optional, length d) receives sum_z |A_x(z)|^4 for each x.
 */
double sre_oracle_sum4_direct(const double *psi, int N, double *per_x) {
    const uint64_t d = (uint64_t)1 << N;
    double *px = (double *)malloc(sizeof(double) * d);
    if (!px) return NAN;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t x = 0; x < (int64_t)d; ++x) {
        ksum_t k = {0.0, 0.0};
        for (uint64_t z = 0; z < d; ++z) {
            double re, im;
            sre_oracle_pauli_expectation(psi, N, (uint64_t)x, z, &re, &im);
            const double m2 = re * re + im * im;
            ksum_add(&k, m2 * m2);
        }
        px[x] = ksum_get(&k);
    }
    ksum_t tot = {0.0, 0.0};
    for (uint64_t x = 0; x < d; ++x) ksum_add(&tot, px[x]);
    if (per_x) memcpy(per_x, px, sizeof(double) * d);
    free(px);
    return ksum_get(&tot);
}

/*
 * Unnormalised fast Walsh-Hadamard transform, in place, of a complex vector
 * of length 2^N (interleaved re, im): N stages, stage h pairs entries i and
 * i+h inside blocks of 2h and maps (a, b) -> (a + b, a - b).  This is the
 * recursion H_{2^N} = [[H, H], [H, -H]] of the supplement's FWHT section,
 * so the result is sum_t (-1)^{popc(u&t)} a_t = sqrt(2^N) * WHT(a)(u).
 */
void sre_oracle_fwht(double *a, int N) {
    const uint64_t n = (uint64_t)1 << N;
    for (uint64_t h = 1; h < n; h <<= 1)
        for (uint64_t i = 0; i < n; i += 2 * h)
            for (uint64_t j = i; j < i + h; ++j) {
                const double ur = a[2 * j], ui = a[2 * j + 1];
                const double vr = a[2 * (j + h)], vi = a[2 * (j + h) + 1];
                a[2 * j] = ur + vr;
                a[2 * j + 1] = ui + vi;
                a[2 * (j + h)] = ur - vr;
                a[2 * (j + h) + 1] = ui - vi;
            }
}

/* For one shift x: G[t] = conj(psi[t^x]) psi[t], G <- FWHT(G) (Algorithm 1,
 * the loop body).  G has 2*2^N doubles. */
void sre_oracle_shift_transform(const double *psi, int N, uint64_t x, double *G) {
    const uint64_t d = (uint64_t)1 << N;
    for (uint64_t t = 0; t < d; ++t) {
        const double ar = psi[2 * (t ^ x)], ai = -psi[2 * (t ^ x) + 1];
        const double br = psi[2 * t], bi = psi[2 * t + 1];
        G[2 * t] = ar * br - ai * bi;
        G[2 * t + 1] = ar * bi + ai * br;
    }
    sre_oracle_fwht(G, N);
}

/*
 * O2: S by Algorithm 1 (XOR-FWHT), restated.  For every shift x in
 * [0, d): G[t] = conj(psi[t^x]) psi[t]; G <- FWHT(G); r += sum_u |G[u]|^4.
 * Shifts are independent (the paper's parallel axis); the per-shift sums
 * are kept and added in increasing x afterwards.
 * x_begin/x_end restrict the shift range (pass 0, d for all); per_x
 * (optional, length x_end - x_begin) receives each shift's sum.
 */
double sre_oracle_sum4_xorfwht_range(const double *psi, int N, uint64_t x_begin,
                                     uint64_t x_end, double *per_x) {
    const uint64_t d = (uint64_t)1 << N;
    if (x_end > d) x_end = d;
    if (x_begin >= x_end) return 0.0;
    const uint64_t nx = x_end - x_begin;
    double *px = (double *)malloc(sizeof(double) * nx);
    if (!px) return NAN;
    int fail = 0;
#pragma omp parallel
    {
        double *G = (double *)malloc(sizeof(double) * 2 * d);
        if (!G) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < (int64_t)nx; ++i) {
            if (!G) continue;
            sre_oracle_shift_transform(psi, N, x_begin + (uint64_t)i, G);
            ksum_t k = {0.0, 0.0};
            for (uint64_t u = 0; u < d; ++u) {
                const double m2 = G[2 * u] * G[2 * u] + G[2 * u + 1] * G[2 * u + 1];
                ksum_add(&k, m2 * m2);
            }
            px[i] = ksum_get(&k);
        }
        free(G);
    }
    if (fail) { free(px); return NAN; }
    ksum_t tot = {0.0, 0.0};
    for (uint64_t i = 0; i < nx; ++i) ksum_add(&tot, px[i]);
    if (per_x) memcpy(per_x, px, sizeof(double) * nx);
    free(px);
    return ksum_get(&tot);
}

double sre_oracle_sum4_xorfwht(const double *psi, int N, double *per_x) {
    return sre_oracle_sum4_xorfwht_range(psi, N, 0, (uint64_t)1 << N, per_x);
}

/* ---- general integer Renyi order (Eq. (sre)) ---------------------------
 *
 * Eq. (sre) defines, for Renyi index alpha,
 *     M_alpha = 1/(1 - alpha) * log2( (1/d) sum_P |<psi|P|psi>|^{2 alpha} )
 * over the 4^N Pauli strings of a normalised state.  For the stored state
 * the sum scales as n2^{2 alpha}, so with S_alpha = sum_{x,z} |A_x(z)|^{2 alpha}
 *     M_alpha = log2( S_alpha / (d * n2^{2 alpha}) ) / (1 - alpha).
 * alpha = 2 is M2 above.  Only integer alpha >= 2 is taken (the orders the
 * paper lists as magic monotones), so |A|^{2 alpha} = (|A|^2)^alpha is a plain
 * product of alpha factors.
 */
static double pow_int(double v, int k) {
    double p = 1.0;
    for (int i = 0; i < k; ++i) p *= v;
    return p;
}

/* O1 for order alpha: every expectation from Eq. (Pauli_expect) summed
 * directly, then |.|^{2 alpha} summed over all (x, z).  per_x as in O1. */
double sre_oracle_sum_pow_direct(const double *psi, int N, int alpha, double *per_x) {
    const uint64_t d = (uint64_t)1 << N;
    if (alpha < 1) return NAN;
    double *px = (double *)malloc(sizeof(double) * d);
    if (!px) return NAN;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t x = 0; x < (int64_t)d; ++x) {
        ksum_t k = {0.0, 0.0};
        for (uint64_t z = 0; z < d; ++z) {
            double re, im;
            sre_oracle_pauli_expectation(psi, N, (uint64_t)x, z, &re, &im);
            ksum_add(&k, pow_int(re * re + im * im, alpha));
        }
        px[x] = ksum_get(&k);
    }
    ksum_t tot = {0.0, 0.0};
    for (uint64_t x = 0; x < d; ++x) ksum_add(&tot, px[x]);
    if (per_x) memcpy(per_x, px, sizeof(double) * d);
    free(px);
    return ksum_get(&tot);
}

/* O2 for order alpha: Algorithm 1's loop (product, FWHT per shift) with the
 * exponent 2 alpha in place of 4 in the per-shift sum.  Range and per_x as in
 * sre_oracle_sum4_xorfwht_range. */
double sre_oracle_sum_pow_xorfwht_range(const double *psi, int N, int alpha, uint64_t x_begin,
                                        uint64_t x_end, double *per_x) {
    const uint64_t d = (uint64_t)1 << N;
    if (alpha < 1) return NAN;
    if (x_end > d) x_end = d;
    if (x_begin >= x_end) return 0.0;
    const uint64_t nx = x_end - x_begin;
    double *px = (double *)malloc(sizeof(double) * nx);
    if (!px) return NAN;
    int fail = 0;
#pragma omp parallel
    {
        double *G = (double *)malloc(sizeof(double) * 2 * d);
        if (!G) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < (int64_t)nx; ++i) {
            if (!G) continue;
            sre_oracle_shift_transform(psi, N, x_begin + (uint64_t)i, G);
            ksum_t k = {0.0, 0.0};
            for (uint64_t u = 0; u < d; ++u)
                ksum_add(&k, pow_int(G[2 * u] * G[2 * u] + G[2 * u + 1] * G[2 * u + 1], alpha));
            px[i] = ksum_get(&k);
        }
        free(G);
    }
    if (fail) { free(px); return NAN; }
    ksum_t tot = {0.0, 0.0};
    for (uint64_t i = 0; i < nx; ++i) ksum_add(&tot, px[i]);
    if (per_x) memcpy(per_x, px, sizeof(double) * nx);
    free(px);
    return ksum_get(&tot);
}

/* M_alpha of Eq. (sre) for integer alpha >= 2; method 0 = O1, 1 = O2. */
double sre_oracle_malpha(const double *psi, int N, int alpha, int method) {
    if (alpha < 2) return NAN;
    const double n2 = sre_oracle_norm2(psi, N);
    const double S = method == 0 ? sre_oracle_sum_pow_direct(psi, N, alpha, NULL)
                                 : sre_oracle_sum_pow_xorfwht_range(psi, N, alpha, 0, (uint64_t)1 << N, NULL);
    const double d = ldexp(1.0, N);
    return log2(S / (d * pow_int(n2, 2 * alpha))) / (1.0 - alpha);
}

/* M2 = -log2(S / (d * n2^4)), Algorithm 1's return value for the state
 * normalised to n2 = 1.  method 0 = O1 (direct), 1 = O2 (XOR-FWHT). */
double sre_oracle_m2(const double *psi, int N, int method) {
    const double n2 = sre_oracle_norm2(psi, N);
    const double S = method == 0 ? sre_oracle_sum4_direct(psi, N, NULL)
                                 : sre_oracle_sum4_xorfwht(psi, N, NULL);
    const double d = ldexp(1.0, N);
    return -log2(S / (d * n2 * n2 * n2 * n2));
}
