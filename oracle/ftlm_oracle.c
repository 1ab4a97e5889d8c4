/*
 * ftlm_oracle.c -- plain, slow, FP64 CPU oracle for the FTLM hot path (spin 1/2,
 * and general spin s in the or_spin_* routines at the end).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file; only the test-suite, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code with the CUDA library.
 *
 * Every routine below is the plain definition of the step it implements, written
 * out without blocking, fusion or reordering:
 *
 *   - sector basis:   Eq. 11 (label n = sum_k a_k 2^k, a_k = m_k + 1/2) and Eq. 17
 *                     (digit sum A_tot = N/2 + M); the basis is every N-bit label
 *                     with that digit sum, in increasing label order (Sec. 2, CLT
 *                     paragraph).  Enumerated by brute force over all 2^N labels.
 *   - index map:      a full lookup table, one int32 per label of the full space
 *                     (Sec. 2, "State-to-index mapping"), or a binary search of the
 *                     sorted basis.  Neither is the CLT nor the combinatorial rank.
 *   - CLT arrays:     Eq. 18 built by one pass over the sorted basis followed by a
 *                     cumulative popcount (Sec. 2, CLT construction); the lookup of
 *                     Eq. 19-20 / Algorithm 2 is provided to pin the worked example.
 *   - H.v:            Eq. 12 with the ladder coefficients of Eq. 13-14 evaluated at
 *                     s = 1/2, per-bond J_b, summed in bond-list order.
 *   - start vectors:  splitmix64 (Steele, Lea & Flood, OOPSLA 2014) used as a
 *                     counter-based generator; Gaussian entries by the Box-Muller
 *                     transform (Box & Muller 1958), Rademacher entries from the top
 *                     bit.  The vector definition is stated in or_start_vector.
 *   - Lanczos:        three-term recurrence without reorthogonalization (Sec. 2,
 *                     FTLM paragraph), in Paige's ordering, FP64 throughout.
 *
 * The small tridiagonal eigenproblem and the thermodynamic sums (Eq. 4-9) live in
 * the Python half of the oracle (ftlm.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_S 0.5 /* local spin */

static int or_bit(uint64_t n, int k) { return (int)((n >> k) & 1u); }

/* Digit sum of an N-bit label (Eq. 11 with d = 2: the number of up spins). */
static int or_digit_sum(uint64_t n, int N)
{
    (void)N; /* labels passed here are below 2^N */
    return __builtin_popcountll(n);
}

/* Sector basis (Eq. 11, Eq. 17): all labels 0 <= n < 2^N whose digit sum equals
 * K = A_tot, in increasing order.  Writes at most cap labels; returns the sector
 * dimension D (which may exceed cap, in which case only the first cap are stored).
 */
int64_t or_basis_enumerate(int N, int K, uint64_t *out, int64_t cap)
{
    int64_t D = 0;
    uint64_t full = (uint64_t)1 << N;
    for (uint64_t n = 0; n < full; ++n) {
        if (or_digit_sum(n, N) != K) continue;
        if (out && D < cap) out[D] = n;
        ++D;
    }
    return D;
}

/* Full lookup table (Sec. 2): lut[n] = sector index of label n, -1 if n is not in
 * the sector.  lut has 2^N entries. */
void or_full_lut(int N, const uint64_t *basis, int64_t D, int32_t *lut)
{
    uint64_t full = (uint64_t)1 << N;
    for (uint64_t n = 0; n < full; ++n) lut[n] = -1;
    for (int64_t t = 0; t < D; ++t) lut[basis[t]] = (int32_t)t;
}

/* Sector index of a label by binary search of the sorted basis; -1 if absent. */
int64_t or_index_bsearch(const uint64_t *basis, int64_t D, uint64_t label)
{
    int64_t lo = 0, hi = D; /* search [lo, hi) */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (basis[mid] < label) lo = mid + 1;
        else hi = mid;
    }
    if (lo < D && basis[lo] == label) return lo;
    return -1;
}

/* CLT construction (Eq. 18): blocks of 32 labels over the full label space
 * [0, 2^N); mask bit j of block b is set iff label 32b + j is in the sector;
 * prefix[b] is the number of in-sector labels in blocks 0..b-1.  nblocks must be
 * ceil(2^N / 32). */
void or_clt_build(int N, const uint64_t *basis, int64_t D, uint32_t *mask, uint32_t *prefix,
                  int64_t nblocks)
{
    (void)N;
    memset(mask, 0, (size_t)nblocks * sizeof(uint32_t));
    for (int64_t t = 0; t < D; ++t) {
        uint64_t n = basis[t];
        mask[n / 32] |= (uint32_t)1 << (n % 32);
    }
    uint64_t running = 0;
    for (int64_t b = 0; b < nblocks; ++b) {
        prefix[b] = (uint32_t)running;
        running += (uint64_t)__builtin_popcount(mask[b]);
    }
}

/* CLT lookup (Eq. 19-20, Algorithm 2); -1 when the occupancy bit is clear. */
int64_t or_clt_lookup(const uint32_t *mask, const uint32_t *prefix, uint64_t n)
{
    uint64_t b = n / 32;
    uint32_t j = (uint32_t)(n % 32);
    if (((mask[b] >> j) & 1u) == 0) return -1;
    uint32_t below = (j == 0) ? 0u : (mask[b] & ((1u << j) - 1u));
    return (int64_t)prefix[b] + __builtin_popcount(below);
}

/* Index of a label: full LUT when given, else binary search. */
static int64_t or_index(const uint64_t *basis, int64_t D, const int32_t *lut, uint64_t n)
{
    if (lut) return lut[n];
    return or_index_bsearch(basis, D, n);
}

/* One row of Eq. 12 with s = 1/2:
 *   y[t] = sum_b J_b m_i m_j x[t] + sum_b ( c+_b x[idx(n+_b)] + c-_b x[idx(n-_b)] )
 * where n+ is the source label with (m_i - 1, m_j + 1) and coefficient Eq. 13,
 * and n- the source label with (m_i + 1, m_j - 1) and coefficient Eq. 14; both
 * coefficients use the m values of the row (target) state n_t. */
static double or_hv_row(int nb, const int *bi, const int *bj, const double *J,
                        const uint64_t *basis, int64_t D, const int32_t *lut, const double *x,
                        int64_t t)
{
    const double s = OR_S, ss1 = OR_S * (OR_S + 1.0);
    uint64_t n = basis[t];
    double diag = 0.0, off = 0.0;
    for (int b = 0; b < nb; ++b) {
        int i = bi[b], j = bj[b];
        double mi = (double)or_bit(n, i) - s;
        double mj = (double)or_bit(n, j) - s;
        diag += J[b] * mi * mj;
        /* s_i^+ s_j^- term: source has m_i - 1 >= -s and m_j + 1 <= s (Eq. 13). */
        if (mi - 1.0 >= -s && mj + 1.0 <= s) {
            double cp = 0.5 * J[b] * sqrt(ss1 - mi * (mi - 1.0)) * sqrt(ss1 - mj * (mj + 1.0));
            uint64_t src = n - ((uint64_t)1 << i) + ((uint64_t)1 << j);
            int64_t k = or_index(basis, D, lut, src);
            off += cp * x[k];
        }
        /* s_i^- s_j^+ term: source has m_i + 1 <= s and m_j - 1 >= -s (Eq. 14). */
        if (mi + 1.0 <= s && mj - 1.0 >= -s) {
            double cm = 0.5 * J[b] * sqrt(ss1 - mi * (mi + 1.0)) * sqrt(ss1 - mj * (mj - 1.0));
            uint64_t src = n + ((uint64_t)1 << i) - ((uint64_t)1 << j);
            int64_t k = or_index(basis, D, lut, src);
            off += cm * x[k];
        }
    }
    return diag * x[t] + off;
}

/* Rows t0 <= t < t1 of H.v (Eq. 12) into y[t - t0]; rows are independent, so the
 * OpenMP split over rows does not change any result. */
void or_hv_range(int nb, const int *bi, const int *bj, const double *J, const uint64_t *basis,
                 int64_t D, const int32_t *lut, const double *x, double *y, int64_t t0, int64_t t1)
{
#pragma omp parallel for schedule(static)
    for (int64_t t = t0; t < t1; ++t)
        y[t - t0] = or_hv_row(nb, bi, bj, J, basis, D, lut, x, t);
}

/* H.v over the whole sector. */
void or_hv(int nb, const int *bi, const int *bj, const double *J, const uint64_t *basis,
           int64_t D, const int32_t *lut, const double *x, double *y)
{
    or_hv_range(nb, bi, bj, J, basis, D, lut, x, y, 0, D);
}

/* Number of nonzero off-diagonal terms applied by one H.v (each valid ladder move
 * of each row); with the D diagonal entries this is N_nz of Eq. 10. */
int64_t or_offdiag_terms(int nb, const int *bi, const int *bj, const uint64_t *basis, int64_t D)
{
    int64_t cnt = 0;
    for (int64_t t = 0; t < D; ++t)
        for (int b = 0; b < nb; ++b)
            if (or_bit(basis[t], bi[b]) != or_bit(basis[t], bj[b])) ++cnt;
    return cnt;
}

/* ---- counter-based random start vectors --------------------------------------
 * splitmix64 output function applied to the generator state (published constants
 * of Steele, Lea & Flood 2014).  The c-th output (c = 0, 1, ...) of a splitmix64
 * generator started from state k is F(k + (c + 1) * GAMMA).
 */
static const uint64_t OR_GAMMA = 0x9E3779B97F4A7C15ull;

static uint64_t or_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* c-th output of splitmix64 started from state k. */
uint64_t or_splitmix64_at(uint64_t k, uint64_t c) { return or_mix64(k + (c + 1) * OR_GAMMA); }

/* Key of chain r of sector (N, K) under seed:
 *   key = F(F(seed + GAMMA) + tag + GAMMA),  tag = N << 48 | K << 32 | r. */
uint64_t or_chain_key(uint64_t seed, int N, int K, uint32_t r)
{
    uint64_t tag = ((uint64_t)N << 48) | ((uint64_t)K << 32) | (uint64_t)r;
    return or_mix64(or_mix64(seed + OR_GAMMA) + tag + OR_GAMMA);
}

/* Start vector of chain r (not normalized; the recurrence normalizes it):
 *   dist 0 (Gaussian):   U1 = ((u(2t) >> 11) + 1) 2^-53,  U2 = (u(2t+1) >> 11) 2^-53,
 *                        x_t = sqrt(-2 ln U1) cos(2 pi U2);
 *   dist 1 (Rademacher): x_t = +1 if the top bit of u(t) is 0, else -1;
 * where u(c) is the c-th splitmix64 output from the chain key and t is the sector
 * index (the basis is ordered by label, so index and label are in bijection). */
void or_start_vector(uint64_t seed, int N, int K, uint32_t r, int dist, int64_t D, double *out)
{
    const double two53 = 9007199254740992.0; /* 2^53 */
    const double pi = 3.14159265358979323846;
    uint64_t key = or_chain_key(seed, N, K, r);
    for (int64_t t = 0; t < D; ++t) {
        if (dist == 1) {
            uint64_t u = or_splitmix64_at(key, (uint64_t)t);
            out[t] = (u >> 63) ? -1.0 : 1.0;
        } else {
            uint64_t u1 = or_splitmix64_at(key, 2 * (uint64_t)t);
            uint64_t u2 = or_splitmix64_at(key, 2 * (uint64_t)t + 1);
            double U1 = ((double)(u1 >> 11) + 1.0) / two53;
            double U2 = (double)(u2 >> 11) / two53;
            out[t] = sqrt(-2.0 * log(U1)) * cos(2.0 * pi * U2);
        }
    }
}

/* ---- Lanczos recurrence (Sec. 2, FTLM paragraph), Paige's ordering -----------
 *   q_0 = 0, beta_0 = 0, q_1 = r / ||r||;  for j = 1 .. m_max = min(M, D):
 *     y = H q_j - beta_{j-1} q_{j-1};  alpha_j = <q_j, y>;  w = y - alpha_j q_j;
 *     stop after step j when j = m_max;  beta_j = ||w||;
 *     stop after step j (m_eff = j) when beta_j <= tau;  q_{j+1} = w / beta_j.
 * Writes alpha[0..m_eff-1], beta[0..m_eff-2] (beta_j for j < m_eff) and returns
 * m_eff.  No reorthogonalization. */
int or_lanczos(int nb, const int *bi, const int *bj, const double *J, const uint64_t *basis,
               int64_t D, const int32_t *lut, const double *r, int M, double tau, double *alpha,
               double *beta)
{
    int m_max = (int64_t)M < D ? M : (int)D;
    double *qp = (double *)calloc((size_t)D, sizeof(double));
    double *q = (double *)malloc((size_t)D * sizeof(double));
    double *y = (double *)malloc((size_t)D * sizeof(double));
    double nr = 0.0;
    for (int64_t t = 0; t < D; ++t) nr += r[t] * r[t];
    nr = sqrt(nr);
    for (int64_t t = 0; t < D; ++t) q[t] = r[t] / nr;
    double beta_prev = 0.0;
    int m_eff = m_max;
    for (int j = 1; j <= m_max; ++j) {
        or_hv(nb, bi, bj, J, basis, D, lut, q, y);
        for (int64_t t = 0; t < D; ++t) y[t] -= beta_prev * qp[t];
        double a = 0.0;
        for (int64_t t = 0; t < D; ++t) a += q[t] * y[t];
        alpha[j - 1] = a;
        for (int64_t t = 0; t < D; ++t) y[t] -= a * q[t]; /* y now holds w */
        if (j == m_max) break;
        double bsq = 0.0;
        for (int64_t t = 0; t < D; ++t) bsq += y[t] * y[t];
        double bj_ = sqrt(bsq);
        if (bj_ <= tau) {
            m_eff = j;
            break;
        }
        beta[j - 1] = bj_;
        for (int64_t t = 0; t < D; ++t) {
            qp[t] = q[t];
            q[t] = y[t] / bj_;
        }
        beta_prev = bj_;
    }
    free(qp);
    free(q);
    free(y);
    return m_eff;
}

/* ---- general local spin s (Sec. 2: Eq. 10-14 with d = 2s + 1 digits) -----------
 * A label n = sum_k a_k d^k (Eq. 11) carries the shifted quantum numbers
 * a_k = m_k + s in 0 .. 2s as base-d digits; the sector of total S^z = M holds
 * the labels with digit sum A = N s + M (Eq. 17), in increasing label order.
 * two_s = 2s >= 1; two_s = 1 is the spin-1/2 case above. */
static uint64_t or_ipow(uint64_t d, int k)
{
    uint64_t p = 1;
    for (int i = 0; i < k; ++i) p *= d;
    return p;
}

/* k-th base-d digit of n: floor(n / d^k) mod d (Sec. 2, after Eq. 11). */
static int or_spin_digit(uint64_t n, int d, int k) { return (int)((n / or_ipow((uint64_t)d, k)) % (uint64_t)d); }

/* Sector basis for spin s: every label 0 <= n < d^N with digit sum A, ascending.
 * Writes at most cap labels; returns the dimension. */
int64_t or_spin_basis_enumerate(int N, int two_s, int A, uint64_t *out, int64_t cap)
{
    const int d = two_s + 1;
    const uint64_t full = or_ipow((uint64_t)d, N);
    int a[64] = {0}; /* digits of n, counted up like an odometer alongside n */
    int sum = 0;
    int64_t D = 0;
    for (uint64_t n = 0; n < full; ++n) {
        if (sum == A) {
            if (out && D < cap) out[D] = n;
            ++D;
        }
        for (int k = 0; k < N; ++k) { /* n + 1 */
            if (a[k] + 1 < d) {
                ++a[k];
                ++sum;
                break;
            }
            sum -= a[k];
            a[k] = 0;
        }
    }
    return D;
}

/* One row of Eq. 12 for spin s: diagonal sum_b J_b m_i m_j, plus for every bond
 * the source with (m_i - 1, m_j + 1) weighted by Eq. 13 and the source with
 * (m_i + 1, m_j - 1) weighted by Eq. 14 (m values of the row state), each present
 * when the source quantum numbers stay within -s .. s.  Sources are located by
 * binary search of the sorted basis. */
static double or_spin_hv_row(int N, int two_s, int nb, const int *bi, const int *bj, const double *J,
                             const uint64_t *basis, int64_t D, const double *x, int64_t t)
{
    const int d = two_s + 1;
    const double s = 0.5 * two_s, ss1 = s * (s + 1.0);
    const uint64_t n = basis[t];
    double diag = 0.0, off = 0.0;
    (void)N;
    for (int b = 0; b < nb; ++b) {
        const int i = bi[b], j = bj[b];
        const double mi = (double)or_spin_digit(n, d, i) - s;
        const double mj = (double)or_spin_digit(n, d, j) - s;
        const uint64_t di = or_ipow((uint64_t)d, i), dj = or_ipow((uint64_t)d, j);
        diag += J[b] * mi * mj;
        if (mi - 1.0 >= -s && mj + 1.0 <= s) {
            const double cp = 0.5 * J[b] * sqrt(ss1 - mi * (mi - 1.0)) * sqrt(ss1 - mj * (mj + 1.0));
            const int64_t k = or_index_bsearch(basis, D, n - di + dj);
            off += cp * x[k];
        }
        if (mi + 1.0 <= s && mj - 1.0 >= -s) {
            const double cm = 0.5 * J[b] * sqrt(ss1 - mi * (mi + 1.0)) * sqrt(ss1 - mj * (mj - 1.0));
            const int64_t k = or_index_bsearch(basis, D, n + di - dj);
            off += cm * x[k];
        }
    }
    return diag * x[t] + off;
}

void or_spin_hv_range(int N, int two_s, int nb, const int *bi, const int *bj, const double *J,
                      const uint64_t *basis, int64_t D, const double *x, double *y, int64_t t0, int64_t t1)
{
#pragma omp parallel for schedule(static)
    for (int64_t t = t0; t < t1; ++t)
        y[t - t0] = or_spin_hv_row(N, two_s, nb, bi, bj, J, basis, D, x, t);
}

/* Nonzero off-diagonal terms of one spin-s H.v: every ladder move of Eq. 13 or
 * Eq. 14 whose coefficient is nonzero (with the D diagonal entries, N_nz of Eq. 10). */
int64_t or_spin_offdiag_terms(int N, int two_s, int nb, const int *bi, const int *bj, const uint64_t *basis,
                              int64_t D)
{
    const int d = two_s + 1;
    int64_t cnt = 0;
    (void)N;
#pragma omp parallel for schedule(static) reduction(+ : cnt)
    for (int64_t t = 0; t < D; ++t)
        for (int b = 0; b < nb; ++b) {
            const int ai = or_spin_digit(basis[t], d, bi[b]), aj = or_spin_digit(basis[t], d, bj[b]);
            cnt += (ai >= 1 && aj <= two_s - 1) + (ai <= two_s - 1 && aj >= 1);
        }
    return cnt;
}

/* Threads of the following OpenMP loops (ignored when built without OpenMP). */
void or_set_num_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Number of OpenMP threads the H.v loop uses (1 when built without OpenMP). */
int or_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
