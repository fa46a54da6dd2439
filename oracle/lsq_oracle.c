/*
 * Plain, slow CPU oracle for randomized-preconditioned normal equations
 * (Garrison & Ipsen, "Perturbation Analysis for Preconditioned Normal
 * Equations in Mixed Precision", arXiv 2603.16644).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link,
 * load or call this file; only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg do.  It shares no code, header, table or
 * constant generator with the CUDA library.
 *
 * Conventions
 *   - Matrices are column-major: entry (i, j) of an m-by-n matrix with
 *     leading dimension ld sits at [i + j*ld].
 *   - Everything is FP64 unless a step of the method fixes a lower
 *     precision; lower precision is emulated by explicit round-to-nearest-
 *     even (RNE) conversions and, for FP32 arithmetic, by C `float`
 *     operations.  Build with -ffp-contract=off so that no multiply-add is
 *     fused behind our back: every product and sum below is rounded once.
 *   - Loops run in plain index order; there is no blocking, fusion or
 *     reordering, so each function can be checked against its source by eye.
 *   - Loops whose iterations are independent (rows of a substitution,
 *     entries of a Gram matrix, columns of a reflector update, rows of the
 *     sketch) are spread over threads with OpenMP.  Every sum still runs in
 *     its own index order inside one thread, so the result is bit-identical
 *     for any thread count (lsqo_set_threads; a CPU test checks this).
 *
 * Precision codes: 0 FP8-e4m3 (OCP "fn", saturating), 1 BF16, 2 FP16,
 * 3 FP32, 4 FP64, 5 AUTO (choose by the condition estimate of A^T A),
 * 6 AUTO_SKETCH (choose by the condition estimate on a sketch).
 * Sketch kinds: 0 Gaussian, 1 sparse sign, 2 subsampled randomized
 * Walsh-Hadamard transform (the paper's S F D of Eq. e_sketch).
 *
 * Pins (checked by the CPU-only tests against the mathematics, never
 * against the CUDA path): rounding exhaustively against the IEEE/OCP format
 * definitions; Philox against the published known-answer vectors; the
 * sparse-sign stream against its distinctness/uniformity invariants; the
 * Householder least-squares solve against exact rational arithmetic and
 * generated problems with known solutions; QR against the Cholesky factor of
 * the sketch Gram matrix; PNE/HPNE against exact solutions for any
 * nonsingular R_s and against the error bounds Eq. (eq41)/(eq32); the
 * condition estimate against the exact inverse 1-norm (it is a lower bound)
 * and the kappa^2 inequality of Sec. 6.1; the Gaussian entries against
 * the ziggurat evaluated in 40-digit arithmetic (tables from the closure
 * equation solved afresh, within the FP64 error of the libm calls) besides
 * their distribution.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { O_FP8 = 0, O_BF16 = 1, O_FP16 = 2, O_FP32 = 3, O_FP64 = 4, O_AUTO = 5, O_AUTO_SKETCH = 6 };
enum { O_GAUSSIAN = 0, O_SPARSE_SIGN = 1, O_SRFT = 2 };

#define IDX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

/* Threads used by the parallel loops (n <= 0 leaves the setting); returns
 * the previous count.  1 when built without OpenMP. */
int lsqo_set_threads(int n)
{
#ifdef _OPENMP
    int prev = omp_get_max_threads();
    if (n > 0) omp_set_num_threads(n);
    return prev;
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------------
 * Rounding FP64 -> lower precision, one rounding, RNE, subnormals kept.
 * A format is (p significand bits incl. the implicit one, minimum normal
 * exponent emin, largest finite value, saturate-or-overflow).
 * ---------------------------------------------------------------------- */
static double rne_format(double x, int p, int emin, double maxfin, int sat)
{
    if (isnan(x) || x == 0.0) return x;
    if (isinf(x)) return sat ? copysign(maxfin, x) : x;
    double a = fabs(x);
    int E;
    frexp(a, &E);            /* a = f * 2^E with f in [0.5, 1) */
    int e = E - 1;           /* floor(log2(a)) */
    if (e < emin) e = emin;  /* subnormal range: fixed quantum */
    int q = e - (p - 1);     /* exponent of one unit in the last place */
    double r = rint(ldexp(a, -q)); /* exact scaling, then RNE to integer */
    double y = ldexp(r, q);
    if (y > maxfin) y = sat ? maxfin : INFINITY;
    return copysign(y, x);
}

double lsqo_round(double x, int prec)
{
    switch (prec) {
    case O_FP8:  return rne_format(x, 4, -6, 448.0, 1);
    case O_BF16: return rne_format(x, 8, -126, 0x1.fep127, 0);
    case O_FP16: return rne_format(x, 11, -14, 65504.0, 0);
    case O_FP32: return rne_format(x, 24, -126, 0x1.fffffep127, 0);
    default:     return x;
    }
}

void lsqo_round_array(const double* x, int64_t len, int prec, double* y)
{
    for (int64_t i = 0; i < len; ++i) y[i] = lsqo_round(x[i], prec);
}

/* ------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random
 * numbers: as easy as 1, 2, 3"): ten rounds of two 32x32->64 multiplies
 * with the published multipliers, key bumped by the published Weyl
 * constants between rounds.
 * ---------------------------------------------------------------------- */
void lsqo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------
 * Sketch operators (Alg. 1 takes a random d-by-m sketch; the sparse-sign
 * and Gaussian families stand in for the paper's SRFT of Eq. (e_sketch)).
 *
 * Sparse sign, column j of Omega (s-by-m): zeta DISTINCT rows in [0, s),
 * drawn in order from the Philox stream key = seed, counter =
 * (block k, j_lo, j_hi, 0), words consumed w0..w3 per block; each word is
 * mapped to [0, s) by Lemire's multiply-shift with rejection of the low
 * product below (2^32 - s) mod s, and duplicates are rejected.  Sign of the
 * t-th accepted row: bit t of word 0 of counter (0, j_lo, j_hi, 1), 1 = -1.
 * ---------------------------------------------------------------------- */
int lsqo_sparse_sign_column(uint64_t seed, int64_t j, int64_t s, int zeta,
                            int32_t* idx, int8_t* sgn)
{
    if (s <= 0 || s > 0x7fffffff || zeta <= 0 || zeta > 32 || zeta > s) return -1;
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t su = (uint32_t)s;
    uint32_t thresh = (uint32_t)(0u - su) % su;
    int got = 0;
    for (uint32_t k = 0; got < zeta; ++k) {
        if (k > (1u << 20)) return -2;
        uint32_t ctr[4] = { k, (uint32_t)j, (uint32_t)((uint64_t)j >> 32), 0u };
        uint32_t w[4];
        lsqo_philox4x32_10(ctr, key, w);
        for (int t = 0; t < 4 && got < zeta; ++t) {
            uint64_t prod = (uint64_t)w[t] * (uint64_t)su;
            if ((uint32_t)prod < thresh) continue;
            int32_t cand = (int32_t)(prod >> 32);
            int dup = 0;
            for (int q = 0; q < got; ++q) dup |= (idx[q] == cand);
            if (!dup) idx[got++] = cand;
        }
    }
    uint32_t ctr[4] = { 0u, (uint32_t)j, (uint32_t)((uint64_t)j >> 32), 1u };
    uint32_t w[4];
    lsqo_philox4x32_10(ctr, key, w);
    for (int t = 0; t < zeta; ++t) sgn[t] = ((w[0] >> t) & 1u) ? (int8_t)-1 : (int8_t)1;
    return 0;
}

int lsqo_sparse_sign_indices(uint64_t seed, int64_t m, int64_t s, int zeta,
                             int32_t* idx /* m*zeta */, int8_t* sgn /* m*zeta */)
{
    int rc = 0;
#pragma omp parallel for schedule(static) reduction(min : rc)
    for (int64_t j = 0; j < m; ++j) {
        int r = lsqo_sparse_sign_column(seed, j, s, zeta, idx + j * zeta, sgn + j * zeta);
        if (r < rc) rc = r;
    }
    return rc;
}

/* ------------------------------------------------------------------------
 * Gaussian entries by the ziggurat method (Marsaglia & Tsang, "The Ziggurat
 * Method for Generating Random Variables", J. Stat. Softw. 5(8), 2000) with
 * 256 layers.  The paper fixes only the distribution of Omega (i.i.d.
 * N(0, 1) entries, the Gaussian embedding of Sec. 6.2); the ziggurat draws
 * it with one table lookup and one product in more than 99 % of the draws.
 *
 * Layers of equal area v under f(x) = exp(-x^2 / 2), x >= 0:
 *   layer 0: the rectangle [0, r] x [0, f(r)] plus the tail x > r, drawn as
 *            a rectangle of width x_0 = v / f(r);
 *   layer i (1 <= i <= 255): [0, x_i] x [f(x_i), f(x_{i+1})], so that
 *            f(x_{i+1}) = f(x_i) + v / x_i, with x_1 = r and x_256 = 0.
 * v = r f(r) + int_r^inf f = r f(r) + sqrt(pi / 2) erfc(r / sqrt(2)), and r
 * is the root of the closure f(x_255) + v / x_255 = 1 (3.6541528853610088,
 * the 256-layer value).
 * ---------------------------------------------------------------------- */
#define ZIG_N 256
#define ZIG_R 3.6541528853610088
#define ZIG_ROUNDS 64
static double zig_x[ZIG_N + 1], zig_f[ZIG_N + 1];

__attribute__((constructor)) static void zig_tables(void)
{
    const double fr = exp(-0.5 * ZIG_R * ZIG_R);
    const double tail = sqrt(0.5 * 3.14159265358979323846) * erfc(ZIG_R / sqrt(2.0));
    const double v = ZIG_R * fr + tail;
    zig_x[0] = v / fr;
    zig_x[1] = ZIG_R;
    zig_f[0] = 0.0;
    zig_f[1] = fr;
    for (int i = 1; i < ZIG_N - 1; ++i) {
        double next = zig_f[i] + v / zig_x[i];   /* f(x_{i+1}) */
        zig_x[i + 1] = sqrt(-2.0 * log(next));
        zig_f[i + 1] = exp(-0.5 * zig_x[i + 1] * zig_x[i + 1]);
    }
    zig_x[ZIG_N] = 0.0;
    zig_f[ZIG_N] = 1.0;
}

/* The tables x_0..x_256, f(x_0..x_256) (f(x_0) stored as 0). */
void lsqo_zig_tables(double* x, double* f)
{
    memcpy(x, zig_x, sizeof zig_x);
    memcpy(f, zig_f, sizeof zig_f);
}

/* Gaussian entry Omega(i, j).  Round k draws the Philox block of counter
 * (i, j_lo, j_hi, 2 + 256 k).  A first-kind round reads
 *   layer L = w0 & 255, sign = bit 8 of w0,
 *   U = (2^30 (w0 >> 9) + (w1 >> 2)) / 2^53 in [0, 1),
 *   V = (2^26 (w2 >> 5) + (w3 >> 6)) / 2^53 in [0, 1),
 * and proposes z = U x_L.  It keeps z if z < x_{L+1} (inside the curve);
 * in layer L >= 1 otherwise if f(x_L) + V (f(x_{L+1}) - f(x_L)) < f(z) (the
 * wedge); else the next round is a first-kind round again.  In layer 0 with
 * z >= r the next rounds sample the tail (Marsaglia 1964): U1, U2 in (0, 1]
 * from (w0, w1) and (w2, w3) as V plus 1 / 2^53, e1 = -ln(U1) / r,
 * e2 = -ln(U2), kept when 2 e2 > e1^2, giving r + e1.  The sign applies last.
 * After 64 rounds (probability below 1e-100) the draw is 0.
 * The entry is the draw rounded to the nearest multiple of 2^-17 (ties to
 * even) and clamped to |Omega| <= 8 - 2^-17: 20 significant bits, so an
 * FP32 value, and three balanced base-128 digits below any row maximum
 * under 8 (the FP64 sketch's digit-sliced product needs no more).  The
 * change of law is below 2^-18 per entry. */
static double zig_grid(double z)
{
    const double lim = 8.0 - 0x1p-17;
    double q = rint(z * 131072.0) * 0x1p-17;
    return q > lim ? lim : (q < -lim ? -lim : q);
}

double lsqo_gaussian_entry(uint64_t seed, int64_t i, int64_t j)
{
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t ctr[4] = { (uint32_t)i, (uint32_t)j, (uint32_t)((uint64_t)j >> 32), 2u };
    uint32_t w[4];
    int tail = 0;
    double sign = 1.0;
    for (uint32_t k = 0; k < ZIG_ROUNDS; ++k) {
        ctr[3] = 2u + 256u * k;
        lsqo_philox4x32_10(ctr, key, w);
        if (tail) {
            double u1 = ((double)((uint64_t)(w[0] >> 5) * 67108864ull + (w[1] >> 6)) + 1.0) * 0x1p-53;
            double u2 = ((double)((uint64_t)(w[2] >> 5) * 67108864ull + (w[3] >> 6)) + 1.0) * 0x1p-53;
            double e1 = -log(u1) / ZIG_R;
            double e2 = -log(u2);
            if (e2 + e2 > e1 * e1) return zig_grid(sign * (ZIG_R + e1));
            continue;
        }
        int L = (int)(w[0] & 255u);
        sign = (w[0] >> 8) & 1u ? -1.0 : 1.0;
        double U = (double)((uint64_t)(w[0] >> 9) * 1073741824ull + (w[1] >> 2)) * 0x1p-53;
        double z = U * zig_x[L];
        if (z < zig_x[L + 1]) return zig_grid(sign * z);
        if (L == 0) {
            tail = 1;
            continue;
        }
        double V = (double)((uint64_t)(w[2] >> 5) * 67108864ull + (w[3] >> 6)) * 0x1p-53;
        double y = zig_f[L] + V * (zig_f[L + 1] - zig_f[L]);
        if (y < exp(-0.5 * z * z)) return zig_grid(sign * z);
    }
    return 0.0;
}

void lsqo_gaussian_operator(uint64_t seed, int64_t s, int64_t m, int prec, double* Om /* s-by-m, ld s */)
{
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < m; ++j)
        for (int64_t i = 0; i < s; ++i)
            Om[IDX(i, j, s)] = lsqo_round(lsqo_gaussian_entry(seed, i, j), prec);
}

/* ------------------------------------------------------------------------
 * Subsampled randomized trigonometric transform, Omega = S F D (Eq. e_sketch,
 * Sec. 6.2), with F the real Sylvester-Walsh-Hadamard transform of order
 * m' = the smallest power of two >= m (A padded with zero rows), unscaled
 * entries +-1:
 *   D: sign of row j < m from the Philox stream key = seed, counter
 *      (j >> 7, 0, 0, 3): bit (j & 31) of word (j >> 5) & 3, set = -1;
 *   F: (F x)_r = sum_j (-1)^popcount(r & j) x_j, evaluated by the butterfly
 *      levels h = 1, 2, 4, ..., m'/2 in that order, (a, b) -> (a + b, a - b)
 *      on the pairs (i, i + h) with i & h = 0;
 *   S: d rows of I_{m'} sampled uniformly WITH replacement: row of sample t
 *      = word (t & 3) of counter (t >> 2, 0, 0, 4), masked to [0, m').
 * ---------------------------------------------------------------------- */
int64_t lsqo_srft_order(int64_t m)
{
    int64_t mp = 1;
    while (mp < m) mp <<= 1;
    return mp;
}

int lsqo_srft_sign(uint64_t seed, int64_t j)
{
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t ctr[4] = { (uint32_t)((uint64_t)j >> 7), 0u, 0u, 3u };
    uint32_t w[4];
    lsqo_philox4x32_10(ctr, key, w);
    return ((w[(j >> 5) & 3] >> (j & 31)) & 1u) ? -1 : 1;
}

int64_t lsqo_srft_row(uint64_t seed, int64_t t, int64_t mp)
{
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t ctr[4] = { (uint32_t)((uint64_t)t >> 2), 0u, 0u, 4u };
    uint32_t w[4];
    lsqo_philox4x32_10(ctr, key, w);
    return (int64_t)(w[t & 3] & (uint32_t)(mp - 1));
}

/* In-place Walsh-Hadamard transform of length mp (a power of two), FP64 and
 * FP32 arithmetic. */
void lsqo_fwht(double* x, int64_t mp)
{
    for (int64_t h = 1; h < mp; h <<= 1)
        for (int64_t i = 0; i < mp; ++i)
            if (!(i & h)) {
                double a = x[i], b = x[i + h];
                x[i] = a + b;
                x[i + h] = a - b;
            }
}

static void fwht32(float* x, int64_t mp)
{
    for (int64_t h = 1; h < mp; h <<= 1)
        for (int64_t i = 0; i < mp; ++i)
            if (!(i & h)) {
                float a = x[i], b = x[i + h];
                x[i] = a + b;
                x[i + h] = a - b;
            }
}

/* ------------------------------------------------------------------------
 * Per-column power-of-two scaling before rounding A to the sketch precision
 * u_p (Alg. 1 computes the sketch in u_p).  Column j is multiplied by
 * 2^e_j so that max_i |a_ij| * 2^e_j lies in [2^(t-1), 2^t) with t = 8 for
 * FP8-e4m3, 15 for FP16, 0 for BF16 and FP32; FP64 is not scaled.
 * ---------------------------------------------------------------------- */
static int scale_target(int prec)
{
    switch (prec) { case O_FP8: return 8; case O_FP16: return 15; default: return 0; }
}

void lsqo_colexp(const double* A, int64_t m, int64_t n, int64_t lda, int prec, int32_t* colexp)
{
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) {
        double mx = 0.0;
        for (int64_t i = 0; i < m; ++i) { double v = fabs(A[IDX(i, j, lda)]); if (v > mx) mx = v; }
        int E = 0;
        frexp(mx, &E);
        colexp[j] = (prec == O_FP64 || mx == 0.0 || !isfinite(mx)) ? 0 : scale_target(prec) - E;
    }
}

/* Ahat = round_p(A * 2^E), m-by-n, ld m. */
void lsqo_quantize(const double* A, int64_t m, int64_t n, int64_t lda, int prec,
                   const int32_t* colexp, double* Ahat)
{
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i)
            Ahat[IDX(i, j, m)] = lsqo_round(ldexp(A[IDX(i, j, lda)], colexp[j]), prec);
}

/* ------------------------------------------------------------------------
 * Sketch A_s = Omega_hat * Ahat (Alg. 1, "Sketch A_s = Omega A" in u_p).
 * Products of two values in FP8/BF16/FP16 are exact in FP32; accumulation
 * is FP32 RNE in ascending column index j of Omega (FP64 when prec = FP64).
 * As is s-by-n, ld s, holding FP32-representable values unless FP64.
 * ---------------------------------------------------------------------- */
int lsqo_sketch(const double* A, int64_t m, int64_t n, int64_t lda, int kind, int64_t s,
                int zeta, uint64_t seed, int prec, double* As, int32_t* colexp)
{
    if (prec < O_FP8 || prec > O_FP64 || s <= 0 || m <= 0 || n <= 0) return -1;
    double* Ahat = (double*)malloc(sizeof(double) * (size_t)m * (size_t)n);
    if (!Ahat) return -3;
    lsqo_colexp(A, m, n, lda, prec, colexp);
    lsqo_quantize(A, m, n, lda, prec, colexp, Ahat);
    int rc = 0;
    if (kind == O_SPARSE_SIGN) {
        /* Column j of Omega adds sgn * Ahat[j, :] to the rows idx of A_s; every
         * entry of A_s is summed in ascending j (its rows within one column of
         * Omega are distinct).  The columns of A_s are independent. */
        int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)m * (size_t)zeta);
        int8_t* sgn = (int8_t*)malloc((size_t)m * (size_t)zeta);
        if (!idx || !sgn) { free(idx); free(sgn); free(Ahat); return -3; }
        rc = lsqo_sparse_sign_indices(seed, m, s, zeta, idx, sgn);
        if (!rc) {
#pragma omp parallel for schedule(static)
            for (int64_t c = 0; c < n; ++c) {
                if (prec == O_FP64) {
                    for (int64_t i = 0; i < s; ++i) As[IDX(i, c, s)] = 0.0;
                    for (int64_t j = 0; j < m; ++j)
                        for (int t = 0; t < zeta; ++t) {
                            size_t r = IDX(idx[(size_t)j * zeta + t], c, s);
                            As[r] += (double)sgn[(size_t)j * zeta + t] * Ahat[IDX(j, c, m)];
                        }
                } else {
                    float* acc = (float*)calloc((size_t)s, sizeof(float));
                    for (int64_t j = 0; j < m; ++j)
                        for (int t = 0; t < zeta; ++t) {
                            int32_t r = idx[(size_t)j * zeta + t];
                            float term = (float)((double)sgn[(size_t)j * zeta + t] * Ahat[IDX(j, c, m)]);
                            acc[r] = acc[r] + term;
                        }
                    for (int64_t i = 0; i < s; ++i) As[IDX(i, c, s)] = (double)acc[i];
                    free(acc);
                }
            }
        }
        free(idx); free(sgn);
    } else if (kind == O_GAUSSIAN) {
        /* Row i of A_s: Omega_hat[i, :] Ahat, each entry summed in ascending j. */
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < s; ++i) {
            double* om = (double*)malloc(sizeof(double) * (size_t)m);
            for (int64_t j = 0; j < m; ++j) om[j] = lsqo_round(lsqo_gaussian_entry(seed, i, j), prec);
            for (int64_t c = 0; c < n; ++c) {
                if (prec == O_FP64) {
                    double acc = 0.0;
                    for (int64_t j = 0; j < m; ++j) acc += om[j] * Ahat[IDX(j, c, m)];
                    As[IDX(i, c, s)] = acc;
                } else {
                    float acc = 0.0f;
                    for (int64_t j = 0; j < m; ++j) {
                        float prod = (float)om[j] * (float)Ahat[IDX(j, c, m)];
                        acc = acc + prod;
                    }
                    As[IDX(i, c, s)] = (double)acc;
                }
            }
            free(om);
        }
    } else if (kind == O_SRFT) {
        /* Column c of A_s: (F D Ahat[:, c])[rows], the transform in FP32
         * arithmetic (FP64 when prec = FP64) */
        int64_t mp = lsqo_srft_order(m);
        int64_t* rows = (int64_t*)malloc(sizeof(int64_t) * (size_t)s);
        int* sg = (int*)malloc(sizeof(int) * (size_t)m);
        for (int64_t t = 0; t < s; ++t) rows[t] = lsqo_srft_row(seed, t, mp);
        for (int64_t j = 0; j < m; ++j) sg[j] = lsqo_srft_sign(seed, j);
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t c = 0; c < n; ++c) {
            if (prec == O_FP64) {
                double* v = (double*)calloc((size_t)mp, sizeof(double));
                for (int64_t j = 0; j < m; ++j) v[j] = (double)sg[j] * Ahat[IDX(j, c, m)];
                lsqo_fwht(v, mp);
                for (int64_t t = 0; t < s; ++t) As[IDX(t, c, s)] = v[rows[t]];
                free(v);
            } else {
                float* v = (float*)calloc((size_t)mp, sizeof(float));
                for (int64_t j = 0; j < m; ++j) v[j] = (float)((double)sg[j] * Ahat[IDX(j, c, m)]);
                fwht32(v, mp);
                for (int64_t t = 0; t < s; ++t) As[IDX(t, c, s)] = (double)v[rows[t]];
                free(v);
            }
        }
        free(rows); free(sg);
    } else {
        rc = -1;
    }
    free(Ahat);
    return rc;
}

/* ------------------------------------------------------------------------
 * Householder vector (Golub & Van Loan, Matrix Computations, 4th ed.,
 * Alg. 5.1.1, with the sigma = 0, x1 < 0 case mapping x to |x1| e1): for x
 * of length len, returns beta and v with v[0] = 1 such that
 * (I - beta v v^T) x = ||x|| e1.  Two versions: FP64 and FP32 arithmetic.
 * ---------------------------------------------------------------------- */
static double house64(const double* x, int64_t len, double* v, double* mu_out)
{
    double sigma = 0.0;
    for (int64_t i = 1; i < len; ++i) sigma += x[i] * x[i];
    v[0] = 1.0;
    for (int64_t i = 1; i < len; ++i) v[i] = x[i];
    double x1 = x[0];
    if (sigma == 0.0) {
        *mu_out = fabs(x1);
        return x1 >= 0.0 ? 0.0 : 2.0;
    }
    double mu = sqrt(x1 * x1 + sigma);
    double v1 = (x1 <= 0.0) ? x1 - mu : -sigma / (x1 + mu);
    double beta = 2.0 * v1 * v1 / (sigma + v1 * v1);
    for (int64_t i = 1; i < len; ++i) v[i] = v[i] / v1;
    *mu_out = mu;
    return beta;
}

static float house32(const float* x, int64_t len, float* v, float* mu_out)
{
    float sigma = 0.0f;
    for (int64_t i = 1; i < len; ++i) sigma = sigma + x[i] * x[i];
    v[0] = 1.0f;
    for (int64_t i = 1; i < len; ++i) v[i] = x[i];
    float x1 = x[0];
    if (sigma == 0.0f) {
        *mu_out = fabsf(x1);
        return x1 >= 0.0f ? 0.0f : 2.0f;
    }
    float mu = sqrtf(x1 * x1 + sigma);
    float v1 = (x1 <= 0.0f) ? x1 - mu : -sigma / (x1 + mu);
    float beta = 2.0f * v1 * v1 / (sigma + v1 * v1);
    for (int64_t i = 1; i < len; ++i) v[i] = v[i] / v1;
    *mu_out = mu;
    return beta;
}

/* Thin QR of the sketch, R only (Alg. 1, "Thin QR factorization A_s =
 * Q_s R_s"), by unblocked Householder QR (Golub & Van Loan Alg. 5.2.1) in
 * FP32 (prec = FP32) or FP64 arithmetic.  The reflector of column k maps it
 * to (||x||, 0, ...), so diag(R) >= 0.  R is n-by-n upper, ld n, zero below
 * the diagonal.  Returns 0, or -1 on bad arguments. */
int lsqo_qr_r(const double* As, int64_t s, int64_t n, int64_t ldas, int prec, double* R)
{
    if (s < n || n <= 0) return -1;
    if (prec == O_FP64) {
        double* W = (double*)malloc(sizeof(double) * (size_t)s * (size_t)n);
        double* v = (double*)malloc(sizeof(double) * (size_t)s);
        for (int64_t j = 0; j < n; ++j)
            for (int64_t i = 0; i < s; ++i) W[IDX(i, j, s)] = As[IDX(i, j, ldas)];
        for (int64_t k = 0; k < n; ++k) {
            double mu;
            double beta = house64(&W[IDX(k, k, s)], s - k, v, &mu);
            W[IDX(k, k, s)] = mu;
            for (int64_t i = k + 1; i < s; ++i) W[IDX(i, k, s)] = 0.0;
#pragma omp parallel for schedule(static)
            for (int64_t c = k + 1; c < n; ++c) {
                double w = 0.0;
                for (int64_t i = k; i < s; ++i) w += v[i - k] * W[IDX(i, c, s)];
                double t = beta * w;
                for (int64_t i = k; i < s; ++i) W[IDX(i, c, s)] = W[IDX(i, c, s)] - t * v[i - k];
            }
        }
        for (int64_t j = 0; j < n; ++j)
            for (int64_t i = 0; i < n; ++i) R[IDX(i, j, n)] = (i <= j) ? W[IDX(i, j, s)] : 0.0;
        free(W); free(v);
    } else {
        float* W = (float*)malloc(sizeof(float) * (size_t)s * (size_t)n);
        float* v = (float*)malloc(sizeof(float) * (size_t)s);
        for (int64_t j = 0; j < n; ++j)
            for (int64_t i = 0; i < s; ++i) W[IDX(i, j, s)] = (float)As[IDX(i, j, ldas)];
        for (int64_t k = 0; k < n; ++k) {
            float mu;
            float beta = house32(&W[IDX(k, k, s)], s - k, v, &mu);
            W[IDX(k, k, s)] = mu;
            for (int64_t i = k + 1; i < s; ++i) W[IDX(i, k, s)] = 0.0f;
#pragma omp parallel for schedule(static)
            for (int64_t c = k + 1; c < n; ++c) {
                float w = 0.0f;
                for (int64_t i = k; i < s; ++i) w = w + v[i - k] * W[IDX(i, c, s)];
                float t = beta * w;
                for (int64_t i = k; i < s; ++i) W[IDX(i, c, s)] = W[IDX(i, c, s)] - t * v[i - k];
            }
        }
        for (int64_t j = 0; j < n; ++j)
            for (int64_t i = 0; i < n; ++i) R[IDX(i, j, n)] = (i <= j) ? (double)W[IDX(i, j, s)] : 0.0;
        free(W); free(v);
    }
    return 0;
}

/* R_s = R_tilde * 2^(-E): undo the column scaling of the sketch exactly,
 * after promotion to FP64 (Alg. 1, "Promote R_s to double precision"). */
void lsqo_unscale_r(double* R, int64_t n, int64_t ldr, const int32_t* colexp)
{
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i <= j; ++i) R[IDX(i, j, ldr)] = ldexp(R[IDX(i, j, ldr)], -colexp[j]);
}

/* ------------------------------------------------------------------------
 * FP64 steps of Alg. 1.
 * ---------------------------------------------------------------------- */

/* A_p = A R^{-1} (Alg. 1, "Solve A_p = A R_s^{-1}"): for every row a of A,
 * solve y R = a by forward substitution over the columns of R. */
int lsqo_trsm_right_upper(const double* A, int64_t m, int64_t n, int64_t lda,
                          const double* R, int64_t ldr, double* Ap /* ld m */)
{
#pragma omp parallel
    {
        double* y = (double*)malloc(sizeof(double) * (size_t)n);
#pragma omp for schedule(static)
        for (int64_t i = 0; i < m; ++i) {
            for (int64_t j = 0; j < n; ++j) {
                double t = A[IDX(i, j, lda)];
                for (int64_t k = 0; k < j; ++k) t = t - y[k] * R[IDX(k, j, ldr)];
                y[j] = t / R[IDX(j, j, ldr)];
            }
            for (int64_t j = 0; j < n; ++j) Ap[IDX(i, j, m)] = y[j];
        }
        free(y);
    }
    return 0;
}

/* C = X^T Y (n-by-n) and c = X^T b, dot products over the m rows in index
 * order.  PNE: X = Y = A_p (Eq. e_pne).  HPNE: X = A_p, Y = A (Eq. e_hpne). */
void lsqo_gram(const double* X, const double* Y, int64_t m, int64_t n, int64_t ldx, int64_t ldy,
               const double* b, double* C /* ld n */, double* c)
{
#pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (int64_t q = 0; q < n; ++q)
        for (int64_t p = 0; p < n; ++p) {
            double acc = 0.0;
            for (int64_t i = 0; i < m; ++i) acc += X[IDX(i, p, ldx)] * Y[IDX(i, q, ldy)];
            C[IDX(p, q, n)] = acc;
        }
    if (b && c)
#pragma omp parallel for schedule(static)
        for (int64_t p = 0; p < n; ++p) {
            double acc = 0.0;
            for (int64_t i = 0; i < m; ++i) acc += X[IDX(i, p, ldx)] * b[i];
            c[p] = acc;
        }
}

/* Cholesky G = L L^T (Golub & Van Loan Alg. 4.2.1, column form), lower
 * triangle of G overwritten by L, strict upper zeroed.  Returns 0, or k > 0
 * when the k-th pivot (1-based) is not positive or not finite. */
int lsqo_cholesky(double* G, int64_t n, int64_t ld)
{
    for (int64_t j = 0; j < n; ++j) {
        double d = G[IDX(j, j, ld)];
        for (int64_t k = 0; k < j; ++k) d = d - G[IDX(j, k, ld)] * G[IDX(j, k, ld)];
        if (!(d > 0.0) || !isfinite(d)) return (int)(j + 1);
        double ljj = sqrt(d);
        G[IDX(j, j, ld)] = ljj;
#pragma omp parallel for schedule(static)
        for (int64_t i = j + 1; i < n; ++i) {
            double t = G[IDX(i, j, ld)];
            for (int64_t k = 0; k < j; ++k) t = t - G[IDX(i, k, ld)] * G[IDX(j, k, ld)];
            G[IDX(i, j, ld)] = t / ljj;
        }
    }
    for (int64_t j = 1; j < n; ++j)
        for (int64_t i = 0; i < j; ++i) G[IDX(i, j, ld)] = 0.0;
    return 0;
}

/* LU with partial pivoting, P H = L U (Golub & Van Loan Alg. 3.4.1): at
 * step k the pivot is the FIRST row i >= k of largest |h_ik|; rows are
 * swapped in full.  piv[k] = the row swapped with k.  Unit lower L below
 * the diagonal, U on and above.  Returns 0 or k > 0 for a zero pivot. */
int lsqo_lu(double* H, int64_t n, int64_t ld, int32_t* piv)
{
    int info = 0;
    for (int64_t k = 0; k < n; ++k) {
        int64_t p = k;
        double best = fabs(H[IDX(k, k, ld)]);
        for (int64_t i = k + 1; i < n; ++i) {
            double v = fabs(H[IDX(i, k, ld)]);
            if (v > best) { best = v; p = i; }
        }
        piv[k] = (int32_t)p;
        if (p != k)
            for (int64_t j = 0; j < n; ++j) {
                double t = H[IDX(k, j, ld)]; H[IDX(k, j, ld)] = H[IDX(p, j, ld)]; H[IDX(p, j, ld)] = t;
            }
        double d = H[IDX(k, k, ld)];
        if (d == 0.0 || !isfinite(d)) { if (!info) info = (int)(k + 1); continue; }
        for (int64_t i = k + 1; i < n; ++i) H[IDX(i, k, ld)] = H[IDX(i, k, ld)] / d;
#pragma omp parallel for schedule(static)
        for (int64_t j = k + 1; j < n; ++j)
            for (int64_t i = k + 1; i < n; ++i)
                H[IDX(i, j, ld)] = H[IDX(i, j, ld)] - H[IDX(i, k, ld)] * H[IDX(k, j, ld)];
    }
    return info;
}

/* Triangular solves on a vector, in place.
 * lower: L y = c (forward), unit diagonal if unit != 0.
 * lower_t: L^T y = c (backward).
 * upper: U y = c (backward). */
void lsqo_solve_lower(const double* L, int64_t n, int64_t ld, int unit, double* y)
{
    for (int64_t i = 0; i < n; ++i) {
        double t = y[i];
        for (int64_t k = 0; k < i; ++k) t = t - L[IDX(i, k, ld)] * y[k];
        y[i] = unit ? t : t / L[IDX(i, i, ld)];
    }
}

void lsqo_solve_lower_t(const double* L, int64_t n, int64_t ld, double* y)
{
    for (int64_t i = n - 1; i >= 0; --i) {
        double t = y[i];
        for (int64_t k = i + 1; k < n; ++k) t = t - L[IDX(k, i, ld)] * y[k];
        y[i] = t / L[IDX(i, i, ld)];
    }
}

void lsqo_solve_upper(const double* U, int64_t n, int64_t ld, double* y)
{
    for (int64_t i = n - 1; i >= 0; --i) {
        double t = y[i];
        for (int64_t k = i + 1; k < n; ++k) t = t - U[IDX(i, k, ld)] * y[k];
        y[i] = t / U[IDX(i, i, ld)];
    }
}

/* P H x = L U x = P c: apply the row swaps to c, then the two solves. */
void lsqo_lu_solve(const double* LU, int64_t n, int64_t ld, const int32_t* piv, double* y)
{
    for (int64_t k = 0; k < n; ++k) {
        int64_t p = piv[k];
        if (p != k) { double t = y[k]; y[k] = y[p]; y[p] = t; }
    }
    lsqo_solve_lower(LU, n, ld, 1, y);
    lsqo_solve_upper(LU, n, ld, y);
}

/* ------------------------------------------------------------------------
 * Reference least-squares solution (not the method): Householder QR of A in
 * FP64 (Golub & Van Loan Alg. 5.2.1 / Sec. 5.3.3), Q^T b by applying the
 * reflectors, then R x = (Q^T b)(1:n).  Returns 0 or -1.
 * ---------------------------------------------------------------------- */
int lsqo_lstsq_qr(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, double* x)
{
    if (m < n || n <= 0) return -1;
    double* W = (double*)malloc(sizeof(double) * (size_t)m * (size_t)n);
    double* v = (double*)malloc(sizeof(double) * (size_t)m);
    double* qb = (double*)malloc(sizeof(double) * (size_t)m);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i) W[IDX(i, j, m)] = A[IDX(i, j, lda)];
    for (int64_t i = 0; i < m; ++i) qb[i] = b[i];
    for (int64_t k = 0; k < n; ++k) {
        double mu;
        double beta = house64(&W[IDX(k, k, m)], m - k, v, &mu);
        W[IDX(k, k, m)] = mu;
        for (int64_t i = k + 1; i < m; ++i) W[IDX(i, k, m)] = 0.0;
#pragma omp parallel for schedule(static)
        for (int64_t c = k + 1; c < n; ++c) {
            double w = 0.0;
            for (int64_t i = k; i < m; ++i) w += v[i - k] * W[IDX(i, c, m)];
            double t = beta * w;
            for (int64_t i = k; i < m; ++i) W[IDX(i, c, m)] = W[IDX(i, c, m)] - t * v[i - k];
        }
        double w = 0.0;
        for (int64_t i = k; i < m; ++i) w += v[i - k] * qb[i];
        double t = beta * w;
        for (int64_t i = k; i < m; ++i) qb[i] = qb[i] - t * v[i - k];
    }
    for (int64_t i = 0; i < n; ++i) x[i] = qb[i];
    lsqo_solve_upper(W, n, m, x);
    free(W); free(v); free(qb);
    return 0;
}

/* ------------------------------------------------------------------------
 * Low-precision condition estimate (Sec. 6.1 and Alg. 1, first line).
 * In FP32: G = fl32(A^T A) with each product rounded then summed in row
 * order; ||G||_1; Cholesky of G; and Hager's 1-norm estimate of
 * ||G^{-1}||_1 (Hager 1984, with Higham's 1988 stopping test and
 * alternating-sign extra vector), at most 5 iterations, each application of
 * G^{-1} by the two Cholesky solves.  Then, in FP64 from those FP32 values,
 * kappa0 = 0.5 * log10(n * ||G||_1 * gamma), because
 * kappa(A)^2 = kappa(A^T A) <= n ||A^T A||_1 ||(A^T A)^{-1}||_1.
 * A Cholesky breakdown or a non-finite value is the "overflow" case and
 * returns kappa0 = +inf.  The precision table (reading of Sec. 6.1 extended
 * to the two 8-bit-class formats):
 *   kappa0 < 2 FP8, < 3 BF16, < 4 FP16, <= 8 FP32, otherwise FP64.
 * ---------------------------------------------------------------------- */
static int chol32(float* G, int64_t n)
{
    for (int64_t j = 0; j < n; ++j) {
        float d = G[IDX(j, j, n)];
        for (int64_t k = 0; k < j; ++k) d = d - G[IDX(j, k, n)] * G[IDX(j, k, n)];
        if (!(d > 0.0f) || !isfinite(d)) return (int)(j + 1);
        float ljj = sqrtf(d);
        G[IDX(j, j, n)] = ljj;
#pragma omp parallel for schedule(static)
        for (int64_t i = j + 1; i < n; ++i) {
            float t = G[IDX(i, j, n)];
            for (int64_t k = 0; k < j; ++k) t = t - G[IDX(i, k, n)] * G[IDX(j, k, n)];
            G[IDX(i, j, n)] = t / ljj;
        }
    }
    return 0;
}

/* y <- G^{-1} y with G = L L^T, L lower in the FP32 array. */
static void chol32_solve(const float* L, int64_t n, float* y)
{
    for (int64_t i = 0; i < n; ++i) {
        float t = y[i];
        for (int64_t k = 0; k < i; ++k) t = t - L[IDX(i, k, n)] * y[k];
        y[i] = t / L[IDX(i, i, n)];
    }
    for (int64_t i = n - 1; i >= 0; --i) {
        float t = y[i];
        for (int64_t k = i + 1; k < n; ++k) t = t - L[IDX(k, i, n)] * y[k];
        y[i] = t / L[IDX(i, i, n)];
    }
}

static float norm1_32(const float* y, int64_t n)
{
    float s = 0.0f;
    for (int64_t i = 0; i < n; ++i) s = s + fabsf(y[i]);
    return s;
}

int lsqo_precision_from_kappa0(double kappa0)
{
    if (!(kappa0 == kappa0) || isinf(kappa0)) return O_FP64;
    if (kappa0 < 2.0) return O_FP8;
    if (kappa0 < 3.0) return O_BF16;
    if (kappa0 < 4.0) return O_FP16;
    if (kappa0 <= 8.0) return O_FP32;
    return O_FP64;
}

/* Hager/Higham estimate of ||G^{-1}||_1 using the FP32 Cholesky factor L.
 * G^{-1} is symmetric, so the transpose products reuse the same solve. */
static float hager_inv_norm1(const float* L, int64_t n, int maxit)
{
    float* x = (float*)malloc(sizeof(float) * (size_t)n);
    float* y = (float*)malloc(sizeof(float) * (size_t)n);
    float* xi = (float*)malloc(sizeof(float) * (size_t)n);
    float* z = (float*)malloc(sizeof(float) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) x[i] = 1.0f / (float)n;
    for (int64_t i = 0; i < n; ++i) y[i] = x[i];
    chol32_solve(L, n, y);
    float est = norm1_32(y, n);
    for (int64_t i = 0; i < n; ++i) xi[i] = (y[i] >= 0.0f) ? 1.0f : -1.0f;
    for (int64_t i = 0; i < n; ++i) z[i] = xi[i];
    chol32_solve(L, n, z);
    int64_t jlast = -1;
    for (int it = 1; it < maxit; ++it) {
        /* j = first index of max |z_i|; stop when ||z||_inf <= z^T x. */
        int64_t j = 0;
        float zmax = fabsf(z[0]);
        for (int64_t i = 1; i < n; ++i) if (fabsf(z[i]) > zmax) { zmax = fabsf(z[i]); j = i; }
        float ztx = 0.0f;
        for (int64_t i = 0; i < n; ++i) ztx = ztx + z[i] * x[i];
        if (zmax <= ztx || j == jlast) break;
        jlast = j;
        for (int64_t i = 0; i < n; ++i) x[i] = 0.0f;
        x[j] = 1.0f;
        for (int64_t i = 0; i < n; ++i) y[i] = x[i];
        chol32_solve(L, n, y);
        float est_new = norm1_32(y, n);
        int same = 1;
        for (int64_t i = 0; i < n; ++i) same &= (((y[i] >= 0.0f) ? 1.0f : -1.0f) == xi[i]);
        if (same || est_new <= est) { if (est_new > est) est = est_new; break; }
        est = est_new;
        for (int64_t i = 0; i < n; ++i) xi[i] = (y[i] >= 0.0f) ? 1.0f : -1.0f;
        for (int64_t i = 0; i < n; ++i) z[i] = xi[i];
        chol32_solve(L, n, z);
    }
    /* Higham's extra vector x_i = (-1)^i (1 + i/(n-1)), estimate 2||y||_1/(3n). */
    for (int64_t i = 0; i < n; ++i) {
        float mag = (n > 1) ? 1.0f + (float)i / (float)(n - 1) : 1.0f;
        y[i] = (i % 2 == 0) ? mag : -mag;
    }
    chol32_solve(L, n, y);
    float alt = 2.0f * norm1_32(y, n) / (3.0f * (float)n);
    if (alt > est) est = alt;
    free(x); free(y); free(xi); free(z);
    return est;
}

int lsqo_condest(const double* A, int64_t m, int64_t n, int64_t lda,
                 double* kappa0, int32_t* chosen, double* norm1_out, double* gamma_out)
{
    float* G = (float*)malloc(sizeof(float) * (size_t)n * (size_t)n);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < n; ++q)
        for (int64_t p = q; p < n; ++p) {
            float acc = 0.0f;
            for (int64_t i = 0; i < m; ++i) {
                float prod = (float)A[IDX(i, p, lda)] * (float)A[IDX(i, q, lda)];
                acc = acc + prod;
            }
            G[IDX(p, q, n)] = acc;
            G[IDX(q, p, n)] = acc;
        }
    float nrm = 0.0f;
    for (int64_t q = 0; q < n; ++q) {
        float cs = 0.0f;
        for (int64_t p = 0; p < n; ++p) cs = cs + fabsf(G[IDX(p, q, n)]);
        if (cs > nrm) nrm = cs;
    }
    double k0;
    float gam = 0.0f;
    int info = chol32(G, n);
    if (info != 0 || !isfinite(nrm)) {
        k0 = INFINITY;
    } else {
        gam = hager_inv_norm1(G, n, 5);
        double prod = (double)n * (double)nrm * (double)gam;
        k0 = (isfinite(prod) && prod > 0.0) ? 0.5 * log10(prod) : INFINITY;
    }
    if (kappa0) *kappa0 = k0;
    if (chosen) *chosen = lsqo_precision_from_kappa0(k0);
    if (norm1_out) *norm1_out = (double)nrm;
    if (gamma_out) *gamma_out = (double)gam;
    free(G);
    return info;
}

/* ------------------------------------------------------------------------
 * Condition estimate on the sketch (a reading of Alg. 1's first line,
 * "estimate kappa0 ~ log10 kappa(A) in single precision", that replaces the
 * m n^2 Gram A^T A of Sec. 6.1 by the Gram of a sketch):
 *   1. A_e = Omega_e A, an FP32 sparse-sign sketch (s_e = min(2n, m) rows,
 *      zeta = min(8, s_e), Philox stream keyed by `seed`), so that
 *      G_s = A_e^T A_e approximates A^T A on range(A) (Omega_e embeds it);
 *   2. R_e by Householder QR of A_e in FP32, unscaled to A's columns;
 *   3. the estimator of Sec. 6.1 on G_s = fl32(A_e^T A_e) (with the sketch's
 *      column scaling undone): ||G_s||_1, and Hager's estimate gamma of
 *      ||G_s^{-1}||_1 with G_s^{-1} applied through the triangular factor
 *      L = R_e^T from the QR (R_e^T R_e = G_s) instead of an FP32 Cholesky
 *      of G_s, which breaks down once kappa(A)^2 > 1/u32;
 *      kappa0 = 0.5 log10(n ||G_s||_1 gamma);
 *   4. an FP32 R_e resolves kappa(A) only while u32 kappa(R_e) < 1 (Lemma
 *      rscond for the FP32 factor itself): if Hager's estimate of
 *      kappa_1(R_e) = ||R_e||_1 ||R_e^{-1}||_1 gives u32 kappa_1 > 1, the
 *      estimate is the "overflow" case, kappa0 = +inf (FP64).
 * ---------------------------------------------------------------------- */
static void upper32_solve(const float* R, int64_t n, float* y)        /* R y = c */
{
    for (int64_t i = n - 1; i >= 0; --i) {
        float t = y[i];
        for (int64_t k = i + 1; k < n; ++k) t = t - R[IDX(i, k, n)] * y[k];
        y[i] = t / R[IDX(i, i, n)];
    }
}

static void upper32_solve_t(const float* R, int64_t n, float* y)      /* R^T y = c */
{
    for (int64_t i = 0; i < n; ++i) {
        float t = y[i];
        for (int64_t k = 0; k < i; ++k) t = t - R[IDX(k, i, n)] * y[k];
        y[i] = t / R[IDX(i, i, n)];
    }
}

/* Hager / Higham estimate of ||R^{-1}||_1 for upper triangular R (FP32):
 * products with R^{-1} and R^{-T} by substitution. */
static float hager_rinv_norm1(const float* R, int64_t n, int maxit)
{
    float* x = (float*)malloc(sizeof(float) * (size_t)n);
    float* y = (float*)malloc(sizeof(float) * (size_t)n);
    float* xi = (float*)malloc(sizeof(float) * (size_t)n);
    float* z = (float*)malloc(sizeof(float) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) x[i] = 1.0f / (float)n;
    for (int64_t i = 0; i < n; ++i) y[i] = x[i];
    upper32_solve(R, n, y);
    float est = norm1_32(y, n);
    for (int64_t i = 0; i < n; ++i) xi[i] = (y[i] >= 0.0f) ? 1.0f : -1.0f;
    for (int64_t i = 0; i < n; ++i) z[i] = xi[i];
    upper32_solve_t(R, n, z);
    int64_t jlast = -1;
    for (int it = 1; it < maxit; ++it) {
        int64_t j = 0;
        float zmax = fabsf(z[0]);
        for (int64_t i = 1; i < n; ++i) if (fabsf(z[i]) > zmax) { zmax = fabsf(z[i]); j = i; }
        float ztx = 0.0f;
        for (int64_t i = 0; i < n; ++i) ztx = ztx + z[i] * x[i];
        if (zmax <= ztx || j == jlast) break;
        jlast = j;
        for (int64_t i = 0; i < n; ++i) x[i] = 0.0f;
        x[j] = 1.0f;
        for (int64_t i = 0; i < n; ++i) y[i] = x[i];
        upper32_solve(R, n, y);
        float est_new = norm1_32(y, n);
        int same = 1;
        for (int64_t i = 0; i < n; ++i) same &= (((y[i] >= 0.0f) ? 1.0f : -1.0f) == xi[i]);
        if (same || est_new <= est) { if (est_new > est) est = est_new; break; }
        est = est_new;
        for (int64_t i = 0; i < n; ++i) xi[i] = (y[i] >= 0.0f) ? 1.0f : -1.0f;
        for (int64_t i = 0; i < n; ++i) z[i] = xi[i];
        upper32_solve_t(R, n, z);
    }
    for (int64_t i = 0; i < n; ++i) {
        float mag = (n > 1) ? 1.0f + (float)i / (float)(n - 1) : 1.0f;
        y[i] = (i % 2 == 0) ? mag : -mag;
    }
    upper32_solve(R, n, y);
    float alt = 2.0f * norm1_32(y, n) / (3.0f * (float)n);
    if (alt > est) est = alt;
    free(x); free(y); free(xi); free(z);
    return est;
}

/* kappa_1(R) = ||R||_1 * Hager's estimate of ||R^{-1}||_1, R n-by-n upper
 * (FP64 storage, ld) taken to FP32; +inf if not finite or not positive. */
double lsqo_kappa1_upper32(const double* R, int64_t n, int64_t ld)
{
    float* Rf = (float*)calloc((size_t)n * (size_t)n, sizeof(float));
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i <= j; ++i) Rf[IDX(i, j, n)] = (float)R[IDX(i, j, ld)];
    float rn = 0.0f;
    for (int64_t j = 0; j < n; ++j) {
        float cs = 0.0f;
        for (int64_t i = 0; i <= j; ++i) cs = cs + fabsf(Rf[IDX(i, j, n)]);
        if (cs > rn) rn = cs;
    }
    float inv = hager_rinv_norm1(Rf, n, 5);
    free(Rf);
    double k1 = (double)rn * (double)inv;
    return (isfinite(k1) && k1 > 0.0) ? k1 : INFINITY;
}

int lsqo_condest_sketch(const double* A, int64_t m, int64_t n, int64_t lda, uint64_t seed,
                        double* kappa0, int32_t* chosen, double* kappa1_out)
{
    int64_t se = 2 * n < m ? 2 * n : m;
    int zeta = se < 8 ? (int)se : 8;
    double* As = (double*)malloc(sizeof(double) * (size_t)se * (size_t)n);
    int32_t* ce = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    double* R = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
    float* G = (float*)malloc(sizeof(float) * (size_t)n * (size_t)n);
    float* L = (float*)calloc((size_t)n * (size_t)n, sizeof(float));
    int rc = lsqo_sketch(A, m, n, lda, O_SPARSE_SIGN, se, zeta, seed, O_FP32, As, ce);
    if (!rc) rc = lsqo_qr_r(As, se, n, se, O_FP32, R);
    double k1 = INFINITY, k0 = INFINITY;
    if (!rc) {
        lsqo_unscale_r(R, n, n, ce);
        k1 = lsqo_kappa1_upper32(R, n, n);
        /* G_s = fl32(A_e^T A_e) of the unscaled sketch, products rounded then
         * summed in row order (as for A^T A in lsqo_condest) */
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t q = 0; q < n; ++q)
            for (int64_t p = q; p < n; ++p) {
                float acc = 0.0f;
                for (int64_t i = 0; i < se; ++i) {
                    float prod = (float)ldexp(As[IDX(i, p, se)], -ce[p]) * (float)ldexp(As[IDX(i, q, se)], -ce[q]);
                    acc = acc + prod;
                }
                G[IDX(p, q, n)] = acc;
                G[IDX(q, p, n)] = acc;
            }
        float nrm = 0.0f;
        for (int64_t q = 0; q < n; ++q) {
            float cs = 0.0f;
            for (int64_t p = 0; p < n; ++p) cs = cs + fabsf(G[IDX(p, q, n)]);
            if (cs > nrm) nrm = cs;
        }
        for (int64_t j = 0; j < n; ++j)
            for (int64_t i = j; i < n; ++i) L[IDX(i, j, n)] = (float)R[IDX(j, i, n)];
        float gam = hager_inv_norm1(L, n, 5);
        double prod = (double)n * (double)nrm * (double)gam;
        if (isfinite(k1) && 0x1p-24 * k1 <= 1.0 && isfinite(prod) && prod > 0.0) k0 = 0.5 * log10(prod);
    }
    if (kappa0) *kappa0 = k0;
    if (chosen) *chosen = lsqo_precision_from_kappa0(k0);
    if (kappa1_out) *kappa1_out = k1;
    free(As); free(ce); free(R); free(G); free(L);
    return rc;
}

/* ------------------------------------------------------------------------
 * LU with partial pivoting of a tall s-by-n matrix (s >= n), Golub & Van
 * Loan Alg. 3.4.1 run over the n columns with the pivot searched over all s
 * rows (the FIRST row of largest magnitude): P A = L U with L s-by-n unit
 * lower trapezoidal and U n-by-n upper.  In FP64 or FP32 arithmetic; U is
 * returned in FP64 (n-by-n, ld n, zero below the diagonal).  Returns 0 or
 * k > 0 for a zero pivot at step k.
 * ---------------------------------------------------------------------- */
int lsqo_lu_tall_u(const double* As, int64_t s, int64_t n, int64_t ldas, int prec, double* U)
{
    if (s < n || n <= 0) return -1;
    int info = 0;
    if (prec == O_FP64) {
        double* W = (double*)malloc(sizeof(double) * (size_t)s * (size_t)n);
        for (int64_t j = 0; j < n; ++j)
            for (int64_t i = 0; i < s; ++i) W[IDX(i, j, s)] = As[IDX(i, j, ldas)];
        for (int64_t k = 0; k < n; ++k) {
            int64_t p = k;
            double best = fabs(W[IDX(k, k, s)]);
            for (int64_t i = k + 1; i < s; ++i)
                if (fabs(W[IDX(i, k, s)]) > best) { best = fabs(W[IDX(i, k, s)]); p = i; }
            if (p != k)
                for (int64_t j = 0; j < n; ++j) {
                    double t = W[IDX(k, j, s)]; W[IDX(k, j, s)] = W[IDX(p, j, s)]; W[IDX(p, j, s)] = t;
                }
            double d = W[IDX(k, k, s)];
            if (d == 0.0 || !isfinite(d)) { if (!info) info = (int)(k + 1); continue; }
            for (int64_t i = k + 1; i < s; ++i) W[IDX(i, k, s)] = W[IDX(i, k, s)] / d;
#pragma omp parallel for schedule(static)
            for (int64_t j = k + 1; j < n; ++j)
                for (int64_t i = k + 1; i < s; ++i)
                    W[IDX(i, j, s)] = W[IDX(i, j, s)] - W[IDX(i, k, s)] * W[IDX(k, j, s)];
        }
        for (int64_t j = 0; j < n; ++j)
            for (int64_t i = 0; i < n; ++i) U[IDX(i, j, n)] = (i <= j) ? W[IDX(i, j, s)] : 0.0;
        free(W);
    } else {
        float* W = (float*)malloc(sizeof(float) * (size_t)s * (size_t)n);
        for (int64_t j = 0; j < n; ++j)
            for (int64_t i = 0; i < s; ++i) W[IDX(i, j, s)] = (float)As[IDX(i, j, ldas)];
        for (int64_t k = 0; k < n; ++k) {
            int64_t p = k;
            float best = fabsf(W[IDX(k, k, s)]);
            for (int64_t i = k + 1; i < s; ++i)
                if (fabsf(W[IDX(i, k, s)]) > best) { best = fabsf(W[IDX(i, k, s)]); p = i; }
            if (p != k)
                for (int64_t j = 0; j < n; ++j) {
                    float t = W[IDX(k, j, s)]; W[IDX(k, j, s)] = W[IDX(p, j, s)]; W[IDX(p, j, s)] = t;
                }
            float d = W[IDX(k, k, s)];
            if (d == 0.0f || !isfinite(d)) { if (!info) info = (int)(k + 1); continue; }
            for (int64_t i = k + 1; i < s; ++i) W[IDX(i, k, s)] = W[IDX(i, k, s)] / d;
#pragma omp parallel for schedule(static)
            for (int64_t j = k + 1; j < n; ++j)
                for (int64_t i = k + 1; i < s; ++i)
                    W[IDX(i, j, s)] = W[IDX(i, j, s)] - W[IDX(i, k, s)] * W[IDX(k, j, s)];
        }
        for (int64_t j = 0; j < n; ++j)
            for (int64_t i = 0; i < n; ++i) U[IDX(i, j, n)] = (i <= j) ? (double)W[IDX(i, j, s)] : 0.0;
        free(W);
    }
    return info;
}

/* U^T y = c for upper U (forward substitution with the transpose). */
void lsqo_solve_upper_t(const double* U, int64_t n, int64_t ld, double* y)
{
    for (int64_t i = 0; i < n; ++i) {
        double t = y[i];
        for (int64_t k = 0; k < i; ++k) t = t - U[IDX(k, i, ld)] * y[k];
        y[i] = t / U[IDX(i, i, ld)];
    }
}

/* HPNE through a QR factorization of H = A_p^T A (Sec. 1 lists QR beside LU
 * for Eq. e_hpne): the Householder R of the (n+1)-by-(n+1) matrix
 * [[H, c], [0, 1]] holds R_H in its leading block and Q_H^T c in the top of
 * its last column (the reflectors of the first n columns leave the zero row
 * alone), so x = R_H^{-1} (Q_H^T c).  FP64. */
static int hpne_qr_solve(const double* H, int64_t n, const double* c, double* x)
{
    int64_t n1 = n + 1;
    double* M = (double*)calloc((size_t)n1 * (size_t)n1, sizeof(double));
    double* R = (double*)malloc(sizeof(double) * (size_t)n1 * (size_t)n1);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i) M[IDX(i, j, n1)] = H[IDX(i, j, n)];
    for (int64_t i = 0; i < n; ++i) M[IDX(i, n, n1)] = c[i];
    M[IDX(n, n, n1)] = 1.0;
    int rc = lsqo_qr_r(M, n1, n1, n1, O_FP64, R);
    int info = 0;
    for (int64_t i = 0; i < n && !rc; ++i)
        if (!(R[IDX(i, i, n1)] != 0.0) || !isfinite(R[IDX(i, i, n1)])) { info = (int)(i + 1); break; }
    if (!rc && !info) {
        for (int64_t i = 0; i < n; ++i) x[i] = R[IDX(i, n, n1)];
        lsqo_solve_upper(R, n, n1, x);
    }
    free(M); free(R);
    return rc ? -1 : info;
}

/* ------------------------------------------------------------------------
 * Alg. 1 end to end with one of the solution methods, a randomized
 * preconditioner computed in precision u_p, then optionally one FP64
 * residual-refinement step (not part of the paper's algorithm):
 *   method 0  PNE (Eq. e_pne):  A_p^T A_p y = A_p^T b (Cholesky), R_s x = y;
 *   method 1  HPNE (Eq. e_hpne): A_p^T A x = A_p^T b, LU with partial pivoting;
 *   method 2  HPNE with a QR factorization of A_p^T A (above);
 *   method 3  seminormal equations (Eq. e_sne) R^T R x = A^T b, with R the
 *             triangular factor of a thin QR of A obtained from the
 *             preconditioner: A_p = A R_s^{-1} = Q R_p with
 *             R_p^T R_p = A_p^T A_p (Cholesky, R_p = L^T), so A = Q (R_p R_s)
 *             and R = L^T R_s, applied in factored form:
 *             x = R_s^{-1} L^{-T} L^{-1} R_s^{-T} (A^T b);
 *   method 4  not-normal equations (Eq. e_nne) B^T A x = B^T b with
 *             B = A U_s^{-1}, U_s the upper factor of the LU with partial
 *             pivoting of the sketch A_s in u_p (so B has the column space of
 *             A and Omega B = P^T L_s is well conditioned), solved by LU with
 *             partial pivoting.
 * Refinement: r = b - A x, then the same method for the correction with the
 * factorizations reused (PNE, HPNE: A_p^T r; SNE: A^T r; NNE: B^T r; HPNE
 * through QR: a second QR with the new right-hand side), x = x + delta.
 * Returns 0, k > 0 for a factorization breakdown at pivot k, -1 for bad
 * arguments.  Rs_out (n-by-n, may be NULL) receives R_s (U_s for method 4);
 * kappa0_out and prec_out (may be NULL) the estimate and the precision used.
 * ---------------------------------------------------------------------- */
int lsqo_solve_method(const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
                      int method, int kind, int64_t s, int zeta, uint64_t seed,
                      int sketch_prec, int qr_prec, int refine_steps,
                      double* x, double* Rs_out, double* kappa0_out, int32_t* prec_out)
{
    if (m <= 0 || n <= 0 || s < n || m < s || method < 0 || method > 4) return -1;
    double k0 = NAN;
    int prec = sketch_prec;
    if (prec == O_AUTO) {
        int32_t ch;
        lsqo_condest(A, m, n, lda, &k0, &ch, NULL, NULL);
        prec = ch;
    } else if (prec == O_AUTO_SKETCH) {
        int32_t ch;
        lsqo_condest_sketch(A, m, n, lda, seed, &k0, &ch, NULL);
        prec = ch;
    }
    if (prec < O_FP8 || prec > O_FP64) return -1;
    int qp = (prec == O_FP64) ? O_FP64 : qr_prec;
    if (qp != O_FP32 && qp != O_FP64) qp = O_FP32;
    if (kappa0_out) *kappa0_out = k0;
    if (prec_out) *prec_out = prec;
    int hp = (method == 1 || method == 2 || method == 4);  /* nonsymmetric n-by-n system */

    size_t mn = (size_t)m * (size_t)n, nn = (size_t)n * (size_t)n;
    double* As = (double*)malloc(sizeof(double) * (size_t)s * (size_t)n);
    int32_t* ce = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    double* R = (double*)malloc(sizeof(double) * nn);
    double* Ap = (double*)malloc(sizeof(double) * mn);
    double* G = (double*)malloc(sizeof(double) * nn);
    double* c = (double*)malloc(sizeof(double) * (size_t)n);
    double* r = (double*)malloc(sizeof(double) * (size_t)m);
    int32_t* piv = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int rc = lsqo_sketch(A, m, n, lda, kind, s, zeta, seed, prec, As, ce);
    int info = 0;
    if (!rc) {
        if (method == 4) info = lsqo_lu_tall_u(As, s, n, s, qp, R);
        else rc = lsqo_qr_r(As, s, n, s, qp, R);
    }
    if (!rc && !info) {
        lsqo_unscale_r(R, n, n, ce);
        if (Rs_out) memcpy(Rs_out, R, sizeof(double) * nn);
        lsqo_trsm_right_upper(A, m, n, lda, R, n, Ap);
        if (hp) lsqo_gram(Ap, A, m, n, m, lda, b, G, c);
        else    lsqo_gram(Ap, Ap, m, n, m, m, b, G, c);
        if (method == 3) {
            /* c = A^T b, then R_s^{-T} c */
#pragma omp parallel for schedule(static)
            for (int64_t p = 0; p < n; ++p) {
                double acc = 0.0;
                for (int64_t i = 0; i < m; ++i) acc += A[IDX(i, p, lda)] * b[i];
                c[p] = acc;
            }
            lsqo_solve_upper_t(R, n, n, c);
        }
        if (method == 1 || method == 4) info = lsqo_lu(G, n, n, piv);
        else if (method != 2) info = lsqo_cholesky(G, n, n);
        if (!info) {
            for (int64_t i = 0; i < n; ++i) x[i] = c[i];
            if (method == 1 || method == 4) {
                lsqo_lu_solve(G, n, n, piv, x);
            } else if (method == 2) {
                info = hpne_qr_solve(G, n, c, x);
            } else {
                lsqo_solve_lower(G, n, n, 0, x);
                lsqo_solve_lower_t(G, n, n, x);
                lsqo_solve_upper(R, n, n, x);
            }
            for (int step = 0; step < refine_steps && !info; ++step) {
#pragma omp parallel for schedule(static)
                for (int64_t i = 0; i < m; ++i) {
                    double t = b[i];
                    for (int64_t j = 0; j < n; ++j) t = t - A[IDX(i, j, lda)] * x[j];
                    r[i] = t;
                }
                const double* X = (method == 3) ? A : Ap;
                int64_t ldX = (method == 3) ? lda : m;
#pragma omp parallel for schedule(static)
                for (int64_t p = 0; p < n; ++p) {
                    double acc = 0.0;
                    for (int64_t i = 0; i < m; ++i) acc += X[IDX(i, p, ldX)] * r[i];
                    c[p] = acc;
                }
                if (method == 1 || method == 4) {
                    lsqo_lu_solve(G, n, n, piv, c);
                } else if (method == 2) {
                    double* d = (double*)malloc(sizeof(double) * (size_t)n);
                    info = hpne_qr_solve(G, n, c, d);
                    memcpy(c, d, sizeof(double) * (size_t)n);
                    free(d);
                } else {
                    if (method == 3) lsqo_solve_upper_t(R, n, n, c);
                    lsqo_solve_lower(G, n, n, 0, c);
                    lsqo_solve_lower_t(G, n, n, c);
                    lsqo_solve_upper(R, n, n, c);
                }
                for (int64_t j = 0; j < n; ++j) x[j] = x[j] + c[j];
            }
        }
    }
    free(As); free(ce); free(R); free(Ap); free(G); free(c); free(r); free(piv);
    return rc ? -1 : info;
}

/* PNE (hpne = 0) or HPNE with LU (hpne = 1): lsqo_solve_method 0 or 1. */
int lsqo_solve(const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
               int hpne, int kind, int64_t s, int zeta, uint64_t seed,
               int sketch_prec, int qr_prec, int refine_steps,
               double* x, double* Rs_out, double* kappa0_out, int32_t* prec_out)
{
    return lsqo_solve_method(A, m, n, lda, b, hpne ? 1 : 0, kind, s, zeta, seed, sketch_prec, qr_prec,
                             refine_steps, x, Rs_out, kappa0_out, prec_out);
}

/* ------------------------------------------------------------------------
 * Learned precision proposal (not in the paper): a multilayer perceptron
 * d -> 64 -> 64 -> 64 -> 4 with ReLU hidden layers and a softmax
 * cross-entropy loss, in FP64.  Parameters are packed layer by layer as
 * W_l (out x in, row-major) followed by b_l (out).
 * ---------------------------------------------------------------------- */
#define MLP_H 64
#define MLP_C 4

int64_t lsqo_mlp_param_count(int d)
{
    return (int64_t)MLP_H * d + MLP_H + 2 * ((int64_t)MLP_H * MLP_H + MLP_H) + (int64_t)MLP_C * MLP_H + MLP_C;
}

static void mlp_layer(const double* W, const double* b, int out, int in, const double* x, double* z)
{
    for (int o = 0; o < out; ++o) {
        double acc = b[o];
        for (int i = 0; i < in; ++i) acc += W[(int64_t)o * in + i] * x[i];
        z[o] = acc;
    }
}

/* Forward pass for `batch` rows of X (batch x d, row-major) -> logits
 * (batch x 4).  Returns the mean cross-entropy if labels != NULL. */
double lsqo_mlp_forward(const double* params, int d, int batch, const double* X, const int32_t* labels,
                        double* logits)
{
    const double* W1 = params;
    const double* b1 = W1 + MLP_H * d;
    const double* W2 = b1 + MLP_H;
    const double* b2 = W2 + MLP_H * MLP_H;
    const double* W3 = b2 + MLP_H;
    const double* b3 = W3 + MLP_H * MLP_H;
    const double* W4 = b3 + MLP_H;
    const double* b4 = W4 + MLP_C * MLP_H;
    double h1[MLP_H], h2[MLP_H], h3[MLP_H], z[MLP_C];
    double loss = 0.0;
    for (int s = 0; s < batch; ++s) {
        mlp_layer(W1, b1, MLP_H, d, X + (int64_t)s * d, h1);
        for (int o = 0; o < MLP_H; ++o) h1[o] = h1[o] > 0.0 ? h1[o] : 0.0;
        mlp_layer(W2, b2, MLP_H, MLP_H, h1, h2);
        for (int o = 0; o < MLP_H; ++o) h2[o] = h2[o] > 0.0 ? h2[o] : 0.0;
        mlp_layer(W3, b3, MLP_H, MLP_H, h2, h3);
        for (int o = 0; o < MLP_H; ++o) h3[o] = h3[o] > 0.0 ? h3[o] : 0.0;
        mlp_layer(W4, b4, MLP_C, MLP_H, h3, z);
        if (logits)
            for (int c = 0; c < MLP_C; ++c) logits[(int64_t)s * MLP_C + c] = z[c];
        if (labels) {
            double mx = z[0];
            for (int c = 1; c < MLP_C; ++c) if (z[c] > mx) mx = z[c];
            double se = 0.0;
            for (int c = 0; c < MLP_C; ++c) se += exp(z[c] - mx);
            loss += -(z[labels[s]] - mx - log(se));
        }
    }
    return labels ? loss / batch : 0.0;
}

/* Gradient of the mean cross-entropy with respect to every parameter
 * (same packing), by backpropagation.  Returns the loss. */
double lsqo_mlp_backward(const double* params, int d, int batch, const double* X, const int32_t* labels,
                         double* grad)
{
    const double* W1 = params;
    const double* b1 = W1 + MLP_H * d;
    const double* W2 = b1 + MLP_H;
    const double* b2 = W2 + MLP_H * MLP_H;
    const double* W3 = b2 + MLP_H;
    const double* b3 = W3 + MLP_H * MLP_H;
    const double* W4 = b3 + MLP_H;
    const double* b4 = W4 + MLP_C * MLP_H;
    double* gW1 = grad;
    double* gb1 = gW1 + MLP_H * d;
    double* gW2 = gb1 + MLP_H;
    double* gb2 = gW2 + MLP_H * MLP_H;
    double* gW3 = gb2 + MLP_H;
    double* gb3 = gW3 + MLP_H * MLP_H;
    double* gW4 = gb3 + MLP_H;
    double* gb4 = gW4 + MLP_C * MLP_H;
    int64_t np = lsqo_mlp_param_count(d);
    for (int64_t q = 0; q < np; ++q) grad[q] = 0.0;
    double z1[MLP_H], z2[MLP_H], z3[MLP_H], h1[MLP_H], h2[MLP_H], h3[MLP_H], z[MLP_C];
    double d4[MLP_C], d3[MLP_H], d2[MLP_H], d1[MLP_H];
    double loss = 0.0;
    for (int s = 0; s < batch; ++s) {
        const double* x = X + (int64_t)s * d;
        mlp_layer(W1, b1, MLP_H, d, x, z1);
        for (int o = 0; o < MLP_H; ++o) h1[o] = z1[o] > 0.0 ? z1[o] : 0.0;
        mlp_layer(W2, b2, MLP_H, MLP_H, h1, z2);
        for (int o = 0; o < MLP_H; ++o) h2[o] = z2[o] > 0.0 ? z2[o] : 0.0;
        mlp_layer(W3, b3, MLP_H, MLP_H, h2, z3);
        for (int o = 0; o < MLP_H; ++o) h3[o] = z3[o] > 0.0 ? z3[o] : 0.0;
        mlp_layer(W4, b4, MLP_C, MLP_H, h3, z);
        double mx = z[0];
        for (int c = 1; c < MLP_C; ++c) if (z[c] > mx) mx = z[c];
        double se = 0.0;
        for (int c = 0; c < MLP_C; ++c) se += exp(z[c] - mx);
        loss += -(z[labels[s]] - mx - log(se));
        for (int c = 0; c < MLP_C; ++c) d4[c] = (exp(z[c] - mx) / se - (c == labels[s] ? 1.0 : 0.0)) / batch;
        for (int i = 0; i < MLP_H; ++i) {
            double t = 0.0;
            for (int c = 0; c < MLP_C; ++c) t += W4[(int64_t)c * MLP_H + i] * d4[c];
            d3[i] = z3[i] > 0.0 ? t : 0.0;
        }
        for (int i = 0; i < MLP_H; ++i) {
            double t = 0.0;
            for (int o = 0; o < MLP_H; ++o) t += W3[(int64_t)o * MLP_H + i] * d3[o];
            d2[i] = z2[i] > 0.0 ? t : 0.0;
        }
        for (int i = 0; i < MLP_H; ++i) {
            double t = 0.0;
            for (int o = 0; o < MLP_H; ++o) t += W2[(int64_t)o * MLP_H + i] * d2[o];
            d1[i] = z1[i] > 0.0 ? t : 0.0;
        }
        for (int c = 0; c < MLP_C; ++c) {
            gb4[c] += d4[c];
            for (int i = 0; i < MLP_H; ++i) gW4[(int64_t)c * MLP_H + i] += d4[c] * h3[i];
        }
        for (int o = 0; o < MLP_H; ++o) {
            gb3[o] += d3[o];
            gb2[o] += d2[o];
            gb1[o] += d1[o];
            for (int i = 0; i < MLP_H; ++i) {
                gW3[(int64_t)o * MLP_H + i] += d3[o] * h2[i];
                gW2[(int64_t)o * MLP_H + i] += d2[o] * h1[i];
            }
            for (int i = 0; i < d; ++i) gW1[(int64_t)o * d + i] += d1[o] * x[i];
        }
    }
    return loss / batch;
}

/* Features of A for the precision proposal, in FP64 (feature k):
 *  0 log2(m) / 16, 1 log2(n) / 10,
 *  2 log10(max/min column 2-norm), 3 std of log10 column norms,
 *  4 log10(max/min |diag R|), 5 std of log10 |diag R|,
 *  6 least-squares slope of log10 |diag R_j| against j / n,
 *  7 log10(max/min |diag R|) over the last quarter of the columns,
 *  8 fraction of columns with |diag R_j| < 1e-2 max |diag R|,
 *  9 log10(min |diag R| / (||A||_F / sqrt(n))).
 * diag R is the diagonal of the preconditioner from an FP8-e4m3 sparse-sign
 * sketch (s = min(2n, m), zeta = min(8, s)) and an FP32 QR, unscaled. */
int lsqo_features(const double* A, int64_t m, int64_t n, int64_t lda, uint64_t seed, double* f)
{
    int64_t s = 2 * n < m ? 2 * n : m;
    int zeta = s < 8 ? (int)s : 8;
    double* As = (double*)malloc(sizeof(double) * (size_t)s * (size_t)n);
    int32_t* ce = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    double* R = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
    double* cn = (double*)malloc(sizeof(double) * (size_t)n);
    double* ld = (double*)malloc(sizeof(double) * (size_t)n);
    int rc = lsqo_sketch(A, m, n, lda, O_SPARSE_SIGN, s, zeta, seed, O_FP8, As, ce);
    if (!rc) rc = lsqo_qr_r(As, s, n, s, O_FP32, R);
    if (!rc) {
        lsqo_unscale_r(R, n, n, ce);
        double fro = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double t = 0.0;
            for (int64_t i = 0; i < m; ++i) t += A[IDX(i, j, lda)] * A[IDX(i, j, lda)];
            fro += t;
            cn[j] = log10(sqrt(t) > 1e-300 ? sqrt(t) : 1e-300);
            double dj = fabs(R[IDX(j, j, n)]);
            ld[j] = log10(dj > 1e-300 ? dj : 1e-300);
        }
        double cmax = cn[0], cmin = cn[0], cmean = 0.0, dmax = ld[0], dmin = ld[0], dmean = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (cn[j] > cmax) cmax = cn[j];
            if (cn[j] < cmin) cmin = cn[j];
            if (ld[j] > dmax) dmax = ld[j];
            if (ld[j] < dmin) dmin = ld[j];
            cmean += cn[j];
            dmean += ld[j];
        }
        cmean /= n;
        dmean /= n;
        double cvar = 0.0, dvar = 0.0, sxy = 0.0, sxx = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double t = (double)j / (double)n - 0.5 * (double)(n - 1) / (double)n;
            cvar += (cn[j] - cmean) * (cn[j] - cmean);
            dvar += (ld[j] - dmean) * (ld[j] - dmean);
            sxy += t * (ld[j] - dmean);
            sxx += t * t;
        }
        int64_t q0 = n - (n + 3) / 4;
        double tmax = ld[q0], tmin = ld[q0];
        for (int64_t j = q0; j < n; ++j) {
            if (ld[j] > tmax) tmax = ld[j];
            if (ld[j] < tmin) tmin = ld[j];
        }
        int64_t small = 0;
        for (int64_t j = 0; j < n; ++j) small += (ld[j] < dmax - 2.0);
        f[0] = log2((double)m) / 16.0;
        f[1] = log2((double)n) / 10.0;
        f[2] = cmax - cmin;
        f[3] = sqrt(cvar / n);
        f[4] = dmax - dmin;
        f[5] = sqrt(dvar / n);
        f[6] = sxx > 0.0 ? sxy / sxx : 0.0;
        f[7] = tmax - tmin;
        f[8] = (double)small / (double)n;
        f[9] = dmin - log10(sqrt(fro / (double)n) > 1e-300 ? sqrt(fro / (double)n) : 1e-300);
    }
    free(As); free(ce); free(R); free(cn); free(ld);
    return rc;
}
