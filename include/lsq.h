/*
 * liblsq — randomized-preconditioned normal equations on NVIDIA GB300.
 *
 * The method is that of Garrison & Ipsen, "Perturbation Analysis for
 * Preconditioned Normal Equations in Mixed Precision" (arXiv 2603.16644):
 * for A (m x n, rank n) and b, Alg. 1
 *   1. estimates kappa0 ~ log10 kappa(A) in single precision (Sec. 6.1) and
 *      picks the preconditioner precision u_p;
 *   2. sketches A_s = Omega A in u_p and takes the thin QR A_s = Q_s R_s;
 *   3. promotes R_s to FP64 and forms A_p = A R_s^{-1} in FP64;
 *   4. solves PNE  (A_p^T A_p y = A_p^T b, R_s x = y;   Eq. e_pne)  or
 *             HPNE (A_p^T A x = A_p^T b;                 Eq. e_hpne).
 * This library adds, as options: Gaussian and sparse-sign sketches (the
 * paper uses a subsampled Fourier transform, Eq. e_sketch), FP8-e4m3 and
 * BF16 sketch precisions with per-column power-of-two scaling, and one FP64
 * residual-refinement step.
 *
 * Conventions for every call
 *   - Matrices are column-major FP64: entry (i, j) at A[i + j*lda], lda >= m.
 *   - Pointers are DEVICE pointers unless the name ends in _host.  The caller
 *     owns every buffer; inputs (const) are never modified.  The library
 *     never allocates device memory: scratch comes from the caller's
 *     workspace `ws` of at least lsq_workspace_size(...) bytes (256-byte
 *     aligned base recommended; the library aligns internally).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  All work is
 *     enqueued asynchronously on it, except where a call documents a
 *     host synchronisation.
 *   - Errors: the return value reports argument and launch errors.
 *     Conditions found on the device are written to the device int32 `info`
 *     (LAPACK style): 0 success, k > 0 breakdown (non-positive Cholesky
 *     pivot or zero LU pivot) at the k-th pivot, -1 non-finite value,
 *     -2 timeout.  Nothing throws across this interface.
 *   - Precondition: rank(A) = n and n <= s <= m (Sec. 1).  Rank deficiency
 *     shows up as a breakdown in info, not as undefined behaviour.
 */
#ifndef LSQ_H_
#define LSQ_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LSQ_OK = 0,
    LSQ_ERR_ARG = 1,        /* invalid argument (sizes, precision, null pointer) */
    LSQ_ERR_BREAKDOWN = 2,  /* reserved for synchronous callers: see info */
    LSQ_ERR_NONFINITE = 3,
    LSQ_ERR_TIMEOUT = 4,
    LSQ_ERR_CUDA = 5,       /* a CUDA launch or copy failed */
    LSQ_ERR_NOMEM = 6       /* workspace smaller than lsq_workspace_size() */
} lsq_status;

/* Precisions.  For the sketch, u_p of Alg. 1; AUTO runs the condition
 * estimate of Sec. 6.1 on A^T A (lsq_condest) and applies the precision
 * table below; AUTO_SKETCH runs the same estimator on the Gram of a sketch
 * (lsq_condest_sketch), which avoids the m n^2 pass and the FP32 Cholesky
 * breakdown of A^T A once kappa(A)^2 > 1/u32. */
typedef enum {
    LSQ_FP8_E4M3 = 0,  /* OCP FP8 e4m3 ("fn": no infinities, saturating) */
    LSQ_BF16 = 1,
    LSQ_FP16 = 2,      /* the paper's "half precision" */
    LSQ_FP32 = 3,      /* "single precision" */
    LSQ_FP64 = 4,      /* "double precision" */
    LSQ_AUTO = 5,
    LSQ_AUTO_SKETCH = 6
} lsq_prec;

typedef enum {
    LSQ_GAUSSIAN = 0,     /* Omega_ij ~ N(0, 1), unscaled */
    LSQ_SPARSE_SIGN = 1,  /* zeta distinct +-1 entries per column of Omega */
    LSQ_SRFT = 2          /* Omega = S F D of Eq. e_sketch: random signs D, the
                             unscaled Walsh-Hadamard transform F of order
                             m' = 2^ceil(log2 m) (A padded with zero rows),
                             s rows sampled with replacement (S) */
} lsq_sketch_kind;

typedef enum {
    LSQ_OP_SKETCH = 0,
    LSQ_OP_PRECOND_QR = 1,
    LSQ_OP_CONDEST = 2,
    LSQ_OP_PNE = 3,
    LSQ_OP_HPNE = 4,
    LSQ_OP_TRSM_GRAM = 5,
    LSQ_OP_FACTOR_SOLVE = 6,
    LSQ_OP_PNE_HOST = 7,
    LSQ_OP_HPNE_HOST = 8,
    LSQ_OP_CONDEST_SKETCH = 9,
    LSQ_OP_HPNE_QR = 10,
    LSQ_OP_SNE = 11,
    LSQ_OP_NNE = 12
} lsq_op;

/* Solver options (fixed-width fields; zero-initialise unused ones).
 *   kind          lsq_sketch_kind
 *   zeta          nonzeros per column of a sparse-sign Omega (1..32, <= s)
 *   s             sketch rows d of Omega (n <= s <= m; the paper uses 3n)
 *   seed          key of the Philox4x32-10 stream that draws Omega
 *   sketch_prec   u_p for the sketch (lsq_prec, AUTO allowed)
 *   qr_prec       arithmetic of the sketch QR: LSQ_FP32 or LSQ_FP64; forced
 *                 to FP64 when the sketch precision is FP64
 *   refine_steps  0 or 1 FP64 refinement steps (not in the paper)
 *   row_offset    0, or, when A is one row shard of a larger problem (see
 *                 lsq_set_reduce_hook), the global index of its first row:
 *                 the sketch operator's columns are drawn for the global
 *                 rows (Gaussian and sparse sign; not SRFT)            */
typedef struct {
    int32_t kind;
    int32_t zeta;
    int64_t s;
    uint64_t seed;
    int32_t sketch_prec;
    int32_t qr_prec;
    int32_t refine_steps;
    int32_t row_offset;
} lsq_opts;

/* ---- Row-sharded solves (the reduction is the caller's) ----------------
 * When A's rows are split over processes (A_k on GPU k, the rows of b
 * alike), every sum over rows in the path must be combined across the
 * shards: the column maxima of the sketch's power-of-two scaling (max), the
 * sketch A_s = sum_k Omega_k A_k, the Gram and right-hand side
 * sum_k A_pk^T A_pk (or A_pk^T A_k), sum_k A_pk^T b_k (A^T b for the
 * seminormal equations), the refinement's A_p^T r and the condition
 * estimate's A^T A.  The rest of the path (QR, factorizations, solves) is
 * replicated.  A hook registered here is called by the solve (host code, on
 * the solve's stream, enqueue order) right after each such partial result is
 * formed in device memory and before it is used; it must replace the
 * `count` entries of `buf` by their reduction over all shards (an
 * all-reduce on `stream`, or a synchronous one) and return LSQ_OK.  The
 * batched solver, the learned proposal and SRFT sketches do not take part.
 * No hook (the default, fn = NULL): single-process solves.  The library
 * builds no collective itself.  Process-wide; returns the previous hook. */
typedef enum {
    LSQ_REDUCE_SUM_F32 = 0,   /* float sum */
    LSQ_REDUCE_SUM_F64 = 1,   /* double sum */
    LSQ_REDUCE_MAX_U64 = 2    /* unsigned 64-bit max (column maxima as FP64 bit patterns) */
} lsq_reduce_kind;
typedef int32_t (*lsq_reduce_fn)(void* buf, int64_t count, int32_t kind, void* stream, void* user);
lsq_reduce_fn lsq_set_reduce_hook(lsq_reduce_fn fn, void* user);

/* Library version (major*10000 + minor*100 + patch). */
int32_t lsq_version(void);

/* Human-readable status name; static storage. */
const char* lsq_status_string(int32_t status);

/* Bytes of workspace the operation `op` (lsq_op) needs for an m x n problem
 * with the given options (opts may be NULL for ops that take none).
 * Returns 0 for invalid arguments. */
size_t lsq_workspace_size(int32_t op, int64_t m, int64_t n, const lsq_opts* opts);

/* Precision chosen by the table of Sec. 6.1 for an estimate kappa0
 * (reading extended to the 8-bit formats): kappa0 < 2 FP8-e4m3, < 3 BF16,
 * < 4 FP16 (the paper's half), <= 8 FP32, otherwise or non-finite FP64. */
int32_t lsq_precision_from_kappa0(double kappa0);

/* Sketch operator, for inspection and tests (Alg. 1 input Omega).
 * Sparse sign: idx[j*zeta + t] (int32, row of the t-th nonzero of column j,
 * distinct within a column, in draw order) and sgn[j*zeta + t] (+1/-1) for
 * j < m.  Draw rule: Philox4x32-10 with key = seed and counter
 * (k, j_lo, j_hi, 0), words in order, Lemire multiply-shift with rejection,
 * duplicates rejected; sign of the t-th row = bit t of word 0 of counter
 * (0, j_lo, j_hi, 1), set = -1. */
lsq_status lsq_sparse_sign_operator(uint64_t seed, int64_t m, int64_t s, int32_t zeta,
                                    int32_t* idx, int8_t* sgn, void* stream);

/* Gaussian operator rounded to `prec`, returned as FP64 values in Om
 * (s x m column-major, ld s).  Entry (i, j): the ziggurat of Marsaglia &
 * Tsang (2000) with 256 layers (r = 3.6541528853610088; tables built in FP64
 * from the equal-area recurrence f(x_{i+1}) = f(x_i) + v / x_i,
 * f(x) = exp(-x^2/2)).  Round k uses the Philox block of counter
 * (i, j_lo, j_hi, 2 + 256 k): layer = w0 & 255, sign = bit 8 of w0,
 * U = (2^30 (w0 >> 9) + (w1 >> 2)) 2^-53, proposal z = U x_layer; the wedge
 * test uses V = (2^26 (w2 >> 5) + (w3 >> 6)) 2^-53; the tail (layer 0 past
 * r) takes later rounds, e1 = -ln(U1)/r, e2 = -ln(U2), U1, U2 = V + 2^-53,
 * kept when 2 e2 > e1^2, value r + e1. */
lsq_status lsq_gaussian_operator(uint64_t seed, int64_t s, int64_t m, int32_t prec,
                                 double* Om, void* stream);

/* Sketch A_s = Omega (A 2^E) in precision opts->sketch_prec (Alg. 1,
 * "Sketch A_s = Omega A" in u_p).  Column j of A is scaled by 2^colexp[j]
 * before rounding to u_p so that its largest magnitude lies in
 * [2^(t-1), 2^t), t = 8 (FP8), 15 (FP16), 0 (BF16, FP32); FP64 is unscaled.
 * Products accumulate in FP32 (FP64 when u_p = FP64).  As (s x n,
 * column-major, ld ldas >= s) is float* for FP8/BF16/FP16/FP32 and double*
 * for FP64.  colexp: n int32 (device).  Sparse-sign sums run in ascending
 * column index of Omega.  SRFT: D from bit (j & 31) of word (j >> 5) & 3
 * of Philox counter (j >> 7, 0, 0, 3) (set = -1), F by butterfly levels
 * h = 1, 2, ..., m'/2 in order, (a, b) -> (a + b, a - b), in FP32 (FP64 for
 * an FP64 sketch) on the rounded, scaled A, sample t = word (t & 3) of
 * counter (t >> 2, 0, 0, 4) masked to [0, m'); bit-identical to a sequential
 * sweep.  AUTO is not accepted here.  info (device int32,
 * may be NULL) receives -3 if a row of a sparse-sign Omega holds more
 * nonzeros than the deterministic row sort supports, -2 if the index draw
 * did not terminate. */
lsq_status lsq_sketch(const double* A, int64_t m, int64_t n, int64_t lda, const lsq_opts* opts,
                      void* As, int64_t ldas, int32_t* colexp, int32_t* info, void* ws,
                      size_t ws_bytes, void* stream);

/* Preconditioner (Alg. 1, "Thin QR factorization A_s = Q_s R_s", then
 * "Promote R_s"): Householder QR of A_s (s x n; float* if as_prec = LSQ_FP32,
 * double* if LSQ_FP64) in qr_prec arithmetic (FP32 or FP64), R with positive
 * diagonal, promoted to FP64 and unscaled, R_s[:, j] = R[:, j] 2^-colexp[j]
 * (colexp may be NULL = no scaling).  Rs: n x n FP64, ld ldr >= n; only the
 * upper triangle is written.  info: device int32. */
lsq_status lsq_precond_qr(const void* As, int64_t s, int64_t n, int64_t ldas, int32_t as_prec,
                          int32_t qr_prec, const int32_t* colexp, double* Rs, int64_t ldr,
                          int32_t* info, void* ws, size_t ws_bytes, void* stream);

/* Low-precision condition estimate (Sec. 6.1; Alg. 1 first line): in FP32,
 * G = A^T A, ||G||_1, Cholesky of G and Hager's estimate gamma of
 * ||G^{-1}||_1 (at most 5 iterations, Higham's extra vector), then
 * kappa0 = 0.5 log10(n ||G||_1 gamma) in FP64; a breakdown or non-finite
 * value gives kappa0 = +inf.  kappa0 (double) and chosen (int32, lsq_prec by
 * lsq_precision_from_kappa0) are device pointers. */
lsq_status lsq_condest(const double* A, int64_t m, int64_t n, int64_t lda, double* kappa0,
                       int32_t* chosen, void* ws, size_t ws_bytes, void* stream);

/* Condition estimate on a sketch (a reading of Alg. 1's first line that
 * replaces A^T A of Sec. 6.1 by the Gram of a sketch):
 *   1. A_e = Omega_e A, an FP32 sparse-sign sketch with s_e = min(2n, m)
 *      rows and zeta = min(8, s_e) nonzeros per column, Philox key `seed`
 *      (as lsq_sketch);
 *   2. R_e, the FP32 Householder R of A_e (as lsq_precond_qr);
 *   3. the estimator of Sec. 6.1 on G_s = fl32(A_e^T A_e): ||G_s||_1 and
 *      Hager's estimate gamma of ||G_s^{-1}||_1 with G_s^{-1} applied through
 *      L = R_e^T (R_e^T R_e = G_s), kappa0 = 0.5 log10(n ||G_s||_1 gamma);
 *   4. if Hager's kappa_1(R_e) exceeds 1/u32 (an FP32 factor that does not
 *      resolve A, Lemma rscond), kappa0 = +inf and FP64 is chosen.
 * kappa0 (double) and chosen (int32, by lsq_precision_from_kappa0) are
 * device pointers.  Workspace lsq_workspace_size(LSQ_OP_CONDEST_SKETCH, m, n,
 * NULL). */
lsq_status lsq_condest_sketch(const double* A, int64_t m, int64_t n, int64_t lda, uint64_t seed, double* kappa0,
                              int32_t* chosen, void* ws, size_t ws_bytes, void* stream);

/* FP64 preconditioning and Gram formation (Alg. 1, "Solve A_p = A R_s^{-1}",
 * and the left-hand sides of Eqs. e_pne / e_hpne):
 *   Ap = A Rs^{-1} (m x n, ld ldap >= m; forward substitution by blocks);
 *   hpne = 0: G = Ap^T Ap (full symmetric n x n written);
 *   hpne = 1: G = Ap^T A;
 *   c = Ap^T b (n).   G: ld ldg >= n. */
lsq_status lsq_trsm_gram(const double* A, int64_t m, int64_t n, int64_t lda, const double* Rs,
                         int64_t ldr, const double* b, int32_t hpne, double* Ap, int64_t ldap,
                         double* G, int64_t ldg, double* c, void* ws, size_t ws_bytes,
                         void* stream);

/* lsq_trsm_gram without a workspace and without allocating.  The paper has
 * no counterpart: this is an interface for callers that cannot allocate
 * device memory where they call (inside an allocator or memory-pool
 * callback, in a framework that owns every device allocation, or in a loop
 * that must not take cudaMalloc's implicit device synchronisation).  They
 * pass the same inputs and outputs as lsq_trsm_gram; the scratch (split-K
 * partial Gram matrices and GEMV partial sums) is a fixed 16 MiB array that
 * every GPU loading the library holds until the process exits.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream
 *     capture.  The address is looked up again when the device's current
 *     context changes (after cudaDeviceReset, for instance), so such a call
 *     must not be the first one inside a capture either.
 *   - Sizes whose GEMV partial sums, 8 * ceil(m / 16384) * n bytes, exceed
 *     16 MiB are rejected with LSQ_ERR_ARG; the split-K count is capped so
 *     the partial Gram matrices fit in the rest, so large n runs with fewer
 *     splits (slower, same result up to summation order).
 *   - All calls share the one array and it keeps the last call's contents;
 *     every value read is first written by the same call, but calls that
 *     overlap on the GPU (concurrent streams) race on it.
 *   - No cudaMalloc, cudaFree or allocating library routine is called. */
lsq_status lsq_trsm_gram_noalloc(const double* A, int64_t m, int64_t n, int64_t lda, const double* Rs,
                                 int64_t ldr, const double* b, int32_t hpne, double* Ap, int64_t ldap,
                                 double* G, int64_t ldg, double* c, void* stream);

/* Factor and solve (Eqs. e_pne / e_hpne, right-hand parts), in FP64:
 *   hpne = 0: Cholesky G = L L^T, L L^T y = c, then Rs x = y (Rs may be
 *             NULL: x = y);
 *   hpne = 1: LU with partial pivoting (first largest pivot) P G = L U,
 *             L U x = P c.
 * G is overwritten by the factors (lower L for Cholesky; L\U for LU).
 * piv: n int32 (device, may be NULL for hpne = 0).  info: device int32.
 * The triangular solves run as a wavefront of 32-row blocks, one CTA each,
 * synchronised through flags in the workspace; the Cholesky trailing
 * updates are FP64-accurate tensor-core products (as in lsq_trsm_tc) with
 * their digits in the workspace too.  Workspace:
 * lsq_workspace_size(LSQ_OP_FACTOR_SOLVE, m, n, NULL), about 2 n 64 x 16
 * bytes (LSQ_ERR_NOMEM when smaller).  A wait that runs out (2 s) sets
 * info = -2. */
lsq_status lsq_factor_solve(int32_t hpne, double* G, int64_t n, int64_t ldg, const double* c,
                            const double* Rs, int64_t ldr, double* x, int32_t* piv, int32_t* info,
                            void* ws, size_t ws_bytes, void* stream);

/* Whole method (Alg. 1) with PNE (Eq. e_pne): x (n), Rs_out (n x n, ld n;
 * may be NULL), info (device int32), optional one-step FP64 refinement
 *   r = b - A x, g = A_p^T r, (A_p^T A_p) z = g, x += R_s^{-1} z.
 * With sketch_prec = AUTO the call runs lsq_condest and reads the chosen
 * precision back to the host (one stream synchronisation); the workspace is
 * then sized for the widest case (as for FP64). */
lsq_status lsq_pne_solve(const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
                         const lsq_opts* opts, double* x, double* Rs_out, int32_t* info,
                         void* ws, size_t ws_bytes, void* stream);

/* Same with HPNE (Eq. e_hpne): A_p^T A x = A_p^T b by LU with partial
 * pivoting; refinement r = b - A x, (A_p^T A) d = A_p^T r, x += d. */
lsq_status lsq_hpne_solve(const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
                          const lsq_opts* opts, double* x, double* Rs_out, int32_t* info,
                          void* ws, size_t ws_bytes, void* stream);

/* HPNE (Eq. e_hpne) with a QR factorization of H = A_p^T A instead of LU
 * (Sec. 1 names both): the Householder R of the (n+1) x (n+1) matrix
 * [[H, c], [0, 1]], c = A_p^T b, in FP64 (the preconditioner QR kernel),
 * holds R_H and Q_H^T c, and x = R_H^{-1} (Q_H^T c).  Refinement: the same
 * with A_p^T r in place of c.  Workspace LSQ_OP_HPNE_QR. */
lsq_status lsq_hpne_qr_solve(const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
                             const lsq_opts* opts, double* x, double* Rs_out, int32_t* info, void* ws,
                             size_t ws_bytes, void* stream);

/* Seminormal equations (Sec. 5, Eq. e_sne) R^T R x = A^T b with R the
 * triangular factor of a thin QR of A taken from the preconditioner:
 * A_p = A R_s^{-1} = Q R_p with R_p^T R_p = A_p^T A_p = L L^T (Cholesky), so
 * R = L^T R_s, applied in factored form:
 * x = R_s^{-1} L^{-T} L^{-1} R_s^{-T} (A^T b).  The error grows with
 * kappa(A)^2 (Thm. l_semi), against kappa(A) for PNE; one refinement step
 * (the corrected seminormal equations, A^T r on the right) recovers it.
 * Workspace LSQ_OP_SNE. */
lsq_status lsq_sne_solve(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, const lsq_opts* opts,
                         double* x, double* Rs_out, int32_t* info, void* ws, size_t ws_bytes, void* stream);

/* Not-normal equations (Sec. 5, Eq. e_nne) B^T A x = B^T b with
 * B = A U_s^{-1}, U_s the upper factor of the LU with partial pivoting
 * (first largest pivot) of the sketch A_s, computed in the preconditioner
 * precision (qr_prec arithmetic: FP32 or FP64) and unscaled like R_s; B has
 * A's column space and Omega B = P^T L_s.  Then as HPNE: B^T A by LU with
 * partial pivoting.  Us_out (n x n, may be NULL) receives U_s.  A zero pivot
 * of the sketch's LU is reported in info.  Workspace LSQ_OP_NNE. */
lsq_status lsq_nne_solve(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, const lsq_opts* opts,
                         double* x, double* Us_out, int32_t* info, void* ws, size_t ws_bytes, void* stream);

/* End-to-end variants on HOST buffers (pinned memory recommended): copy
 * A_host (ld lda) and b_host into the workspace, solve, copy x back to
 * x_host and info back to info_host; returns after a stream synchronisation.
 * Workspace: lsq_workspace_size(LSQ_OP_PNE_HOST / LSQ_OP_HPNE_HOST, ...). */
lsq_status lsq_pne_solve_host(const double* A_host, int64_t m, int64_t n, int64_t lda,
                              const double* b_host, const lsq_opts* opts, double* x_host,
                              int32_t* info_host, void* ws, size_t ws_bytes, void* stream);
lsq_status lsq_hpne_solve_host(const double* A_host, int64_t m, int64_t n, int64_t lda,
                               const double* b_host, const lsq_opts* opts, double* x_host,
                               int32_t* info_host, void* ws, size_t ws_bytes, void* stream);

/* Dense contraction on the tensor cores (tcgen05, TMA-fed, FP32 accumulators
 * in TMEM), the kernel behind the Gaussian sketch (Alg. 1, "Sketch
 * A_s = Omega A"): C (M x N, column-major ld ldc, FP32) = X Y^T with X (M x K)
 * and Y (N x K) both K-contiguous (row r of X at X + r*ldx), stored as
 * FP8-e4m3 (prec = LSQ_FP8_E4M3, bytes), BF16 or FP16.  ldx, ldy multiples of
 * 16 elements; X, Y 16-byte aligned.  K may be split over CTAs (workspace
 * lsq_tc_gemm_workspace_size); partial sums are reduced in a fixed order.
 * info (device int32, may be NULL) receives -2 if a pipeline wait timed out. */
size_t lsq_tc_gemm_workspace_size(int32_t prec, int64_t M, int64_t N, int64_t K);
lsq_status lsq_tc_gemm(int32_t prec, const void* X, int64_t ldx, const void* Y, int64_t ldy, int64_t M, int64_t N,
                       int64_t K, float* C, int64_t ldc, int32_t* info, void* ws, size_t ws_bytes, void* stream);

/* FP64 Gram G = X^T X (the left-hand side of Eq. e_pne with X = A_p) on the
 * FP8 tensor cores: every column p of X (m x n, ld) is written as 14
 * base-16 digits in [-15, 15] relative to 2^(e_p) > max_i |x_ip| (56 bits,
 * extracted with integer operations); the digit-pair products t + u <= 13
 * are exact integer sums in the FP32 accumulators (K chunks of 65536 rows)
 * and are combined in FP64 smallest weight first, then scaled by
 * 2^(e_p + e_q).  Per entry the error is below ~2^-55 m max|x_p| max|x_q|,
 * the order of FP64 rounding.  G: n x n FP64, full symmetric, ld ldg.
 * Workspace lsq_gram_tc_workspace_size(m, n) (about 14 m n bytes of digits
 * plus 64 KiB per digit tile).  info (device, may be NULL): -2 on a pipeline
 * timeout. */
size_t lsq_gram_tc_workspace_size(int64_t m, int64_t n);
lsq_status lsq_gram_tc(const double* X, int64_t m, int64_t n, int64_t ld, double* G, int64_t ldg, int32_t* info,
                       void* ws, size_t ws_bytes, void* stream);

/* G = X^T Y (n x n, FP64 accuracy) for two m x n column-major FP64 matrices,
 * by the same FP8 digit slicing as lsq_gram_tc with one exponent per column
 * of X and of Y; the HPNE matrix A_p^T A (Eq. e_hpne).  All 105 digit-pair
 * blocks are formed (no symmetry).  Per entry the error is below ~2^-55 m
 * max|x_p| max|y_q|.  Workspace lsq_gemm_tn_tc_workspace_size(m, n) (about
 * 28 m n bytes of digits plus 64 KiB per digit tile).  info (device, may be
 * NULL): -2 on a pipeline timeout. */
size_t lsq_gemm_tn_tc_workspace_size(int64_t m, int64_t n);
lsq_status lsq_gemm_tn_tc(const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t m, int64_t n,
                          double* G, int64_t ldg, int32_t* info, void* ws, size_t ws_bytes, void* stream);

/* A_p = A R^{-1} (Alg. 1, the preconditioned matrix formed by substitution)
 * in FP64 with the off-diagonal products on the tensor cores.  The columns
 * are split recursively; diagonal blocks of up to 32 columns are solved by
 * FP64 substitution, and each update A_p[:, right] = A[:, right] -
 * A_p[:, left] R[left, right] (left part <= 512 columns) is an FP64-accurate
 * product of BF16 digit slices: every value becomes 8 balanced base-128
 * digits relative to the largest magnitude of its row (of A_p) or column (of
 * R); the 36 digit pairs with t + u <= 7 accumulate exactly in FP32 and are
 * combined as exact 64-bit integers, rounded once to FP64.  Per product the
 * error is below 2^-52.6 2^(E_i + E_j) where 2^E bounds the row / column,
 * the order of FP64 rounding.
 * A: m x n FP64 column-major (ld lda); R: n x n upper triangular (ld ldr,
 * nonzero diagonal); Ap: m x n output (ld ldap; must not overlap A unless
 * Ap == A with ldap == lda, the in-place form).  Device pointers, caller-owned.
 * Workspace lsq_trsm_tc_workspace_size(m, n) (about 8 m min(n/2, 512) x 2
 * bytes of digits).  info (device, may be NULL): -2 on a pipeline timeout.
 * Returns LSQ_ERR_ARG when the tensor-map encoder is unavailable. */
size_t lsq_trsm_tc_workspace_size(int64_t m, int64_t n);
lsq_status lsq_trsm_tc(const double* A, int64_t m, int64_t n, int64_t lda, const double* R, int64_t ldr, double* Ap,
                       int64_t ldap, int32_t* info, void* ws, size_t ws_bytes, void* stream);

/* Use the tensor-core FP64 products (lsq_gram_tc for the symmetric Gram of
 * PNE, lsq_gemm_tn_tc for A_p^T A of HPNE, lsq_trsm_tc for A_p and the
 * Cholesky updates) inside the solves (1, the
 * default) or the FP64 CUDA-core kernels (0); returns the previous setting.
 * Process-wide; for comparisons. */
int32_t lsq_set_fp64_emulation(int32_t enable);

/* Test-only fault injection (no GPU fault): the bound, in nanoseconds, of
 * each wait of the wavefront triangular solves for another block's solution
 * (default 2e9).  A wait that runs out records -2 in `info` and passes NaN on
 * to the blocks after it; the kernel returns normally and the context stays
 * usable.  Process-wide; returns the previous bound, or -1 (unchanged) for
 * ns <= 0. */
int64_t lsq_test_set_solve_wait_ns(int64_t ns);

/* ---- Batched solves (many independent problems of uneven shape) --------- */

/* One problem of a batch: device pointers A (m x n, ld lda), b (m), x (n),
 * info (device int32), and its own options (sketch kind, s, zeta, seed,
 * sketch precision including AUTO and AUTO_SKETCH, QR precision, refinement). */
typedef struct {
    const double* A;
    int64_t m;
    int64_t n;
    int64_t lda;
    const double* b;
    double* x;
    int32_t* info;
    int32_t reserved0;
    int32_t reserved1;
    lsq_opts opts;
} lsq_batch_problem;

/* Workspace bytes for a batch (hpne = 0 PNE, 1 HPNE); 0 on invalid input. */
size_t lsq_batched_workspace_size(int32_t hpne, int32_t count, const lsq_batch_problem* probs);

/* Alg. 1 with PNE (Eq. e_pne) or HPNE (Eq. e_hpne) on `count` independent
 * problems.  The problems are spread over 16 internal streams (or
 * $LSQ_BATCH_STREAMS, 1 to 64, read once per process; the workspace size
 * grows with it), heaviest first to the least-loaded stream, and the whole
 * fan-out is captured into one
 * CUDA graph launched on `stream`; the executable graph is cached and
 * replayed while the descriptors (pointers, shapes, options, workspace) stay
 * the same.  Problems with sketch_prec = AUTO or AUTO_SKETCH first get one
 * batched condition-estimate pass (the same fan-out, in a cached graph of
 * its own) and one readback of the chosen precisions (a stream
 * synchronisation).  Each problem's status goes to its own info.
 * Every problem still runs its own kernel sequence inside the graph (no
 * single persistent kernel walks the batch).  Not thread safe: one batched
 * call at a time per process. */
lsq_status lsq_pne_solve_batched(int32_t count, const lsq_batch_problem* probs, void* ws, size_t ws_bytes,
                                 void* stream);
lsq_status lsq_hpne_solve_batched(int32_t count, const lsq_batch_problem* probs, void* ws, size_t ws_bytes,
                                  void* stream);

/* Batched sketch (Alg. 1, "Sketch A_s = Omega A" in u_p, for many problems):
 * each entry is one lsq_sketch call (its own shape, options and outputs; the
 * precision must not be AUTO).  The calls are spread over the internal
 * streams and captured into one CUDA graph like the batched solves (cached
 * while the descriptors stay the same); results are those of separate
 * lsq_sketch calls. */
typedef struct {
    const double* A;
    int64_t m;
    int64_t n;
    int64_t lda;
    void* As;          /* s x n, ld ldas: float* (FP8/BF16/FP16/FP32) or double* (FP64) */
    int64_t ldas;
    int32_t* colexp;   /* n int32 (device) */
    int32_t* info;     /* device int32, may be NULL */
    lsq_opts opts;
} lsq_sketch_problem;
size_t lsq_sketch_batched_workspace_size(int32_t count, const lsq_sketch_problem* probs);
lsq_status lsq_sketch_batched(int32_t count, const lsq_sketch_problem* probs, void* ws, size_t ws_bytes,
                              void* stream);

/* Batched preconditioner QR (Alg. 1, "Thin QR factorization", "Promote
 * R_s"): each entry is one lsq_precond_qr call; same fan-out and graph as
 * above; results are those of separate calls. */
typedef struct {
    const void* As;        /* s x n, ld ldas, float* (as_prec FP32) or double* (FP64) */
    int64_t s;
    int64_t n;
    int64_t ldas;
    int32_t as_prec;
    int32_t qr_prec;
    const int32_t* colexp; /* may be NULL */
    double* Rs;            /* n x n, ld ldr */
    int64_t ldr;
    int32_t* info;         /* device int32 */
} lsq_qr_problem;
size_t lsq_precond_qr_batched_workspace_size(int32_t count, const lsq_qr_problem* probs);
lsq_status lsq_precond_qr_batched(int32_t count, const lsq_qr_problem* probs, void* ws, size_t ws_bytes,
                                  void* stream);

/* ---- Learned precision proposal (an addition to the paper; the paper's
 * estimator of Sec. 6.1, on the Gram of a sketch, judges every proposal that
 * could lose accuracy and is the fallback) -------------------------------- */

/* Number of MLP parameters for d input features (d -> 64 -> 64 -> 64 -> 4,
 * packed W1 b1 W2 b2 W3 b3 W4 b4, W row-major out x in), and d itself. */
int64_t lsq_mlp_param_count(int32_t d);
int32_t lsq_mlp_num_features(void);

/* The 10 proposal features of A (FP32, device f[10]): log2 m / 16,
 * log2 n / 10, log10 spread and std of the column 2-norms, and statistics of
 * log10 |diag R| for the preconditioner R of an FP8-e4m3 sparse-sign sketch
 * (s = min(2n, m), zeta = min(8, s), key seed) with an FP32 QR: spread, std,
 * slope against j/n, spread over the last quarter, fraction more than 100x
 * below the largest, and the smallest relative to ||A||_F / sqrt(n). */
size_t lsq_features_workspace_size(int64_t m, int64_t n);
lsq_status lsq_features(const double* A, int64_t m, int64_t n, int64_t lda, uint64_t seed, float* f, void* ws,
                        size_t ws_bytes, void* stream);

/* MLP in FP32 on the device.  forward: logits (batch x 4) for X (batch x d,
 * row-major).  backward: gradient of the mean softmax cross-entropy against
 * labels (0 FP8-e4m3, 1 BF16, 2 FP32, 3 FP64) in the parameter packing, and
 * the loss (device float, may be NULL); sums over the batch run in sample
 * order (deterministic).  adam: one Adam step (step counts from 1). */
lsq_status lsq_mlp_forward(const float* params, int32_t d, int32_t batch, const float* X, float* logits,
                           void* stream);
size_t lsq_mlp_backward_workspace_size(int32_t d, int32_t batch);
lsq_status lsq_mlp_backward(const float* params, int32_t d, int32_t batch, const float* X, const int32_t* labels,
                            float* grad, float* loss, void* ws, size_t ws_bytes, void* stream);
lsq_status lsq_mlp_adam(float* params, const float* grad, float* m1, float* m2, int64_t count, float lr,
                        float beta1, float beta2, float eps, int32_t step, void* stream);

/* Features + MLP: proposed sketch precision (device int32, lsq_prec) and
 * the class probabilities (device float[4], may be NULL).  Workspace:
 * lsq_features_workspace_size(m, n). */
lsq_status lsq_propose_precision(const double* A, int64_t m, int64_t n, int64_t lda, uint64_t seed,
                                 const float* params, int32_t d, int32_t* prec, float* probs, void* ws,
                                 size_t ws_bytes, void* stream);

/* Judge of a computed preconditioner R_s (n x n upper FP64): Hager's
 * single-precision 1-norm estimate (Sec. 6.1) of kappa_1(R_s) -> kappa1
 * (device double); accept (device int32) = 1 iff u_p * kappa1 <= 1 for the
 * precision u_p it was computed in, i.e. Lemma rscond's eps kappa(R_s) < 1. */
size_t lsq_judge_workspace_size(int64_t n);
lsq_status lsq_judge_preconditioner(const double* Rs, int64_t n, int64_t ldr, int32_t prec, int32_t* accept,
                                    double* kappa1, void* ws, size_t ws_bytes, void* stream);

/* PNE (Alg. 1) with the learned proposal: the MLP proposes u_p.  A proposal
 * below FP64 could lose accuracy, so the paper's estimator judges it
 * (lsq_condest_sketch, key opts->seed): when the estimate's own choice is a
 * higher precision, that choice replaces the proposal (the fallback; one
 * escalation).  The preconditioner is then computed in u_p and its FP32
 * kappa_1 estimate gives a second opinion (u_p kappa_1(R_s) <= 1, Lemma
 * rscond), escalating FP8 -> BF16 -> FP32 -> FP64 until accepted.  An FP64
 * proposal needs no judge (and skips the estimate).  The solve finishes with
 * the accepted R_s.  used_prec and escalations are HOST int32 outputs; the
 * call synchronises the stream after the proposal, the estimate and each
 * judged candidate.  opts gives the sketch kind, s, zeta, seed and
 * refinement; its precisions are ignored. */
size_t lsq_learned_workspace_size(int64_t m, int64_t n, const lsq_opts* opts);
lsq_status lsq_pne_solve_learned(const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
                                 const lsq_opts* opts, const float* params, int32_t d, double* x, int32_t* info,
                                 int32_t* used_prec, int32_t* escalations, void* ws, size_t ws_bytes,
                                 void* stream);

/* ---- Instrumentation (no counterpart in the paper) --------------------- */

/* Route Gaussian sketches in FP8-e4m3 / BF16 / FP16 to the tensor-core
 * kernel (enable = 1, the default) or to the CUDA-core GEMM (0); returns
 * the previous setting.  Process-wide; for tests and comparisons. */
int32_t lsq_set_tensor_core_sketch(int32_t enable);

/* The CUDA error string behind the most recent LSQ_ERR_CUDA of this
 * process ("no error" if none). */
const char* lsq_last_cuda_error(void);

/* Number of kernel launches this library has issued since it was loaded. */
int64_t lsq_launch_count(void);

/* Stage timing.  lsq_profile(1) clears the records and starts recording a
 * CUDA event pair around each step of Alg. 1 inside the solve calls (stage
 * indices: 0 condition estimate, 1 sketch, 2 QR, 3 TRSM A R_s^{-1},
 * 4 Gram + right-hand side, 5 factorization, 6 solves, 7 refinement;
 * 8 single launches of the tensor-core FP64 update kernel (lsq_trsm_tc,
 * the Cholesky updates), 9 single launches of the QR panel kernel, 10 single
 * launches of the tensor-core sketch GEMM, 11 single launches of the update
 * kernel with three-digit X (the K chunks of an FP64 Gaussian sketch));
 * lsq_profile(0) stops.  lsq_profile_collect waits for the recorded events,
 * writes the summed milliseconds and the number of records per stage
 * (arrays of at least 8; indices >= nstages are skipped), and clears the
 * records; lsq_profile_collect_work also writes the summed algorithmic work
 * per stage (flops: 36 digit-pair products of 2 M N K each for the update
 * kernel, 21 for its three-digit form, the Householder panel flops for the
 * QR panel, 2 M N K of the
 * launch's K for the sketch GEMM, which is six times the product's for an
 * FP32 sketch of BF16 pieces; 0 for the steps).
 * Host-side state, not thread safe across concurrent solves on different
 * streams. */
int32_t lsq_profile(int32_t enable);
int32_t lsq_profile_collect(double* ms_by_stage, int32_t* count_by_stage, int32_t nstages);
int32_t lsq_profile_collect_work(double* ms_by_stage, int32_t* count_by_stage, double* work_by_stage,
                                 int32_t nstages);
/* The individual records of one stage since the last collect (before
 * lsq_profile_collect*, which clears them): milliseconds and work of the
 * first `cap` records into ms / work; returns the number of records of that
 * stage (negative status on error).  Waits for the events. */
int32_t lsq_profile_records(int32_t stage, double* ms, double* work, int32_t cap);

#ifdef __cplusplus
}
#endif

#endif /* LSQ_H_ */
