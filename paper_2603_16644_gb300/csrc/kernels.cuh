// Internal launcher declarations shared by the translation units of liblsq.
#pragma once
#include "common.cuh"

namespace lsq {

__device__ __forceinline__ int64_t ceil_div_dev(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Conversion of a stored element to the accumulation type (exact for every
// stored format into float; double -> float rounds to nearest even).
template <typename TS, typename TACC>
__device__ __forceinline__ TACC to_acc(TS v);
template <> __device__ __forceinline__ float to_acc<__nv_fp8_storage_t, float>(__nv_fp8_storage_t v) {
    return __half2float(__half(__nv_cvt_fp8_to_halfraw(v, __NV_E4M3)));
}
template <> __device__ __forceinline__ float to_acc<__nv_bfloat16, float>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ float to_acc<__half, float>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float to_acc<float, float>(float v) { return v; }
template <> __device__ __forceinline__ float to_acc<double, float>(double v) { return __double2float_rn(v); }
template <> __device__ __forceinline__ double to_acc<double, double>(double v) { return v; }
template <> __device__ __forceinline__ double to_acc<float, double>(float v) { return (double)v; }

// ---- sketch.cu --------------------------------------------------------------
lsq_status launch_sparse_gen(uint64_t seed, int64_t m, int64_t s, int zeta, int32_t* idx, int8_t* sgn, int32_t* err,
                             int64_t j0,
                             cudaStream_t st);
int sort_cap_for(int64_t m, int64_t s, int zeta);
lsq_status launch_sparse_csr(const int32_t* idx, const int8_t* sgn, int64_t m, int64_t s, int zeta, int32_t* counts,
                             int32_t* rowptr, int32_t* cursor, uint32_t* col, int32_t* maxcount, int32_t* err,
                             cudaStream_t st);
lsq_status launch_colexp(const double* A, int64_t m, int64_t n, int64_t lda, int prec, unsigned long long* colmax,
                         int32_t* colexp, cudaStream_t st);
lsq_status launch_quantize_rm(const double* A, int64_t m, int64_t n, int64_t lda, const int32_t* colexp, int prec,
                              void* out, cudaStream_t st);
lsq_status launch_quantize_cm(const double* A, int64_t m, int64_t n, int64_t lda, const int32_t* colexp, int prec,
                              void* out, int64_t ldq, cudaStream_t st);
lsq_status launch_sparse_gather(const int32_t* rowptr, const uint32_t* col, const void* Ahat, int prec, int64_t s,
                                int64_t n, void* As, int64_t ldas, cudaStream_t st);
// j0: global index of A's first row (row-sharded A), the column offset of Omega
lsq_status launch_gauss_gen(uint64_t seed, int64_t s, int64_t m, int prec, void* Om, int64_t ldo, int64_t j0,
                            cudaStream_t st);
lsq_status launch_gauss_inspect(uint64_t seed, int64_t s, int64_t m, int prec, double* Om, cudaStream_t st);
// FP32 Gaussian sketch as one BF16 GEMM over six K segments of length L
// (three BF16 pieces per FP32 value, pairs t + u <= 2).
lsq_status launch_gauss_split3(uint64_t seed, int64_t s, int64_t m, int64_t L, uint16_t* X, int64_t j0,
                               cudaStream_t st);
lsq_status launch_quantize_split3(const double* A, int64_t m, int64_t n, int64_t lda, const int32_t* colexp,
                                  int64_t L, uint16_t* Y, cudaStream_t st);
// FP32 Gram X^T X (X: m x n, FP64 or FP32, rounded to FP32) as one BF16 GEMM:
// seven K segments per column (h l h m m h h); X at Z, Y at Z + L, ld 7L, K 6L.
template <typename TI>
lsq_status launch_gram_split3(const TI* A, int64_t m, int64_t n, int64_t lda, int64_t L, uint16_t* Z, cudaStream_t st);
// Row-sharded use: hand a partial sum to the caller's reduction hook
// (lsq_set_reduce_hook); LSQ_OK without a hook.
lsq_status reduce_partial(void* buf, int64_t count, int kind, cudaStream_t st);
// Gaussian sketches in FP8/BF16/FP16/FP32 and the FP32 Gram of the condition
// estimate on the tensor cores (lsq_set_tensor_core_sketch).
bool tensor_core_sketch_enabled();
// Subsampled randomized Walsh-Hadamard sketch (kind LSQ_SRFT): W is
// srft_ws_bytes of scratch (the signed, padded, transformed columns).
int64_t srft_order(int64_t m);
size_t srft_ws_bytes(int64_t m, int64_t n, int prec);
lsq_status launch_srft(const double* A, int64_t m, int64_t n, int64_t lda, const int32_t* colexp, int prec,
                       uint64_t seed, int64_t s, void* W, void* As, int64_t ldas, cudaStream_t st);
// Columns [k0, k0 + kc) of -Omega (FP64), s x kc column-major, ld s.

// ---- gemm.cu: dense contractions on CUDA cores ------------------------------
// C (M x N, column-major, ldc) = sum_k X[i*ldx + k] * Y[j*ldy + k]  (both
// operands K-contiguous), split over K into `splits` partial products reduced
// in a fixed order.  sym: only tiles i >= j are computed and C is mirrored.
// xprec/yprec: storage precision of X/Y (lsq_prec); acc: LSQ_FP32 or LSQ_FP64.
struct GemmPlan {
    int64_t M, N, K;
    int splits;
    int64_t kchunk;
    bool sym;
    int acc;
};
GemmPlan plan_gemm_kmajor(int64_t M, int64_t N, int64_t K, bool sym, int acc, int num_sms);
size_t gemm_kmajor_ws_bytes(const GemmPlan& p);
lsq_status launch_gemm_kmajor(const GemmPlan& p, const void* X, int xprec, int64_t ldx, const void* Y, int yprec,
                              int64_t ldy, void* C, int64_t ldc, void* ws, cudaStream_t st);

// FP64 right triangular solve Ap = A R^{-1} (R upper, n x n).
lsq_status launch_trsm_right_upper(const double* A, int64_t m, int64_t n, int64_t lda, const double* R, int64_t ldr,
                                   double* Ap, int64_t ldap, cudaStream_t st);

// c = X^T v over m rows (X column-major ldx), deterministic.
lsq_status launch_gemv_t(const double* X, int64_t m, int64_t n, int64_t ldx, const double* v, double* c,
                         double* partial, int64_t max_partial, cudaStream_t st);
size_t gemv_t_ws_bytes(int64_t m, int64_t n);
// r = b - A x over m rows.
lsq_status launch_residual(const double* A, int64_t m, int64_t n, int64_t lda, const double* x, const double* b,
                           double* r, cudaStream_t st);
// x += d
lsq_status launch_axpy1(double* x, const double* d, int64_t n, cudaStream_t st);

// ---- factor.cu: n x n factorizations and triangular solves ------------------
// FP64 with ws (>= cholesky_ws_bytes(n)): trailing updates on the tensor cores.
template <typename T>
lsq_status launch_cholesky(T* G, int64_t n, int64_t ld, int32_t* info, cudaStream_t st, void* ws = nullptr,
                           size_t ws_bytes = 0);
size_t cholesky_ws_bytes(int64_t n);
lsq_status launch_lu(double* H, int64_t n, int64_t ld, int32_t* piv, int32_t* info, cudaStream_t st);
enum TrsvKind { TRSV_LOWER = 0, TRSV_LOWER_T = 1, TRSV_UPPER = 2, TRSV_UNIT_LOWER = 3, TRSV_UPPER_T = 4 };
// sync: trsv_sync_ints(n) int32 of scratch (cleared by the launch); err: the
// device status word that a timed-out wait sets to -2 (may be NULL).
size_t trsv_sync_ints(int64_t n);
// Bound of the wavefront solves' waits (process-wide; returns the previous one).
uint64_t set_trsv_wait_ns(uint64_t ns);
template <typename T>
lsq_status launch_trsv(int kind, const T* M, int64_t n, int64_t ld, T* y, const int32_t* info, int32_t* sync,
                       int32_t* err, cudaStream_t st);
lsq_status launch_apply_piv(const int32_t* piv, int64_t n, double* y, const int32_t* info, cudaStream_t st);

template <typename T>
lsq_status rank_update_ext(T* C, int64_t ldc, const T* P, int64_t psi, int64_t psk, const T* Q, int64_t qsj,
                           int64_t qsk, int64_t M, int64_t N, int K, bool lower, const int32_t* info, cudaStream_t st);

// ---- sketch_tc.cu: tcgen05 Gaussian sketch for 8/16-bit u_p --------------
bool sketch_tc_supported(int prec);
size_t sketch_tc_ws_bytes(int64_t s, int64_t n, int64_t m, int prec, int sms);
lsq_status launch_sketch_tc(const void* Om, int64_t ldo, const void* Ahat, int64_t ldq, int prec, int64_t s,
                            int64_t n, int64_t m, float* As, int64_t ldas, void* ws, size_t ws_bytes, int32_t* err,
                            cudaStream_t st, bool blocked = false);

// ---- ozaki.cu: FP64 Gram on the FP8 tensor cores (digit slicing) ----------
size_t oz_gram_ws_bytes(int64_t m, int64_t n);
lsq_status oz_gram(const double* X, int64_t m, int64_t n, int64_t ld, double* G, int64_t ldg, void* ws,
                   size_t ws_bytes, int32_t* err, cudaStream_t st);
// G = X^T Y (both m x n column-major), FP64 accuracy, non-symmetric.
size_t oz_gemm_tn_ws_bytes(int64_t m, int64_t n);
lsq_status oz_gemm_tn(const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t m, int64_t n, double* G,
                      int64_t ldg, void* ws, size_t ws_bytes, int32_t* err, cudaStream_t st);

// ---- oz_trsm.cu: FP64 Ap = A R^{-1} with tensor-core updates -------------
bool ot_trsm_supported();
// FP64 products on the tensor cores (lsq_set_fp64_emulation; default on).
bool fp64_emulation_enabled();
size_t ot_trsm_ws_bytes(int64_t m, int64_t n);
lsq_status ot_trsm(const double* A, int64_t m, int64_t n, int64_t lda, const double* R, int64_t ldr, double* Ap,
                   int64_t ldap, void* ws, size_t ws_bytes, int32_t* err, cudaStream_t st);
// C_out = C_in - X Y with FP64 accuracy on the tensor cores (X: M x K
// column-major, ld ldx; Y entry (k, j) at Y[k sk + j sj]; K <= 512, or
// K <= 1024 with x_digits = 3).
// xmode 2: X's digit planes were written by ot_gauss_digits (X unused).
// x_digits = 3 when every row of X has at most three nonzero balanced
// base-128 digits below its maximum (X on a 2^-17 grid, |X| < 8: the
// Gaussian sketch operator); the product is then the same with 21 digit
// pairs instead of 36.
size_t ot_update_ws_bytes(int64_t M, int64_t N, int64_t K);
lsq_status ot_gemm_update(const double* X, int64_t ldx, const double* Y, int64_t sk, int64_t sj, const double* Cin,
                          int64_t ldi, double* Cout, int64_t ldo, int64_t M, int64_t N, int64_t K, void* ws,
                          size_t ws_bytes, int32_t* err, cudaStream_t st, int xmode = 0,
                          const int32_t* Eblk = nullptr, int64_t b0 = 0, int nbk = 0, int x_digits = 8);
// The negated Gaussian operator's columns j0 .. j0 + kc - 1 (rows 0 .. s - 1,
// kc <= 1024) written as the X digit planes of an update's scratch ws (the
// scratch of ot_gemm_update with M = s, N, K = kc), for ot_gemm_update with
// xmode = 2 and x_digits = 3.
lsq_status ot_gauss_digits(uint64_t seed, int64_t s, int64_t j0, int64_t kc, int64_t N, void* ws, size_t ws_bytes,
                           cudaStream_t st);

// ---- hager.cu ----------------------------------------------------------------
// Hager's estimate of ||M^{-1}||_1 in FP32 into *est (device), M n x n
// (ld ld): (L L^T)^{-1} for L lower (upper = false) or R^{-1} for R upper.
// fail (device, may be NULL): nonzero skips every solve (*est = +inf);
// err: set to -2 when a wavefront solve's wait times out.
size_t hager_ws_bytes(int64_t n);
lsq_status hager_inv_norm1(const float* M, int64_t n, int64_t ld, bool upper, const int32_t* fail, float* est,
                           int32_t* err, void* ws, size_t ws_bytes, cudaStream_t st);
// ||M||_1 (upper: of the upper triangle) into *out (device float).
lsq_status launch_colnorm1_max(const float* M, int64_t n, int64_t ld, bool upper, float* out, cudaStream_t st);

// ---- qr.cu -------------------------------------------------------------------
size_t qr_ws_bytes(int64_t s, int64_t n, int prec);
lsq_status launch_precond_qr(const void* As, int64_t s, int64_t n, int64_t ldas, int as_prec, int qr_prec,
                             const int32_t* colexp, double* Rs, int64_t ldr, int32_t* info, void* ws, size_t ws_bytes,
                             cudaStream_t st);

// ---- condest.cu --------------------------------------------------------------
size_t condest_ws_bytes(int64_t m, int64_t n, int num_sms);
// Estimate on a sketch: finish from G_s (FP32, of the scaled sketch; colexp
// undoes the scaling), R_e and the FP32 judge's verdict on R_e.
size_t condest_sketch_finish_ws_bytes(int64_t n);
// LU with partial pivoting of the sketch (s x n) in FP32 or FP64 arithmetic;
// U_s = U 2^-colexp promoted to FP64 (the not-normal equations' B = A U_s^{-1}).
size_t lu_precond_ws_bytes(int64_t s, int64_t n, int prec);
lsq_status launch_lu_precond(const void* As, int64_t s, int64_t n, int64_t ldas, int as_prec, int lu_prec,
                             const int32_t* colexp, double* Us, int64_t ldu, int32_t* info, void* ws, size_t ws_bytes,
                             cudaStream_t st);
lsq_status launch_condest_sketch_finish(float* G, const int32_t* colexp, const double* Re, int64_t n, int64_t ldr,
                                        const int32_t* accept, double* kappa0, int32_t* chosen, void* ws,
                                        size_t ws_bytes, cudaStream_t st);
// FP32 judge of a preconditioner (mlp.cu): Hager's kappa_1(R_s), accept = u_p kappa_1 <= 1.
size_t judge_ws_bytes(int64_t n);
lsq_status launch_judge(const double* Rs, int64_t n, int64_t ldr, int prec, int32_t* accept, double* kappa1, void* ws,
                        size_t ws_bytes, cudaStream_t st);
lsq_status launch_condest(const double* A, int64_t m, int64_t n, int64_t lda, double* kappa0, int32_t* chosen,
                          void* ws, size_t ws_bytes, int num_sms, cudaStream_t st);

int device_sm_count();

}  // namespace lsq
