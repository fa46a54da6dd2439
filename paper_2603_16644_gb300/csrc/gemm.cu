// FP64 (and FP32-accumulated) dense contractions on CUDA cores:
//   - K-major split-K GEMM C = X^T Y, used for the Gram matrices of Eqs.
//     e_pne / e_hpne (X = A_p, Y = A_p or A; K = m), the FP32 Gram of the
//     condition estimate (Sec. 6.1) and the CUDA-core Gaussian sketch;
//   - the tall-skinny right triangular solve A_p = A R_s^{-1} (Alg. 1);
//   - GEMVs for the right-hand side A_p^T b and the refinement residual.
// On GB300 FP64 runs on CUDA cores only, at ~1/64 of the FP32 rate, so the
// FP64 kernels are bound by DFMA issue: the design goal is that every SM
// issues exactly the algorithmic DFMAs (no redundant work, balanced waves),
// not data reuse.
#include "common.cuh"
#include "kernels.cuh"

#include <algorithm>
#include <cmath>

namespace lsq {

int device_sm_count() {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

// ---------------------------------------------------------------------------
// Split-K GEMM on K-contiguous operands.  64x64 output tile, 256 threads,
// 4x4 register micro-tile per thread, BK = 32 staged through shared memory.
// ---------------------------------------------------------------------------
constexpr int GBM = 64, GBN = 64, GBK = 32;

__device__ __forceinline__ void tile_of(int64_t t, bool sym, int64_t tilesN, int64_t& ti, int64_t& tj) {
    if (!sym) {
        ti = t / tilesN;
        tj = t % tilesN;
        return;
    }
    // lower-triangular enumeration: t = ti*(ti+1)/2 + tj, 0 <= tj <= ti
    int64_t r = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    while (r * (r + 1) / 2 > t) --r;
    ti = r;
    tj = t - r * (r + 1) / 2;
}

template <typename TX, typename TY, typename TA>
__global__ void __launch_bounds__(256) k_gemm_kmajor(const TX* __restrict__ X, int64_t ldx, const TY* __restrict__ Y,
                                                     int64_t ldy, int64_t M, int64_t N, int64_t K, int64_t kchunk,
                                                     bool sym, int64_t tilesN, TA* __restrict__ out, int64_t ldo,
                                                     int64_t split_stride) {
    __shared__ TA Xs[GBK][GBM + 2];
    __shared__ TA Ys[GBK][GBN + 2];
    int64_t ti, tj;
    tile_of(blockIdx.x, sym, tilesN, ti, tj);
    int64_t i0 = ti * GBM, j0 = tj * GBN;
    int64_t kb = (int64_t)blockIdx.y * kchunk;
    int64_t ke = min(K, kb + kchunk);
    int tid = threadIdx.x;
    int tx = tid & 15, ty = tid >> 4;
    TA acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = (TA)0;
    int lr = tid >> 2;        // 0..63: row of the tile this thread loads
    int lk = (tid & 3) * 8;   // 8 consecutive k
    for (int64_t k0 = kb; k0 < ke; k0 += GBK) {
        {
            int64_t gi = i0 + lr;
            const TX* xp = X + gi * ldx + k0 + lk;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                int64_t gk = k0 + lk + q;
                Xs[lk + q][lr] = (gi < M && gk < ke) ? to_acc<TX, TA>(xp[q]) : (TA)0;
            }
            int64_t gj = j0 + lr;
            const TY* yp = Y + gj * ldy + k0 + lk;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                int64_t gk = k0 + lk + q;
                Ys[lk + q][lr] = (gj < N && gk < ke) ? to_acc<TY, TA>(yp[q]) : (TA)0;
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < GBK; ++k) {
            TA xa[4], yb[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) xa[a] = Xs[k][ty * 4 + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) yb[b] = Ys[k][tx * 4 + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(xa[a], yb[b], acc[a][b]);
        }
        __syncthreads();
    }
    TA* o = out + (int64_t)blockIdx.y * split_stride;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            int64_t gi = i0 + ty * 4 + a, gj = j0 + tx * 4 + b;
            if (gi < M && gj < N) o[gi + gj * ldo] = acc[a][b];
        }
}

// Fixed-order reduction of split partials (M x N each, ld M) into C (ld ldc);
// with sym, entries with i >= j are reduced and mirrored.
template <typename TA>
__global__ void k_reduce_splits(const TA* __restrict__ part, int splits, int64_t M, int64_t N, bool sym,
                                TA* __restrict__ C, int64_t ldc) {
    int64_t total = M * N;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = q % M, j = q / M;
        if (sym && i < j) continue;
        TA s = (TA)0;
        for (int z = 0; z < splits; ++z) s += part[(int64_t)z * total + q];
        C[i + j * ldc] = s;
        if (sym && i != j) C[j + i * ldc] = s;
    }
}

template <typename TA>
__global__ void k_mirror(TA* __restrict__ C, int64_t M, int64_t ldc) {
    int64_t total = M * M;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = q % M, j = q / M;
        if (i > j) C[j + i * ldc] = C[i + j * ldc];
    }
}

GemmPlan plan_gemm_kmajor(int64_t M, int64_t N, int64_t K, bool sym, int acc, int num_sms) {
    GemmPlan p;
    p.M = M;
    p.N = N;
    p.K = K;
    p.sym = sym;
    p.acc = acc;
    int64_t tm = ceil_div(M, GBM), tn = ceil_div(N, GBN);
    int64_t tiles = sym ? tm * (tm + 1) / 2 : tm * tn;
    // Choose the split count that fills whole waves best: resident slots =
    // SMs x 2 CTAs; each split must keep at least 512 k-steps of work.
    int64_t slots = (int64_t)num_sms * 2;
    int best = 1;
    double best_eff = -1.0;
    int64_t max_splits = std::max<int64_t>(1, std::min<int64_t>(64, K / 512));
    for (int sp = 1; sp <= max_splits; ++sp) {
        int64_t units = tiles * sp;
        double waves = (double)units / (double)slots;
        double eff = waves / std::ceil(waves);
        // prefer more parallelism until there is at least one full wave
        double score = eff * std::min(1.0, waves);
        if (score > best_eff + 1e-9) { best_eff = score; best = sp; }
    }
    p.splits = best;
    p.kchunk = ceil_div(ceil_div(K, best), GBK) * GBK;
    p.splits = (int)ceil_div(K, p.kchunk);
    if (p.splits < 1) p.splits = 1;
    return p;
}

size_t gemm_kmajor_ws_bytes(const GemmPlan& p) {
    size_t es = p.acc == LSQ_FP64 ? 8 : 4;
    return p.splits > 1 ? align_up((size_t)p.splits * (size_t)p.M * (size_t)p.N * es, 256) : 0;
}

template <typename TX, typename TY, typename TA>
static lsq_status run_gemm(const GemmPlan& p, const void* X, int64_t ldx, const void* Y, int64_t ldy, void* C,
                           int64_t ldc, void* ws, cudaStream_t st) {
    int64_t tm = ceil_div(p.M, GBM), tn = ceil_div(p.N, GBN);
    int64_t tiles = p.sym ? tm * (tm + 1) / 2 : tm * tn;
    dim3 grid((unsigned)tiles, (unsigned)p.splits);
    if (p.splits == 1) {
        k_gemm_kmajor<TX, TY, TA><<<grid, 256, 0, st>>>((const TX*)X, ldx, (const TY*)Y, ldy, p.M, p.N, p.K, p.kchunk,
                                                        p.sym, tn, (TA*)C, ldc, 0);
        LSQ_LAUNCH_CHECK();
        if (p.sym) {
            k_mirror<TA><<<(unsigned)std::min<int64_t>(ceil_div(p.M * p.M, 256), 4096), 256, 0, st>>>((TA*)C, p.M, ldc);
            LSQ_LAUNCH_CHECK();
        }
        return LSQ_OK;
    }
    if (!ws) return LSQ_ERR_NOMEM;
    int64_t stride = p.M * p.N;
    k_gemm_kmajor<TX, TY, TA><<<grid, 256, 0, st>>>((const TX*)X, ldx, (const TY*)Y, ldy, p.M, p.N, p.K, p.kchunk,
                                                    p.sym, tn, (TA*)ws, p.M, stride);
    LSQ_LAUNCH_CHECK();
    k_reduce_splits<TA><<<(unsigned)std::min<int64_t>(ceil_div(stride, 256), 8192), 256, 0, st>>>(
        (const TA*)ws, p.splits, p.M, p.N, p.sym, (TA*)C, ldc);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

lsq_status launch_gemm_kmajor(const GemmPlan& p, const void* X, int xprec, int64_t ldx, const void* Y, int yprec,
                              int64_t ldy, void* C, int64_t ldc, void* ws, cudaStream_t st) {
    if (xprec != yprec) return LSQ_ERR_ARG;
    if (p.acc == LSQ_FP64) {
        if (xprec != LSQ_FP64) return LSQ_ERR_ARG;
        return run_gemm<double, double, double>(p, X, ldx, Y, ldy, C, ldc, ws, st);
    }
    switch (xprec) {
    case LSQ_FP8_E4M3: return run_gemm<__nv_fp8_storage_t, __nv_fp8_storage_t, float>(p, X, ldx, Y, ldy, C, ldc, ws, st);
    case LSQ_BF16: return run_gemm<__nv_bfloat16, __nv_bfloat16, float>(p, X, ldx, Y, ldy, C, ldc, ws, st);
    case LSQ_FP16: return run_gemm<__half, __half, float>(p, X, ldx, Y, ldy, C, ldc, ws, st);
    case LSQ_FP32: return run_gemm<float, float, float>(p, X, ldx, Y, ldy, C, ldc, ws, st);
    case LSQ_FP64: return run_gemm<double, double, float>(p, X, ldx, Y, ldy, C, ldc, ws, st);
    default: return LSQ_ERR_ARG;
    }
}

// ---------------------------------------------------------------------------
// A_p = A R^{-1}: each CTA owns TBM rows and sweeps the columns in blocks of
// TNB.  Block J: T = A[:, J] - A_p[:, <J] R[<J, J] (register-tiled update
// with A_p re-read from the CTA's own earlier output), then forward
// substitution with the diagonal block R[J, J] (one thread per row, R block
// in shared memory), then T is written to A_p.  Ragged rows and columns are
// masked; the padding of the last column block behaves as an identity.
// ---------------------------------------------------------------------------
constexpr int TBM = 64, TNB = 64, TBK = 16;

struct TrsmSmem {
    double T[TBM][TNB + 1];
    double Rd[TNB][TNB + 1];
    double Xs[TBK][TBM + 2];
    double Rs[TBK][TNB + 2];
};

__global__ void __launch_bounds__(256) k_trsm_right_upper(const double* __restrict__ A, int64_t m, int64_t n,
                                                          int64_t lda, const double* __restrict__ R, int64_t ldr,
                                                          double* __restrict__ Ap, int64_t ldap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrsmSmem& S = *reinterpret_cast<TrsmSmem*>(smem_raw);
    int64_t r0 = (int64_t)blockIdx.x * TBM;
    int tid = threadIdx.x;
    int tx = tid & 15, ty = tid >> 4;
    int64_t nblk = ceil_div_dev(n, TNB);
    for (int64_t J = 0; J < nblk; ++J) {
        int64_t c0 = J * TNB;
        int ncol = (int)min64(TNB, n - c0);
        // load T = A[rows, J] and the diagonal block of R
        for (int q = tid; q < TBM * TNB; q += 256) {
            int rr = q % TBM, cc = q / TBM;
            int64_t gi = r0 + rr;
            S.T[rr][cc] = (gi < m && cc < ncol) ? A[gi + (c0 + cc) * lda] : 0.0;
        }
        for (int q = tid; q < TNB * TNB; q += 256) {
            int kk = q % TNB, cc = q / TNB;
            double v;
            if (kk < ncol && cc < ncol) v = R[(c0 + kk) + (c0 + cc) * ldr];
            else v = (kk == cc) ? 1.0 : 0.0;
            S.Rd[kk][cc] = v;
        }
        // update with the already-solved columns: acc = A_p[:, <J] R[<J, J]
        double acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
        for (int64_t k0 = 0; k0 < c0; k0 += TBK) {
            __syncthreads();
            for (int q = tid; q < TBK * TBM; q += 256) {
                int rr = q % TBM, kk = q / TBM;
                int64_t gi = r0 + rr;
                S.Xs[kk][rr] = gi < m ? Ap[gi + (k0 + kk) * ldap] : 0.0;
            }
            for (int q = tid; q < TBK * TNB; q += 256) {
                int kk = q % TBK, cc = q / TBK;
                S.Rs[kk][cc] = cc < ncol ? R[(k0 + kk) + (c0 + cc) * ldr] : 0.0;
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < TBK; ++k) {
                double xa[4], rb[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) xa[a] = S.Xs[k][ty * 4 + a];
#pragma unroll
                for (int b = 0; b < 4; ++b) rb[b] = S.Rs[k][tx * 4 + b];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = fma(xa[a], rb[b], acc[a][b]);
            }
        }
        __syncthreads();
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) S.T[ty * 4 + a][tx * 4 + b] -= acc[a][b];
        __syncthreads();
        // forward substitution with R[J, J], one thread per row
        if (tid < TBM) {
            double* t = S.T[tid];
            for (int jj = 0; jj < TNB; ++jj) {
                double v = t[jj];
                for (int kk = 0; kk < jj; ++kk) v = fma(-t[kk], S.Rd[kk][jj], v);
                t[jj] = v / S.Rd[jj][jj];
            }
        }
        __syncthreads();
        for (int q = tid; q < TBM * TNB; q += 256) {
            int rr = q % TBM, cc = q / TBM;
            int64_t gi = r0 + rr;
            if (gi < m && cc < ncol) Ap[gi + (c0 + cc) * ldap] = S.T[rr][cc];
        }
        __syncthreads();
    }
}

lsq_status launch_trsm_right_upper(const double* A, int64_t m, int64_t n, int64_t lda, const double* R, int64_t ldr,
                                   double* Ap, int64_t ldap, cudaStream_t st) {
    size_t smem = sizeof(TrsmSmem);
    LSQ_CUDA_TRY(cudaFuncSetAttribute(k_trsm_right_upper, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_trsm_right_upper<<<(unsigned)ceil_div(m, TBM), 256, smem, st>>>(A, m, n, lda, R, ldr, Ap, ldap);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

// ---------------------------------------------------------------------------
// c = X^T v: block (p, chunk) reduces rows of one column chunk in a fixed
// tree; chunks are summed in order by k_gemv_finish.
// ---------------------------------------------------------------------------
constexpr int64_t GEMV_CHUNK = 16384;

__global__ void k_gemv_t_part(const double* __restrict__ X, int64_t m, int64_t ldx, const double* __restrict__ v,
                              double* __restrict__ part, int64_t n) {
    int64_t p = blockIdx.x;
    int64_t chunk = blockIdx.y;
    int64_t lo = chunk * GEMV_CHUNK, hi = min(m, lo + GEMV_CHUNK);
    const double* col = X + p * ldx;
    double s = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) s = fma(col[i], v[i], s);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    __shared__ double w[32];
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? w[threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (threadIdx.x == 0) part[chunk * n + p] = t;
    }
}

__global__ void k_gemv_finish(const double* __restrict__ part, int64_t chunks, int64_t n, double* __restrict__ c) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    double s = 0.0;
    for (int64_t q = 0; q < chunks; ++q) s += part[q * n + p];
    c[p] = s;
}

size_t gemv_t_ws_bytes(int64_t m, int64_t n) { return align_up(sizeof(double) * (size_t)ceil_div(m, GEMV_CHUNK) * n, 256); }

lsq_status launch_gemv_t(const double* X, int64_t m, int64_t n, int64_t ldx, const double* v, double* c,
                         double* partial, int64_t max_partial, cudaStream_t st) {
    int64_t chunks = ceil_div(m, GEMV_CHUNK);
    if (chunks * n > max_partial) return LSQ_ERR_NOMEM;
    k_gemv_t_part<<<dim3((unsigned)n, (unsigned)chunks), 256, 0, st>>>(X, m, ldx, v, partial, n);
    LSQ_LAUNCH_CHECK();
    k_gemv_finish<<<(unsigned)ceil_div(n, 128), 128, 0, st>>>(partial, chunks, n, c);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

// r = b - A x, one thread per row, x staged through shared memory.
__global__ void k_residual(const double* __restrict__ A, int64_t m, int64_t n, int64_t lda, const double* __restrict__ x,
                           const double* __restrict__ b, double* __restrict__ r) {
    __shared__ double xs[1024];
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double t = i < m ? b[i] : 0.0;
    for (int64_t c0 = 0; c0 < n; c0 += 1024) {
        int cnt = (int)min64(1024, n - c0);
        __syncthreads();
        for (int q = threadIdx.x; q < cnt; q += blockDim.x) xs[q] = x[c0 + q];
        __syncthreads();
        if (i < m)
            for (int q = 0; q < cnt; ++q) t = fma(-A[i + (c0 + q) * lda], xs[q], t);
    }
    if (i < m) r[i] = t;
}

lsq_status launch_residual(const double* A, int64_t m, int64_t n, int64_t lda, const double* x, const double* b,
                           double* r, cudaStream_t st) {
    k_residual<<<(unsigned)ceil_div(m, 128), 128, 0, st>>>(A, m, n, lda, x, b, r);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

__global__ void k_axpy1(double* __restrict__ x, const double* __restrict__ d, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = x[i] + d[i];
}

lsq_status launch_axpy1(double* x, const double* d, int64_t n, cudaStream_t st) {
    k_axpy1<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(x, d, n);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

}  // namespace lsq
