// n x n factorizations and vector triangular solves for Eqs. e_pne / e_hpne:
//   - blocked right-looking Cholesky G = L L^T (FP64 for PNE; FP32 for the
//     condition estimate of Sec. 6.1): diagonal block in shared memory, panel
//     solve one thread per row, trailing update as a register-tiled rank-nb
//     product;
//   - blocked right-looking LU with partial pivoting (first largest |pivot|,
//     as LAPACK's getrf) for HPNE;
//   - blocked triangular solves L y = c, L^T y = c, U y = c, unit L y = c.
// A device status word (info) is written on breakdown; every later kernel of
// the same factorization and the solves return early once it is set.
#include "common.cuh"
#include "kernels.cuh"
#include "trsv_block.cuh"

#include <algorithm>

namespace lsq {

constexpr int CNB = 64;   // Cholesky block
constexpr int LNB = 32;   // LU panel width

// ---------------------------------------------------------------------------
// Generic register-tiled rank-K update  C(i, j) -= sum_k P(i, k) Q(j, k)
// with element strides; 64x64 tiles, K <= 64 staged once.  lower: only tiles
// with tile_i >= tile_j (and entries i >= j written).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_rank_update(T* __restrict__ C, int64_t ldc, const T* __restrict__ P,
                                                     int64_t psi, int64_t psk, const T* __restrict__ Q, int64_t qsj,
                                                     int64_t qsk, int64_t M, int64_t N, int K, bool lower,
                                                     int64_t tilesN, const int32_t* __restrict__ info) {
    if (info && *info != 0) return;
    __shared__ T Ps[32][64 + 1];
    __shared__ T Qs[32][64 + 1];
    int64_t t = blockIdx.x, ti, tj;
    if (lower) {
        int64_t r = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
        while ((r + 1) * (r + 2) / 2 <= t) ++r;
        while (r * (r + 1) / 2 > t) --r;
        ti = r;
        tj = t - r * (r + 1) / 2;
    } else {
        ti = t / tilesN;
        tj = t % tilesN;
    }
    int64_t i0 = ti * 64, j0 = tj * 64;
    int tid = threadIdx.x;
    int tx = tid & 15, ty = tid >> 4;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
    for (int kc = 0; kc < K; kc += 32) {
        int kn = min(32, K - kc);
        __syncthreads();
        for (int q = tid; q < 64 * 32; q += 256) {
            int r = q % 64, k = q / 64;
            int64_t gi = i0 + r, gj = j0 + r;
            bool kin = k < kn;
            Ps[k][r] = (kin && gi < M) ? P[gi * psi + (int64_t)(kc + k) * psk] : (T)0;
            Qs[k][r] = (kin && gj < N) ? Q[gj * qsj + (int64_t)(kc + k) * qsk] : (T)0;
        }
        __syncthreads();
        for (int k = 0; k < kn; ++k) {
            T pa[4], qb[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) pa[a] = Ps[k][ty * 4 + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) qb[b] = Qs[k][tx * 4 + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(pa[a], qb[b], acc[a][b]);
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            int64_t gi = i0 + ty * 4 + a, gj = j0 + tx * 4 + b;
            if (gi < M && gj < N && (!lower || gi >= gj)) C[gi + gj * ldc] -= acc[a][b];
        }
}

template <typename T>
lsq_status rank_update_ext(T* C, int64_t ldc, const T* P, int64_t psi, int64_t psk, const T* Q, int64_t qsj,
                              int64_t qsk, int64_t M, int64_t N, int K, bool lower, const int32_t* info,
                              cudaStream_t st) {
    if (M <= 0 || N <= 0 || K <= 0) return LSQ_OK;
    int64_t tm = ceil_div(M, 64), tn = ceil_div(N, 64);
    int64_t tiles = lower ? tm * (tm + 1) / 2 : tm * tn;
    k_rank_update<T><<<(unsigned)tiles, 256, 0, st>>>(C, ldc, P, psi, psk, Q, qsj, qsk, M, N, K, lower, tn, info);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

template lsq_status rank_update_ext<double>(double*, int64_t, const double*, int64_t, int64_t, const double*, int64_t,
                                           int64_t, int64_t, int64_t, int, bool, const int32_t*, cudaStream_t);
template lsq_status rank_update_ext<float>(float*, int64_t, const float*, int64_t, int64_t, const float*, int64_t,
                                          int64_t, int64_t, int64_t, int, bool, const int32_t*, cudaStream_t);

// ---------------------------------------------------------------------------
// Cholesky
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_potrf_diag(T* __restrict__ G, int64_t ld, int64_t n, int64_t k0,
                                                    int32_t* __restrict__ info) {
    if (*info != 0) return;
    __shared__ T D[CNB][CNB + 1];
    __shared__ int bad;
    int nb = (int)min64(CNB, n - k0);
    int tid = threadIdx.x;
    for (int q = tid; q < nb * nb; q += 256) {
        int i = q % nb, j = q / nb;
        D[i][j] = G[(k0 + i) + (k0 + j) * ld];
    }
    if (tid == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        if (tid == 0) {
            T d = D[j][j];
            if (!(d > (T)0) || !isfinite(d)) {
                bad = j + 1;
            } else {
                D[j][j] = sqrt(d);
            }
        }
        __syncthreads();
        if (bad) break;
        T piv = D[j][j];
        for (int i = j + 1 + tid; i < nb; i += 256) D[i][j] = D[i][j] / piv;
        __syncthreads();
        int rem = nb - j - 1;
        for (int q = tid; q < rem * rem; q += 256) {
            int i = j + 1 + q % rem, c = j + 1 + q / rem;
            if (i >= c) D[i][c] = fma(-D[i][j], D[c][j], D[i][c]);
        }
        __syncthreads();
    }
    if (bad) {
        if (tid == 0) set_info_once(info, (int32_t)(k0 + bad));
        return;
    }
    for (int q = tid; q < nb * nb; q += 256) {
        int i = q % nb, j = q / nb;
        G[(k0 + i) + (k0 + j) * ld] = i >= j ? D[i][j] : (T)0;
    }
}

// L21 = G21 L11^{-T}: one thread per row, 64 rows per block.
template <typename T>
__global__ void __launch_bounds__(64) k_potrf_panel(T* __restrict__ G, int64_t ld, int64_t n, int64_t k0,
                                                    const int32_t* __restrict__ info) {
    if (*info != 0) return;
    extern __shared__ __align__(16) unsigned char panel_raw[];
    T (*L11)[CNB + 1] = reinterpret_cast<T (*)[CNB + 1]>(panel_raw);
    T (*Row)[CNB + 1] = reinterpret_cast<T (*)[CNB + 1]>(panel_raw + sizeof(T) * CNB * (CNB + 1));
    int nb = (int)min64(CNB, n - k0);
    int tid = threadIdx.x;
    for (int q = tid; q < nb * nb; q += 64) {
        int i = q % nb, j = q / nb;
        L11[i][j] = G[(k0 + i) + (k0 + j) * ld];
    }
    int64_t r0 = k0 + nb + (int64_t)blockIdx.x * 64;
    for (int q = tid; q < 64 * nb; q += 64) {
        int rr = q % 64, c = q / 64;
        int64_t gi = r0 + rr;
        Row[rr][c] = gi < n ? G[gi + (k0 + c) * ld] : (T)0;
    }
    __syncthreads();
    T* x = Row[tid];
    for (int jj = 0; jj < nb; ++jj) {
        T v = x[jj];
        for (int kk = 0; kk < jj; ++kk) v = fma(-x[kk], L11[jj][kk], v);
        x[jj] = v / L11[jj][jj];
    }
    __syncthreads();
    for (int q = tid; q < 64 * nb; q += 64) {
        int rr = q % 64, c = q / 64;
        int64_t gi = r0 + rr;
        if (gi < n) G[gi + (k0 + c) * ld] = Row[rr][c];
    }
}

template <typename T>
__global__ void k_zero_upper(T* __restrict__ G, int64_t n, int64_t ld, const int32_t* __restrict__ info) {
    if (*info != 0) return;
    int64_t total = n * n;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = q % n, j = q / n;
        if (i < j) G[i + j * ld] = (T)0;
    }
}

template <typename T>
lsq_status launch_cholesky(T* G, int64_t n, int64_t ld, int32_t* info, cudaStream_t st) {
    for (int64_t k0 = 0; k0 < n; k0 += CNB) {
        int nb = (int)std::min<int64_t>(CNB, n - k0);
        k_potrf_diag<T><<<1, 256, 0, st>>>(G, ld, n, k0, info);
        LSQ_LAUNCH_CHECK();
        int64_t rest = n - k0 - nb;
        if (rest <= 0) break;
        size_t psm = sizeof(T) * (size_t)(CNB + 64) * (CNB + 1);
        LSQ_CUDA_TRY(cudaFuncSetAttribute(k_potrf_panel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm));
        k_potrf_panel<T><<<(unsigned)ceil_div(rest, 64), 64, psm, st>>>(G, ld, n, k0, info);
        LSQ_LAUNCH_CHECK();
        T* L21 = G + (k0 + nb) + k0 * ld;
        lsq_status s = rank_update_ext<T>(G + (k0 + nb) + (k0 + nb) * ld, ld, L21, 1, ld, L21, 1, ld, rest, rest, nb,
                                      true, info, st);
        if (s != LSQ_OK) return s;
    }
    k_zero_upper<T><<<(unsigned)std::min<int64_t>(ceil_div(n * n, 256), 4096), 256, 0, st>>>(G, n, ld, info);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

template lsq_status launch_cholesky<double>(double*, int64_t, int64_t, int32_t*, cudaStream_t);
template lsq_status launch_cholesky<float>(float*, int64_t, int64_t, int32_t*, cudaStream_t);

// ---------------------------------------------------------------------------
// LU with partial pivoting
// ---------------------------------------------------------------------------
// Panel columns [k0, k0+nb), rows [k0, n), one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_lu_panel(double* __restrict__ H, int64_t ld, int64_t n, int64_t k0, int nb,
                                                   int32_t* __restrict__ piv, int32_t* __restrict__ info) {
    __shared__ double wv[32];
    __shared__ int64_t wi[32];
    __shared__ int64_t pivrow;
    int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int jj = 0; jj < nb; ++jj) {
        int64_t j = k0 + jj;
        // pivot: largest |H[i][j]|, smallest i on ties
        double best = -1.0;
        int64_t bi = n;
        for (int64_t i = j + tid; i < n; i += 1024) {
            double v = fabs(H[i + j * ld]);
            if (v > best) { best = v; bi = i; }
        }
        for (int off = 16; off > 0; off >>= 1) {
            double ov = __shfl_xor_sync(0xffffffffu, best, off);
            int64_t oi = __shfl_xor_sync(0xffffffffu, bi, off);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { wv[warp] = best; wi[warp] = bi; }
        __syncthreads();
        if (warp == 0) {
            best = wv[lane];
            bi = wi[lane];
            for (int off = 16; off > 0; off >>= 1) {
                double ov = __shfl_xor_sync(0xffffffffu, best, off);
                int64_t oi = __shfl_xor_sync(0xffffffffu, bi, off);
                if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
            }
            if (lane == 0) {
                pivrow = bi;
                piv[j] = (int32_t)bi;
            }
        }
        __syncthreads();
        int64_t p = pivrow;
        if (p != j)
            for (int c = tid; c < nb; c += 1024) {
                double t = H[j + (k0 + c) * ld];
                H[j + (k0 + c) * ld] = H[p + (k0 + c) * ld];
                H[p + (k0 + c) * ld] = t;
            }
        __syncthreads();
        double d = H[j + j * ld];
        bool zero = (d == 0.0) || !isfinite(d);
        if (zero) {
            if (tid == 0) set_info_once(info, (int32_t)(j + 1));
        } else {
            for (int64_t i = j + 1 + tid; i < n; i += 1024) H[i + j * ld] = H[i + j * ld] / d;
        }
        __syncthreads();
        if (!zero) {
            for (int64_t i = j + 1 + tid; i < n; i += 1024) {
                double l = H[i + j * ld];
                for (int c = jj + 1; c < nb; ++c) {
                    int64_t col = k0 + c;
                    H[i + col * ld] = fma(-l, H[j + col * ld], H[i + col * ld]);
                }
            }
        }
        __syncthreads();
    }
}

// Apply the panel's row swaps (in order) to the columns outside the panel.
__global__ void k_lu_swap(double* __restrict__ H, int64_t ld, int64_t n, int64_t k0, int nb,
                          const int32_t* __restrict__ piv) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n || (c >= k0 && c < k0 + nb)) return;
    for (int jj = 0; jj < nb; ++jj) {
        int64_t j = k0 + jj, p = piv[j];
        if (p != j) {
            double t = H[j + c * ld];
            H[j + c * ld] = H[p + c * ld];
            H[p + c * ld] = t;
        }
    }
}

// U12 = L11^{-1} A12 (unit lower L11), one thread per column right of the panel.
__global__ void k_lu_u12(double* __restrict__ H, int64_t ld, int64_t n, int64_t k0, int nb) {
    __shared__ double L11[LNB][LNB + 1];
    for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) {
        int i = q % nb, j = q / nb;
        L11[i][j] = H[(k0 + i) + (k0 + j) * ld];
    }
    __syncthreads();
    int64_t c = k0 + nb + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    double u[LNB];
    for (int i = 0; i < nb; ++i) u[i] = H[(k0 + i) + c * ld];
    for (int i = 0; i < nb; ++i) {
        double v = u[i];
        for (int k = 0; k < i; ++k) v = fma(-L11[i][k], u[k], v);
        u[i] = v;
    }
    for (int i = 0; i < nb; ++i) H[(k0 + i) + c * ld] = u[i];
}

lsq_status launch_lu(double* H, int64_t n, int64_t ld, int32_t* piv, int32_t* info, cudaStream_t st) {
    for (int64_t k0 = 0; k0 < n; k0 += LNB) {
        int nb = (int)std::min<int64_t>(LNB, n - k0);
        k_lu_panel<<<1, 1024, 0, st>>>(H, ld, n, k0, nb, piv, info);
        LSQ_LAUNCH_CHECK();
        k_lu_swap<<<(unsigned)ceil_div(n, 128), 128, 0, st>>>(H, ld, n, k0, nb, piv);
        LSQ_LAUNCH_CHECK();
        int64_t rest = n - k0 - nb;
        if (rest <= 0) continue;
        k_lu_u12<<<(unsigned)ceil_div(rest, 64), 64, 0, st>>>(H, ld, n, k0, nb);
        LSQ_LAUNCH_CHECK();
        // A22 -= L21 U12:  P(i,k) = H[(k0+nb+i) + (k0+k) ld],  Q(j,k) = H[(k0+k) + (k0+nb+j) ld]
        lsq_status s = rank_update_ext<double>(H + (k0 + nb) + (k0 + nb) * ld, ld, H + (k0 + nb) + k0 * ld, 1, ld,
                                           H + k0 + (k0 + nb) * ld, ld, 1, rest, rest, nb, false, nullptr, st);
        if (s != LSQ_OK) return s;
    }
    return LSQ_OK;
}

// ---------------------------------------------------------------------------
// Triangular solves on a vector, single block, y staged in shared memory.
// Diagonal 32x32 blocks by one warp with shuffles, off-diagonal updates by
// all threads.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(512) k_trsv(int kind, const T* __restrict__ M, int64_t n, int64_t ld,
                                              T* __restrict__ y, const int32_t* __restrict__ info) {
    if (info && *info != 0) return;
    extern __shared__ __align__(16) unsigned char trsv_raw[];
    T* ys = reinterpret_cast<T*>(trsv_raw);
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) ys[i] = y[i];
    block_trsv<T>(kind, M, n, ld, ys);
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) y[i] = ys[i];
}

template <typename T>
lsq_status launch_trsv(int kind, const T* M, int64_t n, int64_t ld, T* y, const int32_t* info, cudaStream_t st) {
    size_t smem = sizeof(T) * (size_t)n;
    if (smem > 200 * 1024) return LSQ_ERR_ARG;
    if (smem > 48 * 1024) LSQ_CUDA_TRY(cudaFuncSetAttribute(k_trsv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_trsv<T><<<1, 512, smem, st>>>(kind, M, n, ld, y, info);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

template lsq_status launch_trsv<double>(int, const double*, int64_t, int64_t, double*, const int32_t*, cudaStream_t);
template lsq_status launch_trsv<float>(int, const float*, int64_t, int64_t, float*, const int32_t*, cudaStream_t);

__global__ void k_apply_piv(const int32_t* __restrict__ piv, int64_t n, double* __restrict__ y,
                            const int32_t* __restrict__ info) {
    if (info && *info != 0) return;
    for (int64_t k = 0; k < n; ++k) {
        int64_t p = piv[k];
        if (p != k) { double t = y[k]; y[k] = y[p]; y[p] = t; }
    }
}

lsq_status launch_apply_piv(const int32_t* piv, int64_t n, double* y, const int32_t* info, cudaStream_t st) {
    k_apply_piv<<<1, 1, 0, st>>>(piv, n, y, info);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

}  // namespace lsq
