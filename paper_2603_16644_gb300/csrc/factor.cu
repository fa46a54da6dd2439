// n x n factorizations and vector triangular solves for Eqs. e_pne / e_hpne:
//   - blocked right-looking Cholesky G = L L^T (FP64 for PNE; FP32 for the
//     condition estimate of Sec. 6.1): diagonal block in shared memory, panel
//     solve one thread per row, trailing update as an FP64-accurate
//     tensor-core product (FP64 with workspace) or a register-tiled rank-nb
//     product on the CUDA cores;
//   - blocked right-looking LU with partial pivoting (first largest |pivot|,
//     as LAPACK's getrf) for HPNE;
//   - triangular solves L y = c, L^T y = c, U y = c, unit L y = c as a
//     wavefront over 32-row blocks, one CTA each.
// A device status word (info) is written on breakdown; every later kernel of
// the same factorization and the solves return early once it is set.
#include "common.cuh"
#include "kernels.cuh"
#include "trsv_block.cuh"

#include <algorithm>
#include <type_traits>

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
// 1 / sqrt(d) for d > 0.  FP64: an FP32 estimate (the operand and the
// estimate moved between FP64 and FP32 with integer operations on the bit
// patterns, no conversion instruction) refined by one third-order step
//   e = 1 - d y^2,  y <- y + y e (1/2 + 3/8 e)
// (from ~23 correct bits to beyond FP64 precision): four dependent FP64
// operations, since each costs about a hundred cycles of latency on this part
// and the pivots form the factorization's critical path.  Relative error a
// few units in the last place.
template <typename T>
__device__ __forceinline__ T rsqrt_pivot(T d) {
    if constexpr (sizeof(T) == 4) {
        return (T)1 / sqrtf(d);
    } else {
        if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
        const unsigned long long b = (unsigned long long)__double_as_longlong(d);
        // d in the FP32 normal range: rebias the exponent, keep 23 bits of the significand
        const uint32_t fb = (uint32_t)((((b >> 52) & 0x7ff) - 1023 + 127) << 23) | (uint32_t)((b >> 29) & 0x7fffff);
        const uint32_t yb = __float_as_uint(rsqrtf(__uint_as_float(fb)));
        double y = __longlong_as_double((long long)(((unsigned long long)(((yb >> 23) & 0xff) - 127 + 1023) << 52) |
                                                    ((unsigned long long)(yb & 0x7fffff) << 29)));
        const double t = d * y;
        const double e = fma(-t, y, 1.0);
        const double c = fma(0.375, e, 0.5);
        const double ye = y * e;
        y = fma(ye, c, y);
        return y;
    }
}

// Diagonal block (CNB x CNB) in one CTA, right-looking.  Per column j the
// column is scaled by r_j = 1/sqrt(d_j) into a separate buffer; then thread 0
// applies column j's update to the next diagonal entry and forms the next
// pivot (L_jj = d r, r = 1/sqrt(d)) while the six warps of the other three
// schedulers (warps 1-3, 5-7) update the rest of the active triangle
// j < c <= r (row-major enumeration from a table, so that every warp issues
// full-width FP64 instructions): the pivot's dependent FP64 chain runs on a
// scheduler whose FP64 pipe the update leaves idle, overlapping the update.
template <typename T>
__global__ void __launch_bounds__(256) k_potrf_diag(T* __restrict__ G, int64_t ld, int64_t n, int64_t k0,
                                                    int32_t* __restrict__ info) {
    if (*info != 0) return;
    __shared__ T D[CNB][CNB + 1];
    __shared__ T colj[CNB];
    __shared__ uint16_t tri[CNB * (CNB - 1) / 2];  // e -> (rr << 8) | cc, lower triangle by rows
    __shared__ T rj;
    __shared__ int bad;
    const int nb = (int)min64(CNB, n - k0);
    const int tid = threadIdx.x;
    {
        // all loads of the block in flight before the stores
        T x[CNB * CNB / 256];
#pragma unroll
        for (int u = 0; u < CNB * CNB / 256; ++u) {
            const int q = tid + 256 * u, r = q & 63, c = q >> 6;
            x[u] = (r < nb && c < nb) ? G[(k0 + r) + (k0 + c) * ld] : (T)0;
        }
#pragma unroll
        for (int u = 0; u < CNB * CNB / 256; ++u) {
            const int q = tid + 256 * u;
            D[q & 63][q >> 6] = x[u];
        }
    }
    for (int e = tid; e < CNB * (CNB - 1) / 2; e += 256) {
        int rr = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
        while ((rr + 1) * (rr + 2) / 2 <= e) ++rr;
        while (rr * (rr + 1) / 2 > e) --rr;
        tri[e] = (uint16_t)((rr << 8) | (e - rr * (rr + 1) / 2));
    }
    __syncthreads();
    if (tid == 0) {
        bad = 0;
        const T d = D[0][0];
        if (!(d > (T)0) || !isfinite(d)) {
            bad = 1;
        } else {
            const T r = rsqrt_pivot<T>(d);
            rj = r;
            D[0][0] = d * r;
        }
    }
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        if (bad) break;
        const T r = rj;
        if (tid > j && tid < nb) {
            const T l = D[tid][j] * r;
            D[tid][j] = l;
            colj[tid] = l;
        }
        __syncthreads();
        if (j + 1 < nb) {
            if (tid == 0) {
                const T d = fma(-colj[j + 1], colj[j + 1], D[j + 1][j + 1]);
                if (!(d > (T)0) || !isfinite(d)) {
                    bad = j + 2;
                } else {
                    const T rn = rsqrt_pivot<T>(d);
                    rj = rn;
                    D[j + 1][j + 1] = d * rn;
                }
            } else if ((tid >> 5) & 3) {
                // entries 1 .. E-1 of the active triangle (entry 0 is the next
                // pivot), over warps 1-3 and 5-7
                const int w = tid >> 5;
                const int widx = (w - 1 - (w > 4 ? 1 : 0)) * 32 + (tid & 31);  // 0 .. 191
                const int a = nb - 1 - j;
                const int E = a * (a + 1) / 2;
                for (int e = widx + 1; e < E; e += 192) {
                    const int rc = tri[e];
                    const int rr = j + 1 + (rc >> 8), cc = j + 1 + (rc & 255);
                    D[rr][cc] = fma(-colj[rr], colj[cc], D[rr][cc]);
                }
            }
        }
        __syncthreads();
    }
    if (bad) {
        if (tid == 0) set_info_once(info, (int32_t)(k0 + bad));
        return;
    }
    for (int q = tid; q < CNB * CNB; q += 256) {
        const int r = q & 63, c = q >> 6;
        if (r < nb && c < nb) G[(k0 + r) + (k0 + c) * ld] = r >= c ? D[r][c] : (T)0;
    }
}

// L21 = G21 L11^{-T}, right-looking with reciprocal pivots.  16 threads per
// row (2 rows per warp), thread `sub` owning columns sub, sub+16, sub+32,
// sub+48 in registers; x_j is broadcast within the half-warp by a shuffle.
template <typename T>
__global__ void __launch_bounds__(128) k_potrf_panel(T* __restrict__ G, int64_t ld, int64_t n, int64_t k0,
                                                     const int32_t* __restrict__ info) {
    if (*info != 0) return;
    __shared__ T L11[CNB][CNB + 1];
    __shared__ T rinv[CNB];
    for (int q = threadIdx.x; q < CNB * CNB; q += 128) {
        int r = q & 63, c = q >> 6;
        L11[r][c] = G[(k0 + r) + (k0 + c) * ld];
    }
    __syncthreads();
    for (int j = threadIdx.x; j < CNB; j += 128) rinv[j] = (T)1 / L11[j][j];
    __syncthreads();
    const int lane = threadIdx.x & 31, sub = lane & 15;
    const int64_t i = k0 + CNB + (int64_t)blockIdx.x * 8 + (threadIdx.x >> 4);
    const bool live = i < n;
    T x[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) x[q] = live ? G[i + (k0 + sub + 16 * q) * ld] : (T)0;
#pragma unroll
    for (int j = 0; j < CNB; ++j) {
        const int qj = j >> 4, sj = j & 15;
        if (sub == sj) x[qj] = x[qj] * rinv[j];
        const T xj = __shfl_sync(0xffffffffu, x[qj], (lane & 16) | sj);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = sub + 16 * q;
            if (k > j) x[q] = fma(-xj, L11[k][j], x[q]);
        }
    }
    if (live) {
#pragma unroll
        for (int q = 0; q < 4; ++q) G[i + (k0 + sub + 16 * q) * ld] = x[q];
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

size_t cholesky_ws_bytes(int64_t n) { return n > CNB ? ot_update_ws_bytes(n - CNB, n - CNB, CNB) : 256; }

template <typename T>
lsq_status launch_cholesky(T* G, int64_t n, int64_t ld, int32_t* info, cudaStream_t st, void* ws, size_t ws_bytes) {
    for (int64_t k0 = 0; k0 < n; k0 += CNB) {
        int nb = (int)std::min<int64_t>(CNB, n - k0);
        k_potrf_diag<T><<<1, 256, 0, st>>>(G, ld, n, k0, info);
        LSQ_LAUNCH_CHECK();
        int64_t rest = n - k0 - nb;
        if (rest <= 0) break;
        k_potrf_panel<T><<<(unsigned)ceil_div(rest, 8), 128, 0, st>>>(G, ld, n, k0, info);
        LSQ_LAUNCH_CHECK();
        T* L21 = G + (k0 + nb) + k0 * ld;
        T* A22 = G + (k0 + nb) + (k0 + nb) * ld;
        lsq_status s;
        if constexpr (std::is_same<T, double>::value) {
            // A22 -= L21 L21^T on the tensor cores (FP64 accuracy; the upper
            // triangle of A22 is updated too and cleared at the end)
            if (ws && ws_bytes >= ot_update_ws_bytes(rest, rest, nb) && ot_trsm_supported()) {
                s = ot_gemm_update(L21, ld, L21, ld, 1, A22, ld, A22, ld, rest, rest, nb, ws, ws_bytes, nullptr, st);
                if (s != LSQ_OK) return s;
                continue;
            }
        }
        s = rank_update_ext<T>(A22, ld, L21, 1, ld, L21, 1, ld, rest, rest, nb, true, info, st);
        if (s != LSQ_OK) return s;
    }
    k_zero_upper<T><<<(unsigned)std::min<int64_t>(ceil_div(n * n, 256), 4096), 256, 0, st>>>(G, n, ld, info);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

template lsq_status launch_cholesky<double>(double*, int64_t, int64_t, int32_t*, cudaStream_t, void*, size_t);
template lsq_status launch_cholesky<float>(float*, int64_t, int64_t, int32_t*, cudaStream_t, void*, size_t);

// ---------------------------------------------------------------------------
// LU with partial pivoting
// ---------------------------------------------------------------------------
// Panel columns [k0, k0+nb), rows [k0, rows), one block of 1024 threads.
template <typename T>
__global__ void __launch_bounds__(1024) k_lu_panel(T* __restrict__ H, int64_t ld, int64_t rows, int64_t k0, int nb,
                                                   int32_t* __restrict__ piv, int32_t* __restrict__ info) {
    __shared__ T wv[32];
    __shared__ int64_t wi[32];
    __shared__ int64_t pivrow;
    int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int jj = 0; jj < nb; ++jj) {
        int64_t j = k0 + jj;
        // pivot: largest |H[i][j]|, smallest i on ties
        T best = (T)-1;
        int64_t bi = rows;
        for (int64_t i = j + tid; i < rows; i += 1024) {
            T v = fabs(H[i + j * ld]);
            if (v > best) { best = v; bi = i; }
        }
        for (int off = 16; off > 0; off >>= 1) {
            T ov = __shfl_xor_sync(0xffffffffu, best, off);
            int64_t oi = __shfl_xor_sync(0xffffffffu, bi, off);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { wv[warp] = best; wi[warp] = bi; }
        __syncthreads();
        if (warp == 0) {
            best = wv[lane];
            bi = wi[lane];
            for (int off = 16; off > 0; off >>= 1) {
                T ov = __shfl_xor_sync(0xffffffffu, best, off);
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
                T t = H[j + (k0 + c) * ld];
                H[j + (k0 + c) * ld] = H[p + (k0 + c) * ld];
                H[p + (k0 + c) * ld] = t;
            }
        __syncthreads();
        T d = H[j + j * ld];
        bool zero = (d == (T)0) || !isfinite(d);
        if (zero) {
            if (tid == 0) set_info_once(info, (int32_t)(j + 1));
        } else {
            for (int64_t i = j + 1 + tid; i < rows; i += 1024) H[i + j * ld] = H[i + j * ld] / d;
        }
        __syncthreads();
        if (!zero) {
            for (int64_t i = j + 1 + tid; i < rows; i += 1024) {
                T l = H[i + j * ld];
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
template <typename T>
__global__ void k_lu_swap(T* __restrict__ H, int64_t ld, int64_t cols, int64_t k0, int nb,
                          const int32_t* __restrict__ piv) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols || (c >= k0 && c < k0 + nb)) return;
    for (int jj = 0; jj < nb; ++jj) {
        int64_t j = k0 + jj, p = piv[j];
        if (p != j) {
            T t = H[j + c * ld];
            H[j + c * ld] = H[p + c * ld];
            H[p + c * ld] = t;
        }
    }
}

// U12 = L11^{-1} A12 (unit lower L11), one thread per column right of the panel.
template <typename T>
__global__ void k_lu_u12(T* __restrict__ H, int64_t ld, int64_t cols, int64_t k0, int nb) {
    __shared__ T L11[LNB][LNB + 1];
    for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) {
        int i = q % nb, j = q / nb;
        L11[i][j] = H[(k0 + i) + (k0 + j) * ld];
    }
    __syncthreads();
    int64_t c = k0 + nb + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    T u[LNB];
    for (int i = 0; i < nb; ++i) u[i] = H[(k0 + i) + c * ld];
    for (int i = 0; i < nb; ++i) {
        T v = u[i];
        for (int k = 0; k < i; ++k) v = fma(-L11[i][k], u[k], v);
        u[i] = v;
    }
    for (int i = 0; i < nb; ++i) H[(k0 + i) + c * ld] = u[i];
}

// Blocked right-looking LU with partial pivoting of a rows x cols matrix
// (rows >= cols): P H = L U, L unit lower trapezoidal, U cols x cols upper.
template <typename T>
lsq_status launch_lu_rect(T* H, int64_t rows, int64_t cols, int64_t ld, int32_t* piv, int32_t* info, cudaStream_t st) {
    if (rows < cols) return LSQ_ERR_ARG;
    for (int64_t k0 = 0; k0 < cols; k0 += LNB) {
        int nb = (int)std::min<int64_t>(LNB, cols - k0);
        k_lu_panel<T><<<1, 1024, 0, st>>>(H, ld, rows, k0, nb, piv, info);
        LSQ_LAUNCH_CHECK();
        k_lu_swap<T><<<(unsigned)ceil_div(cols, 128), 128, 0, st>>>(H, ld, cols, k0, nb, piv);
        LSQ_LAUNCH_CHECK();
        int64_t rest = cols - k0 - nb, rrest = rows - k0 - nb;
        if (rest <= 0) continue;
        k_lu_u12<T><<<(unsigned)ceil_div(rest, 64), 64, 0, st>>>(H, ld, cols, k0, nb);
        LSQ_LAUNCH_CHECK();
        // A22 -= L21 U12:  P(i,k) = H[(k0+nb+i) + (k0+k) ld],  Q(j,k) = H[(k0+k) + (k0+nb+j) ld]
        lsq_status s = rank_update_ext<T>(H + (k0 + nb) + (k0 + nb) * ld, ld, H + (k0 + nb) + k0 * ld, 1, ld,
                                          H + k0 + (k0 + nb) * ld, ld, 1, rrest, rest, nb, false, nullptr, st);
        if (s != LSQ_OK) return s;
    }
    return LSQ_OK;
}

template lsq_status launch_lu_rect<float>(float*, int64_t, int64_t, int64_t, int32_t*, int32_t*, cudaStream_t);
template lsq_status launch_lu_rect<double>(double*, int64_t, int64_t, int64_t, int32_t*, int32_t*, cudaStream_t);

lsq_status launch_lu(double* H, int64_t n, int64_t ld, int32_t* piv, int32_t* info, cudaStream_t st) {
    return launch_lu_rect<double>(H, n, n, ld, piv, info, st);
}

// The sketch's LU preconditioner (not-normal equations): the tall LU of A_s
// (s x n, float or double) in T arithmetic, then U with the column scaling
// undone, U_s[:, j] = U[:, j] 2^-colexp[j], promoted to FP64 (upper
// triangle of Us written, ld ldu).
template <typename TS, typename T>
__global__ void k_lu_load(const TS* __restrict__ As, int64_t s, int64_t n, int64_t ldas, T* __restrict__ W) {
    const int64_t total = s * n;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q % s, j = q / s;
        W[q] = (T)As[i + j * ldas];
    }
}

template <typename T>
__global__ void k_lu_upper_out(const T* __restrict__ W, int64_t s, int64_t n, const int32_t* __restrict__ colexp,
                               double* __restrict__ Us, int64_t ldu) {
    const int64_t total = n * n;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q % n, j = q / n;
        if (i <= j) Us[i + j * ldu] = ldexp((double)W[i + j * s], colexp ? -colexp[j] : 0);
    }
}

size_t lu_precond_ws_bytes(int64_t s, int64_t n, int prec) {
    const size_t es = prec == LSQ_FP64 ? 8 : 4;
    return align_up(es * (size_t)s * n, 256) + align_up(sizeof(int32_t) * (size_t)n, 256) + 256;
}

lsq_status launch_lu_precond(const void* As, int64_t s, int64_t n, int64_t ldas, int as_prec, int lu_prec,
                             const int32_t* colexp, double* Us, int64_t ldu, int32_t* info, void* ws, size_t ws_bytes,
                             cudaStream_t st) {
    if (!ws || ws_bytes < lu_precond_ws_bytes(s, n, lu_prec)) return LSQ_ERR_NOMEM;
    const size_t es = lu_prec == LSQ_FP64 ? 8 : 4;
    char* base = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    int32_t* piv = (int32_t*)(base + align_up(es * (size_t)s * n, 256));
    const unsigned g = (unsigned)std::min<int64_t>(ceil_div(s * n, 256), 8192);
    const unsigned gu = (unsigned)std::min<int64_t>(ceil_div(n * n, 256), 8192);
    lsq_status r;
    if (lu_prec == LSQ_FP64) {
        double* W = (double*)base;
        if (as_prec == LSQ_FP64) k_lu_load<double, double><<<g, 256, 0, st>>>((const double*)As, s, n, ldas, W);
        else k_lu_load<float, double><<<g, 256, 0, st>>>((const float*)As, s, n, ldas, W);
        LSQ_LAUNCH_CHECK();
        if ((r = launch_lu_rect<double>(W, s, n, s, piv, info, st)) != LSQ_OK) return r;
        k_lu_upper_out<double><<<gu, 256, 0, st>>>(W, s, n, colexp, Us, ldu);
    } else {
        float* W = (float*)base;
        if (as_prec == LSQ_FP64) k_lu_load<double, float><<<g, 256, 0, st>>>((const double*)As, s, n, ldas, W);
        else k_lu_load<float, float><<<g, 256, 0, st>>>((const float*)As, s, n, ldas, W);
        LSQ_LAUNCH_CHECK();
        if ((r = launch_lu_rect<float>(W, s, n, s, piv, info, st)) != LSQ_OK) return r;
        k_lu_upper_out<float><<<gu, 256, 0, st>>>(W, s, n, colexp, Us, ldu);
    }
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

// ---------------------------------------------------------------------------
// Triangular solves on a vector, many CTAs in a wavefront.  CTA v takes its
// row block from an atomic counter (v-th CTA to start), so every block it
// waits for belongs to a CTA that has already started.  It stages each
// off-diagonal 32 x 32 block of the operator while the solution of that block
// is still being computed, waits for that solution (bounded: 2 s of
// %globaltimer unless a test shortened it, then -2 is recorded and NaN passed
// on), applies it, and finally solves its diagonal block and publishes y_b.
//
// Publication: the solution is also written to a scratch copy `pub` that the
// launch fills with all-ones bit patterns (a NaN that arithmetic does not
// produce; a computed value with that pattern is published as the default
// NaN).  A waiting CTA polls the 32 entries it needs directly, one lane each,
// so a block's solution reaches the next CTA in one trip through L2 (no flag,
// no fence).
//
// Diagonal block: staged before the first wait with its reciprocal pivots and
// the block's own right-hand side, rows scaled to a unit diagonal.  For the
// Cholesky factor (L and L^T) a CTA that has a block to wait for also forms
// the inverse of its diagonal block while it waits, and applies it as a
// product: a few dependent FP64 operations instead of a 32-step chain.  The
// explicit inverse adds an error of order u kappa(L_bb) |y_b|, below the
// u kappa(A_p)^2 that the normal equations carry; the other factors (R_s, the
// LU factors) keep the substitution.
// Partial sums are combined in a fixed order, so the result does not depend
// on timing.
// ---------------------------------------------------------------------------
template <typename T>
struct TrsvPub;
template <>
struct TrsvPub<double> {
    static __device__ __forceinline__ void put(double* p, double v) {
        unsigned long long b = (unsigned long long)__double_as_longlong(v);
        if (b == ~0ull) b = 0x7ff8000000000000ull;
        asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(b) : "memory");
    }
    // the entry, or false while it is unpublished
    static __device__ __forceinline__ bool get(const double* p, double& v) {
        unsigned long long b;
        asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(b) : "l"(p) : "memory");
        v = __longlong_as_double((long long)b);
        return b != ~0ull;
    }
};
template <>
struct TrsvPub<float> {
    static __device__ __forceinline__ void put(float* p, float v) {
        unsigned b = __float_as_uint(v);
        if (b == ~0u) b = 0x7fc00000u;
        asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(b) : "memory");
    }
    static __device__ __forceinline__ bool get(const float* p, float& v) {
        unsigned b;
        asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(b) : "l"(p) : "memory");
        v = __uint_as_float(b);
        return b != ~0u;
    }
};

template <typename T>
__global__ void __launch_bounds__(128) k_trsv_wave(int kind, const T* __restrict__ M, int64_t n, int64_t ld, T* y,
                                                   int32_t* sync, T* pub, const int32_t* __restrict__ info,
                                                   int32_t* __restrict__ err, uint64_t wait_ns) {
    if (info && *info != 0) return;
    __shared__ T blk[32][33];
    __shared__ T dgb[32][33];  // diagonal block, rows scaled to a unit diagonal (then its inverse, see below)
    __shared__ T xin[32][33];  // inverse of the scaled block
    __shared__ T part[4][32];
    __shared__ T yk[32];
    __shared__ T rin[32];
    __shared__ T wsh[32];
    __shared__ int vb, failed;
    const int tid = threadIdx.x, r = tid & 31, q = tid >> 5;
    const int nblk = (int)((n + 31) / 32);
    if (tid == 0) {
        vb = atomicAdd(&sync[0], 1) + 1;  // the counter starts at -1 (all-ones fill)
        failed = 0;
    }
    __syncthreads();
    const int v = vb;
    const bool forward = (kind == TB_LOWER || kind == TB_UNIT_LOWER || kind == TB_UPPER_T);
    const bool trans = (kind == TB_LOWER_T || kind == TB_UPPER_T);  // operator entry (i, j) = M[j + i ld]
    const bool unit = (kind == TB_UNIT_LOWER);
    const bool use_inv = (kind == TB_LOWER || kind == TB_LOWER_T) && v > 0;
    const int b = forward ? v : nblk - 1 - v;
    const int64_t b0 = (int64_t)b * 32;
    const int bs = (int)min64(32, n - b0);
    // everything that does not depend on other blocks, before the first wait:
    // the diagonal block, the reciprocal pivots and this block's right-hand side
    for (int e = tid; e < 1024; e += 128) {
        int rr, jj;
        if (trans) { jj = e & 31; rr = e >> 5; } else { rr = e & 31; jj = e >> 5; }
        T val = (T)0;
        if (rr < bs && jj < bs) val = trans ? M[(b0 + jj) + (b0 + rr) * ld] : M[(b0 + rr) + (b0 + jj) * ld];
        dgb[rr][jj] = val;
    }
    T vv = (tid < 32 && r < bs) ? y[b0 + r] : (T)0;
    __syncthreads();
    if (tid < 32) rin[r] = (r < bs && !unit) ? (T)1 / dgb[r][r] : (T)1;
    __syncthreads();
    for (int e = tid; e < 1024; e += 128) {
        const int rr = e & 31, jj = e >> 5;
        if (rr != jj) dgb[rr][jj] *= rin[rr];
        if (use_inv) xin[rr][jj] = rr == jj ? (T)1 : (T)0;
    }
    if (use_inv) {
        // X = D'^{-1} for the unit triangular D' (rows and columns in solve
        // order: ascending for L, descending for L^T), right-looking: after
        // step j, row j of X is final and updates the rows solved after it.
        __syncthreads();
        for (int j = 0; j < 31; ++j) {
            const int w = j + 1, cnt = (31 - j) * w;
            for (int e = tid; e < cnt; e += 128) {
                const int ro = j + 1 + e / w, co = e % w;  // solve-order row (> j) and column (<= j)
                const int jr = forward ? j : 31 - j, rr = forward ? ro : 31 - ro, cc = forward ? co : 31 - co;
                xin[rr][cc] = fma(-dgb[rr][jr], xin[jr][cc], xin[rr][cc]);
            }
            __syncthreads();
        }
        // y_b = X diag(rin) w: fold the pivots into the columns
        for (int e = tid; e < 1024; e += 128) {
            const int rr = e & 31, cc = e >> 5;
            dgb[rr][cc] = xin[rr][cc] * rin[cc];
        }
    }
    T acc0 = (T)0, acc1 = (T)0;
    for (int st = 0; st < v; ++st) {
        const int k = forward ? st : nblk - 1 - st;
        const int64_t k0 = (int64_t)k * 32;
        const int ks = (int)min64(32, n - k0);
        for (int e = tid; e < 1024; e += 128) {
            int rr, jj;
            if (trans) { jj = e & 31; rr = e >> 5; } else { rr = e & 31; jj = e >> 5; }
            T val = (T)0;
            if (rr < bs && jj < ks) val = trans ? M[(k0 + jj) + (b0 + rr) * ld] : M[(b0 + rr) + (k0 + jj) * ld];
            blk[rr][jj] = val;
        }
        if (tid < 32) {
            // poll the ks published entries of block k, one lane each
            T got = (T)0;
            bool have = r >= ks;
            bool timed_out = false;
            uint64_t t0;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
            for (;;) {
                if (!have) have = TrsvPub<T>::get(pub + k0 + r, got);
                if (__all_sync(0xffffffffu, have)) break;
                uint64_t t;  // lane 0's clock decides for the warp
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
                if (__shfl_sync(0xffffffffu, t - t0 > wait_ns ? 1 : 0, 0)) {
                    timed_out = true;
                    break;
                }
            }
            yk[r] = r < ks ? got : (T)0;
            if (timed_out && r == 0) failed = 1;
        }
        __syncthreads();
        if (failed) break;
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
            acc0 = fma(-blk[r][q * 8 + j], yk[q * 8 + j], acc0);
            acc1 = fma(-blk[r][q * 8 + j + 1], yk[q * 8 + j + 1], acc1);
        }
        __syncthreads();
    }
    part[q][r] = acc0 + acc1;
    __syncthreads();
    if (use_inv) {
        // w = c_b - sum of the applied blocks, then y_b = (X diag(rin)) w,
        // 8 columns per warp in two chains, the warps' parts summed pairwise
        if (tid < 32) wsh[r] = vv + ((part[0][r] + part[1][r]) + (part[2][r] + part[3][r]));
        __syncthreads();
        T s0 = (T)0, s1 = (T)0;
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
            s0 = fma(dgb[r][q * 8 + j], wsh[q * 8 + j], s0);
            s1 = fma(dgb[r][q * 8 + j + 1], wsh[q * 8 + j + 1], s1);
        }
        part[q][r] = s0 + s1;
        __syncthreads();
        if (tid < 32) vv = (part[0][r] + part[1][r]) + (part[2][r] + part[3][r]);
    }
    if (tid < 32) {
        const bool ok = !failed;
        if (!use_inv) {
            vv = vv + part[0][r] + part[1][r] + part[2][r] + part[3][r];
            vv = vv * rin[r];  // unit-diagonal system from here on
            if (forward) {
                for (int jj = 0; jj < bs; ++jj) {
                    const T vj = __shfl_sync(0xffffffffu, vv, jj);
                    if (r > jj && r < bs) vv = fma(-dgb[r][jj], vj, vv);
                }
            } else {
                for (int jj = bs - 1; jj >= 0; --jj) {
                    const T vj = __shfl_sync(0xffffffffu, vv, jj);
                    if (r < jj) vv = fma(-dgb[r][jj], vj, vv);
                }
            }
        }
        if (r < bs) {
            if (ok) y[b0 + r] = vv;
            // a failed block passes NaN on, so that the blocks after it do not wait
            TrsvPub<T>::put(pub + b0 + r, ok ? vv : (T)NAN);
        }
        if (!ok && r == 0) set_info_once(err, -2);
    }
}

// Scratch: the block counter, then the published copy of the solution (8-byte aligned).
size_t trsv_sync_ints(int64_t n) { return 2 + 2 * (size_t)n; }

// Bound of one wait for another block's solution (2 s; shorter only in tests).
static uint64_t g_trsv_wait_ns = 2000000000ull;

uint64_t set_trsv_wait_ns(uint64_t ns) {
    const uint64_t old = g_trsv_wait_ns;
    g_trsv_wait_ns = ns;
    return old;
}

template <typename T>
lsq_status launch_trsv(int kind, const T* M, int64_t n, int64_t ld, T* y, const int32_t* info, int32_t* sync,
                       int32_t* err, cudaStream_t st) {
    if (!sync || n <= 0 || n > (int64_t)1 << 30 || ((uintptr_t)sync % 8) != 0) return LSQ_ERR_ARG;
    int64_t nblk = ceil_div(n, 32);
    // all ones: the counter reads -1, every published entry is unset
    LSQ_CUDA_TRY(cudaMemsetAsync(sync, 0xff, sizeof(int32_t) * trsv_sync_ints(n), st));
    k_trsv_wave<T><<<(unsigned)nblk, 128, 0, st>>>(kind, M, n, ld, y, sync, (T*)(sync + 2), info, err,
                                                   g_trsv_wait_ns);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

template lsq_status launch_trsv<double>(int, const double*, int64_t, int64_t, double*, const int32_t*, int32_t*,
                                        int32_t*, cudaStream_t);
template lsq_status launch_trsv<float>(int, const float*, int64_t, int64_t, float*, const int32_t*, int32_t*, int32_t*,
                                       cudaStream_t);

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
