// Preconditioner of Alg. 1: thin QR of the sketch A_s (s x n) in FP32 or
// FP64 arithmetic, R only, then promotion to FP64 and removal of the
// column scaling.  Blocked Householder QR with the compact WY form
// (Schreiber & Van Loan 1989):
//   panel of QNB columns in one CTA (Householder vectors as in Golub & Van
//   Loan Alg. 5.1.1, which maps x to +||x|| e1, so diag(R) >= 0), the
//   triangular factor T of  H_1...H_nb = I - V T V^T, and the trailing update
//   C <- (I - V T^T V^T) C as two contractions (W = V^T C, C -= V (T^T W)).
#include "common.cuh"
#include "kernels.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>

namespace lsq {

constexpr int QNB = 32;        // panel width
constexpr int QPT = 512;       // panel threads

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red /* >= 32 */) {
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    T t = (T)0;
    for (int w = 0; w < nw; ++w) t += red[w];  // same order in every thread
    return t;
}

// Factor panel columns [k0, k0+nb) of W (s x n, ld), store v below the
// diagonal (v_j = 1 implicit), R on and above, beta[j]; then build T (nb x
// nb upper, ld QNB) and the explicit V (rows k0..s-1, ld ldv).
template <typename T>
__global__ void __launch_bounds__(QPT) k_qr_panel(T* __restrict__ W, int64_t ld, int64_t s, int64_t k0, int nb,
                                                  T* __restrict__ beta, T* __restrict__ Tm, T* __restrict__ V,
                                                  int64_t ldv) {
    __shared__ T red[32];
    __shared__ T wred[QPT / 32][QNB];
    __shared__ T wcol[QNB];
    __shared__ T sh_v1, sh_beta;
    __shared__ int sh_scale;
    __shared__ T Ys[QNB][QNB + 1];
    __shared__ T Vs[32][QNB + 1];
    __shared__ T Ts[QNB][QNB + 1];
    int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int jj = 0; jj < nb; ++jj) {
        int64_t j = k0 + jj;
        T* colj = W + j * ld;
        T sp = (T)0;
        for (int64_t i = j + 1 + tid; i < s; i += QPT) sp = fma(colj[i], colj[i], sp);
        T sigma = block_sum<T>(sp, red);
        if (tid == 0) {
            T x1 = colj[j];
            T mu, b, v1 = (T)1;
            int scale = 0;
            if (sigma == (T)0) {
                mu = fabs(x1);
                b = x1 >= (T)0 ? (T)0 : (T)2;
            } else {
                mu = sqrt(x1 * x1 + sigma);
                v1 = x1 <= (T)0 ? x1 - mu : -sigma / (x1 + mu);
                b = (T)2 * v1 * v1 / (sigma + v1 * v1);
                scale = 1;
            }
            colj[j] = mu;
            beta[j] = b;
            sh_v1 = v1;
            sh_beta = b;
            sh_scale = scale;
        }
        __syncthreads();
        T v1 = sh_v1, b = sh_beta;
        if (sh_scale)
            for (int64_t i = j + 1 + tid; i < s; i += QPT) colj[i] = colj[i] / v1;
        __syncthreads();
        int rem = nb - jj - 1;
        if (rem > 0 && b != (T)0) {
            T acc[QNB];
#pragma unroll
            for (int c = 0; c < QNB; ++c) acc[c] = (T)0;
            // w_c = W[j][c] + sum_{i>j} v_i W[i][c]
            for (int64_t i = j + tid; i < s; i += QPT) {
                T vi = (i == j) ? (T)1 : colj[i];
#pragma unroll
                for (int c = 0; c < QNB; ++c)
                    if (c < rem) acc[c] = fma(vi, W[i + (j + 1 + c) * ld], acc[c]);
            }
#pragma unroll
            for (int c = 0; c < QNB; ++c) {
                T v = acc[c];
                for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                if (lane == 0) wred[warp][c] = v;
            }
            __syncthreads();
            if (tid < rem) {
                T t = (T)0;
                for (int w = 0; w < QPT / 32; ++w) t += wred[w][tid];
                wcol[tid] = b * t;
            }
            __syncthreads();
            for (int64_t i = j + tid; i < s; i += QPT) {
                T vi = (i == j) ? (T)1 : colj[i];
                for (int c = 0; c < rem; ++c) {
                    T* p = &W[i + (j + 1 + c) * ld];
                    *p = fma(-wcol[c], vi, *p);
                }
            }
        }
        __syncthreads();
    }
    // Y = V^T V over rows k0..s-1 (explicit zeros above, ones on the diagonal)
    int p = tid >> 5, q = lane;  // 16 x 32 threads cover Y in two passes
    T y0 = (T)0, y1 = (T)0;
    for (int64_t r0 = k0; r0 < s; r0 += 32) {
        for (int e = tid; e < 32 * QNB; e += QPT) {
            int rr = e % 32, cc = e / 32;
            int64_t i = r0 + rr;
            T v = (T)0;
            if (cc < nb && i < s) {
                int64_t diag = k0 + cc;
                v = i < diag ? (T)0 : (i == diag ? (T)1 : W[i + diag * ld]);
            }
            Vs[rr][cc] = v;
        }
        __syncthreads();
#pragma unroll 8
        for (int rr = 0; rr < 32; ++rr) {
            y0 = fma(Vs[rr][p], Vs[rr][q], y0);
            y1 = fma(Vs[rr][p + 16], Vs[rr][q], y1);
        }
        // explicit V for the trailing contractions
        for (int e = tid; e < 32 * QNB; e += QPT) {
            int rr = e % 32, cc = e / 32;
            int64_t i = r0 + rr;
            if (i < s) V[(i - k0) + cc * ldv] = Vs[rr][cc];
        }
        __syncthreads();
    }
    Ys[p][q] = y0;
    Ys[p + 16][q] = y1;
    __syncthreads();
    // T: T[j][j] = beta_j, T[0:j, j] = -beta_j T[0:j, 0:j] Y[0:j, j]
    if (warp == 0) {
        for (int c = 0; c < QNB; ++c) Ts[lane][c] = (T)0;
        __syncwarp();
        for (int jj = 0; jj < nb; ++jj) {
            T bj = beta[k0 + jj];
            T t = (T)0;
            if (lane < jj)
                for (int qq = lane; qq < jj; ++qq) t = fma(Ts[lane][qq], Ys[qq][jj], t);
            __syncwarp();
            if (lane < jj) Ts[lane][jj] = -bj * t;
            if (lane == jj) Ts[jj][jj] = bj;
            __syncwarp();
        }
        for (int c = 0; c < QNB; ++c) Tm[lane + c * QNB] = Ts[lane][c];
    }
}

// Same panel factorization by a cluster of QCL CTAs that keep the panel in
// shared memory: CTA r owns rows [r R, (r+1) R) of the panel (local leading
// dimension Rp = R | 1, odd, so that lanes reading different columns of one
// row hit different banks).  Per column j each CTA computes, in one pass over
// its rows below the diagonal, sigma = sum x_i^2 and d_c = sum x_i a_c[i] for
// every later column c (warp = row group, lane = column); the partials and
// the diagonal row (x1, a_c[j], from its owner) are pushed into every CTA's
// shared memory, and after ONE cluster barrier every CTA sums them in rank
// order and gets identical Householder scalars and
//   v^T a_c = a_c[j] + d_c / v1,   w_c = beta v^T a_c
// (v = [1; x(2:)/v1]).  Slots alternate between two buffers by column parity:
// a CTA can only write a buffer again after the next barrier, which every CTA
// reaches after reading it.
constexpr int QCT = 256;

// QCL: CTAs per cluster (16, non-portable, where the device allows it; else
// 8).  Dynamic shared memory: the local panel (Rp x QNB) and, used by rank 0,
// the V^T V partials of every rank (QCL x QNB x (QNB + 1)).
template <typename T, int QCL>
__global__ void __launch_bounds__(QCT)
    k_qr_panel_cl(T* __restrict__ W, int64_t ld, int64_t s, int64_t k0, int nb, T* __restrict__ beta_out,
                  T* __restrict__ Tm, T* __restrict__ V, int64_t ldv) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char cl_raw[];
    T* P = reinterpret_cast<T*>(cl_raw);  // local panel, column-major, ld Rp
    __shared__ T all_part[2][QCL][QNB];  // per rank: d_c (sigma at c = j)
    __shared__ T all_row[2][QNB];        // the diagonal row: x1 at j, a_c[j] at c > j
    __shared__ T part[QCT / 32][QNB];
    __shared__ T wsh[QNB];
    __shared__ T Ts[QNB][QNB + 1];
    __shared__ T bsh[QNB];
    const int rank = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rows = (int)(s - k0);
    const int R = (rows + QCL - 1) / QCL;
    const int Rp = R | 1;
    const int r0 = rank * R;
    const int nloc = r0 < rows ? min(R, rows - r0) : 0;
    T* Yall = P + (int64_t)Rp * QNB;  // [QCL][QNB][QNB + 1], rank 0 only
    const int chunk = (R + (QCT / 32) - 1) / (QCT / 32);
    const int g0 = warp * chunk, g1 = min(nloc, g0 + chunk);  // this warp's rows
    for (int c = 0; c < QNB; ++c)
        for (int i = tid; i < R; i += QCT)
            P[c * Rp + i] = (i < nloc && c < nb) ? W[(k0 + r0 + i) + (k0 + c) * ld] : (T)0;
    __syncthreads();
    for (int jj = 0; jj < nb; ++jj) {
        const int buf = jj & 1;
        const int owner = (int)(jj / R);
        T* xj = P + jj * Rp;
        T* ac = P + lane * Rp;
        const int ib = max(jj + 1 - r0, 0);  // first owned row strictly below the diagonal
        T acc = (T)0;
        if (lane >= jj && lane < nb) {
            T a0 = (T)0, a1 = (T)0, a2 = (T)0, a3 = (T)0;
            int i = max(ib, g0);
            for (; i + 4 <= g1; i += 4) {
                a0 = fma(xj[i], ac[i], a0);
                a1 = fma(xj[i + 1], ac[i + 1], a1);
                a2 = fma(xj[i + 2], ac[i + 2], a2);
                a3 = fma(xj[i + 3], ac[i + 3], a3);
            }
            for (; i < g1; ++i) a0 = fma(xj[i], ac[i], a0);
            acc = (a0 + a1) + (a2 + a3);
        }
        part[warp][lane] = acc;
        __syncthreads();
        if (warp == 0) {
            T t = (T)0;
            for (int g = 0; g < QCT / 32; ++g) t += part[g][lane];
            for (int q = 0; q < QCL; ++q) *cluster.map_shared_rank(&all_part[buf][rank][lane], q) = t;
            if (rank == owner) {
                const T rv = P[lane * Rp + (jj - r0)];
                for (int q = 0; q < QCL; ++q) *cluster.map_shared_rank(&all_row[buf][lane], q) = rv;
            }
        }
        cluster.sync();
        T sigma = (T)0;
        for (int q = 0; q < QCL; ++q) sigma += all_part[buf][q][jj];
        const T x1 = all_row[buf][jj];
        T mu, b, v1 = (T)1;
        bool scale = false;
        if (sigma == (T)0) {
            mu = fabs(x1);
            b = x1 >= (T)0 ? (T)0 : (T)2;
        } else {
            mu = sqrt(x1 * x1 + sigma);
            v1 = x1 <= (T)0 ? x1 - mu : -sigma / (x1 + mu);
            b = (T)2 * v1 * v1 / (sigma + v1 * v1);
            scale = true;
        }
        if (warp == 0 && lane > jj && lane < nb) {
            T d = (T)0;
            for (int q = 0; q < QCL; ++q) d += all_part[buf][q][lane];
            wsh[lane] = b * (all_row[buf][lane] + (scale ? d / v1 : (T)0));
        }
        if (tid == 0) bsh[jj] = b;  // identical in every CTA of the cluster
        // v below the diagonal
        if (scale)
            for (int i = ib + tid; i < nloc; i += QCT) xj[i] = xj[i] / v1;
        __syncthreads();
        if (lane > jj && lane < nb && b != (T)0) {
            const T wc = wsh[lane];
            const int id = max(jj - r0, 0);  // owned rows >= the diagonal
            const int dr = jj - r0;           // local index of the diagonal row
            int i = max(id, g0);
            // blocks of 8 rows: all loads before the stores (the column of v and
            // the updated column never overlap)
            for (; i + 8 <= g1; i += 8) {
                T v[8], a[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    v[q] = (i + q == dr) ? (T)1 : xj[i + q];
                    a[q] = ac[i + q];
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) ac[i + q] = fma(-wc, v[q], a[q]);
            }
            for (; i < g1; ++i) {
                const T vi = (i == dr) ? (T)1 : xj[i];
                ac[i] = fma(-wc, vi, ac[i]);
            }
        }
        __syncthreads();
        if (rank == owner && tid == 0) {
            xj[jj - r0] = mu;
            beta_out[k0 + jj] = b;
        }
        __syncthreads();
    }
    // write R / v back to W and the explicit V (0 above, 1 on the diagonal)
    for (int c = 0; c < QNB; ++c)
        for (int i = tid; i < nloc; i += QCT) {
            const int64_t gi = r0 + i;
            if (c < nb) {
                const T pv = P[c * Rp + i];
                W[(k0 + gi) + (k0 + c) * ld] = pv;
                V[gi + c * ldv] = gi < c ? (T)0 : (gi == c ? (T)1 : pv);
            } else {
                V[gi + c * ldv] = (T)0;
            }
        }
    __syncthreads();
    // make the local panel the explicit V, then Y = V^T V over the owned rows
    for (int c = 0; c < nb; ++c)
        for (int i = tid; i < R && r0 + i <= c; i += QCT) P[c * Rp + i] = r0 + i == c ? (T)1 : (T)0;
    __syncthreads();
    {
        const int p = lane, q0 = warp * 4;  // Y[p][q0 .. q0 + 3]
        T y0 = (T)0, y1 = (T)0, y2 = (T)0, y3 = (T)0;
        const T* vp = P + p * Rp;
        const T* vq = P + q0 * Rp;
        for (int i = 0; i < nloc; ++i) {
            const T a = vp[i];
            y0 = fma(a, vq[i], y0);
            y1 = fma(a, vq[Rp + i], y1);
            y2 = fma(a, vq[2 * Rp + i], y2);
            y3 = fma(a, vq[3 * Rp + i], y3);
        }
        // into rank 0's shared memory (pushed, so that rank 0 sums locally)
        T* dst = cluster.map_shared_rank(Yall, 0) + (rank * QNB + p) * (QNB + 1);
        dst[q0] = y0;
        dst[q0 + 1] = y1;
        dst[q0 + 2] = y2;
        dst[q0 + 3] = y3;
    }
    cluster.sync();
    if (rank == 0) {
        for (int e = tid; e < QNB * QNB; e += QCT) {
            const int p = e % QNB, q = e / QNB;
            T y = (T)0;
            for (int r = 0; r < QCL; ++r) y += Yall[(r * QNB + p) * (QNB + 1) + q];
            Ts[p][q] = y;  // Ts holds Y for now
        }
        __syncthreads();
        if (warp == 0) {
            // column by column: T[0:j, j] = -beta_j T[0:j, 0:j] Y[0:j, j]; lane = row
            T trow[QNB];
#pragma unroll
            for (int jj = 0; jj < QNB; ++jj) {
                T t = (T)0;
#pragma unroll
                for (int qq = 0; qq < jj; ++qq) t = fma(trow[qq], Ts[qq][jj], t);
                const T bj = jj < nb ? bsh[jj] : (T)0;
                trow[jj] = lane < jj ? -bj * t : (lane == jj ? bj : (T)0);
            }
#pragma unroll
            for (int c = 0; c < QNB; ++c) Tm[lane + c * QNB] = trow[c];
        }
    }
    cluster.sync();
}

// W2 = T^T Wp  (nb x nt), T upper (ld QNB), Wp (nb x nt, ld nb).
template <typename T>
__global__ void k_qr_tw(const T* __restrict__ Tm, const T* __restrict__ Wp, int nb, int64_t nt, T* __restrict__ W2) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nb * nt) return;
    int p = (int)(q % nb);
    int64_t c = q / nb;
    T t = (T)0;
    for (int k = 0; k <= p; ++k) t = fma(Tm[k + p * QNB], Wp[k + c * nb], t);
    W2[p + c * nb] = t;
}

template <typename TI, typename T>
__global__ void k_qr_load(const TI* __restrict__ As, int64_t s, int64_t n, int64_t ldas, T* __restrict__ W) {
    int64_t total = s * n;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = q % s, j = q / s;
        W[q] = (T)As[i + j * ldas];
    }
}

template <typename T>
__global__ void k_qr_extract(const T* __restrict__ W, int64_t ld, int64_t n, const int32_t* __restrict__ colexp,
                             double* __restrict__ Rs, int64_t ldr) {
    int64_t total = n * n;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = q % n, j = q / n;
        if (i <= j) {
            double v = (double)W[i + j * ld];
            Rs[i + j * ldr] = colexp ? ldexp(v, -colexp[j]) : v;
        }
    }
}

__global__ void k_check_diag(const double* __restrict__ Rs, int64_t n, int64_t ldr, int32_t* __restrict__ info) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double d = Rs[j + j * ldr];
    if (!(d > 0.0) || !isfinite(d)) set_info_once(info, (int32_t)(j + 1));
}

template <typename T>
static size_t qr_cluster_smem(int64_t rows, int qcl) {
    return sizeof(T) * ((size_t)(ceil_div(rows, qcl) | 1) * QNB + (size_t)qcl * QNB * (QNB + 1));
}

// 16 CTAs per cluster where the device can schedule that with the panel's
// shared memory (non-portable size), else 8; 0 if neither fits (the
// single-CTA panel kernel then runs).  Decided once per precision and size.
template <typename T>
static int qr_cluster_size_query(int64_t s) {
    const size_t lim = 200 * 1024;
    for (int qcl : {16, 8}) {
        const size_t sm = qr_cluster_smem<T>(s, qcl);
        if (sm > lim) continue;
        auto kern = qcl == 16 ? k_qr_panel_cl<T, 16> : k_qr_panel_cl<T, 8>;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess ||
            (qcl > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
            cudaGetLastError();
            continue;
        }
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = qcl;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(qcl);
        cfg.blockDim = dim3(QCT);
        cfg.dynamicSmemBytes = sm;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) == cudaSuccess && nclusters >= 1) return qcl;
        cudaGetLastError();
    }
    return 0;
}

template <typename T>
static int qr_cluster_size(int64_t s) {
    static std::mutex mu;
    static int64_t last_s = -1;
    static int last_dev = -1, last_q = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (s != last_s || dev != last_dev) {
        last_q = qr_cluster_size_query<T>(s);
        last_s = s;
        last_dev = dev;
    }
    return last_q;
}

template <typename T>
static cudaError_t qr_launch_cluster(int qcl, size_t smem, cudaStream_t st, T* W, int64_t s, int64_t k0, int nb,
                                     T* beta, T* Tm, T* V, int64_t rows) {
    auto kern = qcl == 16 ? k_qr_panel_cl<T, 16> : k_qr_panel_cl<T, 8>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = qcl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(qcl);
    cfg.blockDim = dim3(QCT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, W, s, s, k0, nb, beta, Tm, V, rows);
}

// V and T are double-buffered by panel parity; the trailing update of a panel
// has its own scratch for the narrow part (the next panel's columns) and the
// wide part (the rest), which may run at the same time.
struct QrLayout {
    size_t w, beta, tm[2], v[2], wp[2], w2[2], gemm[2];
    size_t total;
};

static QrLayout qr_layout(int64_t s, int64_t n, int es, int num_sms) {
    QrLayout L;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    L.w = take((size_t)s * n * es);
    L.beta = take((size_t)n * es);
    for (int b = 0; b < 2; ++b) {
        L.tm[b] = take((size_t)QNB * QNB * es);
        L.v[b] = take((size_t)s * QNB * es);
        L.wp[b] = take((size_t)QNB * n * es);
        L.w2[b] = take((size_t)QNB * n * es);
        L.gemm[b] = take((size_t)64 * QNB * n * es + 256);  // at most 64 split partials of nb x nt
    }
    (void)num_sms;
    L.total = off;
    return L;
}

// C (rows x nt, ld s) <- (I - V T^T V^T) C, as W = V^T C, W2 = T^T W, C -= V W2.
template <typename T>
static lsq_status qr_apply(const T* V, const T* Tm, int nb, int64_t rows, T* C, int64_t s, int64_t nt, T* Wp, T* W2,
                           void* gws, int sms, cudaStream_t st) {
    if (nt <= 0) return LSQ_OK;
    const int accp = sizeof(T) == 8 ? LSQ_FP64 : LSQ_FP32;
    GemmPlan gp = plan_gemm_kmajor(nb, nt, rows, false, accp, sms);
    lsq_status r = launch_gemm_kmajor(gp, V, accp, rows, C, accp, s, Wp, nb, gws, st);
    if (r != LSQ_OK) return r;
    k_qr_tw<T><<<(unsigned)ceil_div(nb * nt, 256), 256, 0, st>>>(Tm, Wp, nb, nt, W2);
    LSQ_LAUNCH_CHECK();
    // C -= V W2:  P(i,p) = V[i + p rows],  Q(c,p) = W2[p + c nb]
    return rank_update_ext<T>(C, s, V, 1, rows, W2, nb, 1, rows, nt, nb, false, nullptr, st);
}

// Internal streams for the look-ahead QR (one pair per device): panels on a
// high-priority stream, the wide trailing updates on a low-priority one.
struct QrStreams {
    cudaStream_t hi = nullptr, lo = nullptr;
    bool ok = false;
};
static std::mutex g_qr_mu;

static QrStreams* qr_streams() {
    static QrStreams per_dev[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    QrStreams& q = per_dev[dev];
    if (!q.ok) {
        int lo_p = 0, hi_p = 0;
        if (cudaDeviceGetStreamPriorityRange(&lo_p, &hi_p) != cudaSuccess) return nullptr;
        if (cudaStreamCreateWithPriority(&q.hi, cudaStreamNonBlocking, hi_p) != cudaSuccess) return nullptr;
        if (cudaStreamCreateWithPriority(&q.lo, cudaStreamNonBlocking, lo_p) != cudaSuccess) return nullptr;
        q.ok = true;
    }
    return &q;
}

size_t qr_ws_bytes(int64_t s, int64_t n, int prec) {
    int es = prec == LSQ_FP64 ? 8 : 4;
    return qr_layout(s, n, es, device_sm_count()).total + 256;
}

template <typename T>
static lsq_status qr_run(const void* As, int64_t s, int64_t n, int64_t ldas, int as_prec, const int32_t* colexp,
                         double* Rs, int64_t ldr, int32_t* info, void* ws, size_t ws_bytes, cudaStream_t st) {
    int es = sizeof(T);
    int sms = device_sm_count();
    QrLayout L = qr_layout(s, n, es, sms);
    char* base = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    if (!ws || L.total + ((char*)base - (char*)ws) > ws_bytes) return LSQ_ERR_NOMEM;
    T* W = (T*)(base + L.w);
    T* beta = (T*)(base + L.beta);
    unsigned g = (unsigned)std::min<int64_t>(ceil_div(s * n, 256), 8192);
    if (as_prec == LSQ_FP64)
        k_qr_load<double, T><<<g, 256, 0, st>>>((const double*)As, s, n, ldas, W);
    else
        k_qr_load<float, T><<<g, 256, 0, st>>>((const float*)As, s, n, ldas, W);
    LSQ_LAUNCH_CHECK();
    // look-ahead: while panel k + 1 is factored (high-priority stream), the
    // wide part of panel k's trailing update runs on the low-priority stream;
    // the narrow part (the next panel's columns) goes first on the panel
    // stream.  Not while the caller's stream is being captured into a graph
    // (the batched solver), where concurrent problems must not share streams.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    LSQ_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
    QrStreams* qs = (cap == cudaStreamCaptureStatusNone && n > 2 * QNB) ? qr_streams() : nullptr;
    std::unique_lock<std::mutex> lk(g_qr_mu, std::defer_lock);
    cudaEvent_t ev_fork = nullptr, ev_p = nullptr, ev_w[2] = {nullptr, nullptr}, ev_join = nullptr;
    auto cleanup = [&]() {
        for (cudaEvent_t e : {ev_fork, ev_p, ev_w[0], ev_w[1], ev_join})
            if (e) cudaEventDestroy(e);
    };
    cudaStream_t sh = st, sl = st;
    if (qs) {
        lk.lock();
        bool good = cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming) == cudaSuccess &&
                    cudaEventCreateWithFlags(&ev_p, cudaEventDisableTiming) == cudaSuccess &&
                    cudaEventCreateWithFlags(&ev_w[0], cudaEventDisableTiming) == cudaSuccess &&
                    cudaEventCreateWithFlags(&ev_w[1], cudaEventDisableTiming) == cudaSuccess &&
                    cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming) == cudaSuccess &&
                    cudaEventRecord(ev_fork, st) == cudaSuccess && cudaStreamWaitEvent(qs->hi, ev_fork, 0) == cudaSuccess &&
                    cudaStreamWaitEvent(qs->lo, ev_fork, 0) == cudaSuccess;
        if (!good) {
            cleanup();
            return LSQ_ERR_CUDA;
        }
        sh = qs->hi;
        sl = qs->lo;
    }
    lsq_status r = LSQ_OK;
    const int qcl = qr_cluster_size<T>(s);
    int k = 0;
    for (int64_t k0 = 0; k0 < n && r == LSQ_OK; k0 += QNB, ++k) {
        const int b = k & 1;
        int nb = (int)std::min<int64_t>(QNB, n - k0);
        int64_t rows = s - k0;
        T* Tm = (T*)(base + L.tm[b]);
        T* V = (T*)(base + L.v[b]);
        const size_t clsm = qcl > 0 ? qr_cluster_smem<T>(rows, qcl) : 0;
        // Householder panel: sum over its columns of 4 (rows - j)(nb - j) flops
        double pflops = 0.0;
        for (int j = 0; j < nb; ++j) pflops += 4.0 * (double)(rows - j) * (double)(nb - j);
        stage_mark(ST_K_QRPANEL, true, sh);
        if (qcl > 0) {
            if (qr_launch_cluster<T>(qcl, clsm, sh, W, s, k0, nb, beta, Tm, V, rows) != cudaSuccess) {
                r = LSQ_ERR_CUDA;
                break;
            }
        } else {
            k_qr_panel<T><<<1, QPT, 0, sh>>>(W, s, s, k0, nb, beta, Tm, V, rows);
        }
        note_launch();
        if (cudaGetLastError() != cudaSuccess) {
            r = LSQ_ERR_CUDA;
            break;
        }
        stage_mark(ST_K_QRPANEL, false, sh, pflops);
        const int64_t nt = n - k0 - nb;
        if (nt <= 0) break;
        const int64_t nn = std::min<int64_t>(QNB, nt), nw = nt - nn;  // narrow / wide columns
        T* C = W + k0 + (k0 + nb) * s;
        if (qs) {
            // the wide part on the low-priority stream, after this panel
            if (cudaEventRecord(ev_p, sh) != cudaSuccess || cudaStreamWaitEvent(sl, ev_p, 0) != cudaSuccess) {
                r = LSQ_ERR_CUDA;
                break;
            }
            r = qr_apply<T>(V, Tm, nb, rows, C + nn * s, s, nw, (T*)(base + L.wp[1]), (T*)(base + L.w2[1]),
                            base + L.gemm[1], sms, sl);
            if (r != LSQ_OK || cudaEventRecord(ev_w[b], sl) != cudaSuccess) {
                r = r != LSQ_OK ? r : LSQ_ERR_CUDA;
                break;
            }
            // the next panel's columns also hold the previous panel's wide update
            if (k >= 1 && cudaStreamWaitEvent(sh, ev_w[b ^ 1], 0) != cudaSuccess) {
                r = LSQ_ERR_CUDA;
                break;
            }
            r = qr_apply<T>(V, Tm, nb, rows, C, s, nn, (T*)(base + L.wp[0]), (T*)(base + L.w2[0]),
                            base + L.gemm[0], sms, sh);
        } else {
            r = qr_apply<T>(V, Tm, nb, rows, C, s, nt, (T*)(base + L.wp[0]), (T*)(base + L.w2[0]),
                            base + L.gemm[0], sms, st);
        }
    }
    if (qs) {
        // join both internal streams back into the caller's stream
        bool good = cudaEventRecord(ev_join, sh) == cudaSuccess && cudaStreamWaitEvent(st, ev_join, 0) == cudaSuccess &&
                    cudaEventRecord(ev_fork, sl) == cudaSuccess && cudaStreamWaitEvent(st, ev_fork, 0) == cudaSuccess;
        cleanup();
        if (!good && r == LSQ_OK) r = LSQ_ERR_CUDA;
    }
    if (r != LSQ_OK) return r;
    k_qr_extract<T><<<(unsigned)std::min<int64_t>(ceil_div(n * n, 256), 4096), 256, 0, st>>>(W, s, n, colexp, Rs, ldr);
    LSQ_LAUNCH_CHECK();
    if (info) {
        k_check_diag<<<(unsigned)ceil_div(n, 128), 128, 0, st>>>(Rs, n, ldr, info);
        LSQ_LAUNCH_CHECK();
    }
    return LSQ_OK;
}

lsq_status launch_precond_qr(const void* As, int64_t s, int64_t n, int64_t ldas, int as_prec, int qr_prec,
                             const int32_t* colexp, double* Rs, int64_t ldr, int32_t* info, void* ws, size_t ws_bytes,
                             cudaStream_t st) {
    if (qr_prec == LSQ_FP64) return qr_run<double>(As, s, n, ldas, as_prec, colexp, Rs, ldr, info, ws, ws_bytes, st);
    return qr_run<float>(As, s, n, ldas, as_prec, colexp, Rs, ldr, info, ws, ws_bytes, st);
}

}  // namespace lsq
