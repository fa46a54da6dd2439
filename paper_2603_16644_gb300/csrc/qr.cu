// Preconditioner of Alg. 1: thin QR of the sketch A_s (s x n) in FP32 or
// FP64 arithmetic, R only, then promotion to FP64 and removal of the
// column scaling.  Blocked Householder QR with the compact WY form
// (Schreiber & Van Loan 1989):
//   panel of QNB columns in a cluster of CTAs (Householder vectors as in
//   Golub & Van Loan Alg. 5.1.1, which maps x to +||x|| e1, so diag(R) >= 0),
//   the triangular factor T of  H_1...H_nb = I - V T V^T, and the trailing
//   update C <- (I - V T^T V^T) C as W = V^T C, C -= V (T^T W) in one fused
//   cluster kernel.
#include "common.cuh"
#include "kernels.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

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
constexpr int QKG = QCT / 64;  // row groups of the previous-panel product (64 threads each)

constexpr int QRC = 32;  // panel rows per warp kept in registers

// 4 consecutive values from 16-byte aligned shared memory
__device__ __forceinline__ void load4(const float* p, float (&o)[4]) {
    const float4 v = *(const float4*)p;
    o[0] = v.x, o[1] = v.y, o[2] = v.z, o[3] = v.w;
}
__device__ __forceinline__ void load4(const double* p, double (&o)[4]) {
    const double2 v0 = *(const double2*)p, v1 = *(const double2*)(p + 2);
    o[0] = v0.x, o[1] = v0.y, o[2] = v1.x, o[3] = v1.y;
}

__device__ __forceinline__ void store4(float* p, float a, float b, float c, float d) { *(float4*)p = make_float4(a, b, c, d); }
__device__ __forceinline__ void store4(double* p, double a, double b, double c, double d) {
    *(double2*)p = make_double2(a, b);
    *(double2*)(p + 2) = make_double2(c, d);
}

// sum_{q < QCL} x[q * stride], pairwise (the same order in every CTA)
template <typename T, int QCL>
__device__ __forceinline__ T tree_sum(const T* x, int stride) {
    T v[QCL];
#pragma unroll
    for (int q = 0; q < QCL; ++q) v[q] = x[q * stride];
#pragma unroll
    for (int h = QCL / 2; h >= 1; h >>= 1)
#pragma unroll
        for (int q = 0; q < h; ++q) v[q] += v[q + h];
    return v[0];
}

// QCL: CTAs per cluster (16, non-portable, where the device allows it; else
// 8).  Dynamic shared memory: the local panel (Rp x QNB) and, in the fused
// form, the previous panel's reflector rows and the partial products behind it.
template <typename T, int QCL>
__global__ void __launch_bounds__(QCT)
    k_qr_panel_cl(T* __restrict__ W, int64_t ld, int64_t s, int64_t k0, int nb, T* __restrict__ beta_out,
                  T* __restrict__ Tm, T* __restrict__ V, int64_t ldv, const T* __restrict__ Vp, int64_t ldvp,
                  const T* __restrict__ Tp) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char cl_raw[];
    T* P = reinterpret_cast<T*>(cl_raw);  // local panel, column-major, ld Rp
    __shared__ T all_part[2][QCL][QNB];  // per rank: d_c (sigma at c = j)
    __shared__ T all_row[2][QNB];        // the diagonal row: x1 at j, a_c[j] at c > j
    __shared__ T part[QCT / 32][QNB];
    __shared__ T Ts[QNB][QNB + 1];
    __shared__ T bsh[QNB];
    __shared__ T Wr[QNB][QNB + 1];  // this CTA's partial V_p^T C (read by the whole cluster)
    __shared__ T Ysm[QNB][QNB + 1];  // rank 0: Y = V^T V (strictly upper part), built column by column
    __shared__ __align__(16) T bcv[QCT / 32][QRC];  // per warp: v_jj on its rows
    __shared__ __align__(16) T bcx[QCT / 32][QRC];  // per warp: x_{jj+1} below its diagonal
    __shared__ T rowbuf[QNB];                      // row jj of the panel (owning CTA)
    __shared__ T scal_sh[4];                       // FP64: mu, b, v1, 1 / v1 of the column (warp 0)
    __shared__ T wc_sh[QNB];                       // FP64: w_c of the column (warp 0)
    __shared__ int scale_sh;
    const int rank = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rows = (int)(s - k0);
    const int R = (rows + QCL - 1) / QCL;
    const int Rp = R | 1;
    const int r0 = rank * R;
    const int nloc = r0 < rows ? min(R, rows - r0) : 0;
    T* Yall = P + (int64_t)Rp * QNB;  // fused form only: the staging area behind the panel
    const int chunk = (R + (QCT / 32) - 1) / (QCT / 32);
    const int g0 = warp * chunk, g1 = min(nloc, g0 + chunk);  // this warp's rows
    // loads of all columns of a row in flight before the stores
    for (int i = tid; i < R; i += QCT) {
        T x[QNB];
#pragma unroll
        for (int c = 0; c < QNB; ++c) x[c] = (i < nloc && c < nb) ? W[(k0 + r0 + i) + (k0 + c) * ld] : (T)0;
#pragma unroll
        for (int c = 0; c < QNB; ++c) P[c * Rp + i] = x[c];
    }
    __syncthreads();
    // A CTA may write into another CTA's shared memory only once that CTA is
    // running: without a previous panel (below) the first column's exchange
    // is the first such write, so the cluster meets here first.
    if (Vp == nullptr) cluster.sync();
    if (Vp != nullptr) {
        // The previous panel's reflectors applied to this panel's columns,
        // C <- (I - V_p T_p^T V_p^T) C over rows k0 - QNB .. s - 1 (V_p: QNB
        // columns, ld ldvp, row 0 at k0 - QNB): this CTA's rows in shared
        // memory, the QNB rows above the panel by rank 0 from global memory.
        T* Vl = Yall;                      // [QNB][Rp]: rows QNB + r0 + i of V_p
        T* Wk = Yall + (int64_t)QNB * Rp;    // [QKG][QNB][QNB + 1] row-group partials, then W and W2
        T* Ct = Wk + QKG * QNB * (QNB + 1);  // rank 0: [QNB][QNB + 1] the rows above, then their V_p rows
        T* Vt = Ct + QNB * (QNB + 1);
        for (int i = tid; i < R; i += QCT) {
            T x[QNB];
#pragma unroll
            for (int c = 0; c < QNB; ++c) x[c] = i < nloc ? Vp[(QNB + r0 + i) + c * ldvp] : (T)0;
#pragma unroll
            for (int c = 0; c < QNB; ++c) Vl[c * Rp + i] = x[c];
        }
        if (rank == 0 && tid < QNB) {
            T x[QNB], v[QNB];
#pragma unroll
            for (int c = 0; c < QNB; ++c) {
                x[c] = c < nb ? W[(k0 - QNB + tid) + (k0 + c) * ld] : (T)0;
                v[c] = Vp[tid + c * ldvp];
            }
#pragma unroll
            for (int c = 0; c < QNB; ++c) {
                Ct[tid * (QNB + 1) + c] = x[c];
                Vt[tid * (QNB + 1) + c] = v[c];
            }
        }
        __syncthreads();
        {
            // partial W = V_p^T C: QKG row groups of 64 threads, 4 x 4 blocks
            const int kg = tid >> 6, tl = tid & 63, tp = tl & 7, tq = tl >> 3;
            const int span = (R + QKG - 1) / QKG;
            const int i0 = kg * span, i1 = min(nloc, i0 + span);
            T acc[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
            for (int i = i0; i < i1; ++i) {
                T v[4], c[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) v[a] = Vl[(4 * tp + a) * Rp + i];
#pragma unroll
                for (int b = 0; b < 4; ++b) c[b] = P[(4 * tq + b) * Rp + i];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = fma(v[a], c[b], acc[a][b]);
            }
            if (rank == 0 && kg == 0)
                for (int i = 0; i < QNB; ++i) {
                    T v[4], c[4];
#pragma unroll
                    for (int a = 0; a < 4; ++a) v[a] = Vt[i * (QNB + 1) + 4 * tp + a];
#pragma unroll
                    for (int b = 0; b < 4; ++b) c[b] = Ct[i * (QNB + 1) + 4 * tq + b];
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) acc[a][b] = fma(v[a], c[b], acc[a][b]);
                }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) Wk[(kg * QNB + 4 * tp + a) * (QNB + 1) + 4 * tq + b] = acc[a][b];
        }
        __syncthreads();
        for (int q = tid; q < QNB * QNB; q += QCT) {
            const int p = q >> 5, c = q & 31;
            Wr[p][c] = tree_sum<T, QKG>(&Wk[p * (QNB + 1) + c], QNB * (QNB + 1));
        }
        cluster.sync();
        // W: the partials of every rank in rank order (the column loop's
        // cluster barriers keep them in place until every CTA has read them)
        T* Wf = Wk;                     // [QNB][QNB + 1]
        T* W2 = Wk + QNB * (QNB + 1);   // [QNB][QNB]
        for (int q = tid; q < QNB * QNB; q += QCT) {
            const int p = q >> 5, c = q & 31;
            T v[QCL];
#pragma unroll
            for (int r = 0; r < QCL; ++r) v[r] = cluster.map_shared_rank(&Wr[0][0], r)[p * (QNB + 1) + c];
#pragma unroll
            for (int h = QCL / 2; h >= 1; h >>= 1)
#pragma unroll
                for (int r = 0; r < h; ++r) v[r] += v[r + h];
            Wf[p * (QNB + 1) + c] = v[0];
        }
        for (int q = tid; q < QNB * QNB; q += QCT) Ts[q & 31][q >> 5] = Tp[q];  // Ts[k][p] = T_p[k, p]
        __syncthreads();
        for (int q = tid; q < QNB * QNB; q += QCT) {
            const int p = q >> 5, c = q & 31;
            T w = (T)0;
            for (int kk = 0; kk <= p; ++kk) w = fma(Ts[kk][p], Wf[kk * (QNB + 1) + c], w);
            W2[p * QNB + c] = w;  // (T_p^T W)[p, c]
        }
        __syncthreads();
        // C -= V_p W2, one row per thread
        for (int i = tid; i < nloc; i += QCT) {
            T a[QNB];
#pragma unroll
            for (int c = 0; c < QNB; ++c) a[c] = P[c * Rp + i];
            for (int p = 0; p < QNB; ++p) {
                const T v = Vl[p * Rp + i];
#pragma unroll
                for (int c = 0; c < QNB; ++c) a[c] = fma(-v, W2[p * QNB + c], a[c]);
            }
#pragma unroll
            for (int c = 0; c < QNB; ++c) P[c * Rp + i] = a[c];
        }
        if (rank == 0 && tid < QNB) {
            const int64_t gi = k0 - QNB + tid;
            T a[QNB];
#pragma unroll
            for (int c = 0; c < QNB; ++c) a[c] = Ct[tid * (QNB + 1) + c];
            for (int p = 0; p < QNB; ++p) {
                const T v = Vt[tid * (QNB + 1) + p];
#pragma unroll
                for (int c = 0; c < QNB; ++c) a[c] = fma(-v, W2[p * QNB + c], a[c]);
            }
#pragma unroll
            for (int c = 0; c < QNB; ++c)
                if (c < nb) W[gi + (k0 + c) * ld] = a[c];
        }
        __syncthreads();
    }
    // partial dots of column j over this warp's rows strictly below row j
    // (lane = column c >= j): sum x_j[i] a_c[i]; sigma at c = j
    auto dots = [&](int j) -> T {
        if (!(lane >= j && lane < nb)) return (T)0;
        const T* x = P + j * Rp;
        const T* a = P + lane * Rp;
        T a0 = (T)0, a1 = (T)0, a2 = (T)0, a3 = (T)0;
        int i = max(max(j + 1 - r0, 0), g0);
        for (; i + 4 <= g1; i += 4) {
            a0 = fma(x[i], a[i], a0);
            a1 = fma(x[i + 1], a[i + 1], a1);
            a2 = fma(x[i + 2], a[i + 2], a2);
            a3 = fma(x[i + 3], a[i + 3], a3);
        }
        for (; i < g1; ++i) a0 = fma(x[i], a[i], a0);
        return (a0 + a1) + (a2 + a3);
    };
    // After column j: lanes c > j the partial dots of column j + 1 (rows
    // below j + 1), lanes i < j the partial Y[i][j] = v_i^T v_j = v_i[j] +
    // sum_{r > j} v_i[r] v_j[r] (rows of this warp) in the same pass: both
    // read one broadcast column (x_{j+1} or v_j) against the lane's own.
    auto dots_y = [&](int j) -> T {
        const int jn = j + 1;
        const bool ylane = lane < j, dlane = lane >= jn && lane < nb && jn < nb;
        if (!(ylane || dlane)) return (T)0;
        const T* x = P + (ylane ? j : jn) * Rp;
        const T* a = P + lane * Rp;
        T a0 = (T)0, a1 = (T)0, a2 = (T)0, a3 = (T)0;
        int i = max(max(jn + 1 - r0, 0), g0);
        for (; i + 4 <= g1; i += 4) {
            a0 = fma(x[i], a[i], a0);
            a1 = fma(x[i + 1], a[i + 1], a1);
            a2 = fma(x[i + 2], a[i + 2], a2);
            a3 = fma(x[i + 3], a[i + 3], a3);
        }
        for (; i < g1; ++i) a0 = fma(x[i], a[i], a0);
        T acc2 = (a0 + a1) + (a2 + a3);
        if (ylane) {
            const int lj = j - r0, lj1 = jn - r0;
            if (lj1 >= g0 && lj1 < g1) acc2 = fma(x[lj1], a[lj1], acc2);  // row j + 1
            if (lj >= g0 && lj < g1) acc2 += a[lj];                        // row j: v_j = 1 there
        }
        return acc2;
    };
    // Every per-row step (scaling of v, the update, the next column's dots)
    // stays within the warp's own rows, so a column needs one CTA barrier
    // (the partial dots) and one cluster barrier (their exchange), and for
    // FP64 a second CTA barrier (the scalars from warp 0).
    // Column jj's exchange: the partials of every warp summed (part), pushed
    // with the diagonal row (rowv, from the CTA that owns row jj) into every
    // CTA; after the cluster barrier every CTA forms the same Householder
    // scalars, w_c for each column and (rank 0) column jj - 1 of Y.
    struct Scal {
        T mu, b, v1, rv1, wc;
        bool scale;
    };
    // The Householder scalars of column jj from the exchanged partials (the
    // same in every CTA) and, per lane c > jj, w_c.
    auto scalars = [&](int jj, int buf, int owner) -> Scal {
        Scal sc;
        const T sigma = tree_sum<T, QCL>(&all_part[buf][0][jj], QNB);
        const T x1 = all_row[buf][jj];
        sc.v1 = (T)1;
        sc.rv1 = (T)1;
        sc.scale = false;
        if (sigma == (T)0) {
            sc.mu = fabs(x1);
            sc.b = x1 >= (T)0 ? (T)0 : (T)2;
        } else {
            sc.mu = sqrt(x1 * x1 + sigma);
            sc.v1 = x1 <= (T)0 ? x1 - sc.mu : -sigma / (x1 + sc.mu);
            sc.b = (T)2 * sc.v1 * sc.v1 / (sigma + sc.v1 * sc.v1);
            // v is scaled by a reciprocal formed here, in parallel with b
            // (an FP64 division costs ~650 cycles on this GPU)
            sc.rv1 = (T)1 / sc.v1;
            sc.scale = true;
        }
        // lane > jj: d_c of this column; lane < jj - 1: Y[lane][jj - 1] of the previous one
        const T dsum = tree_sum<T, QCL>(&all_part[buf][0][lane], QNB);
        sc.wc = (T)0;
        if (lane > jj && lane < nb) sc.wc = sc.b * (all_row[buf][lane] + (sc.scale ? dsum / sc.v1 : (T)0));
        if (rank == 0 && warp == 0 && lane + 1 < jj) Ysm[lane][jj - 1] = dsum;
        if (tid == 0) bsh[jj] = sc.b;  // identical in every CTA of the cluster
        if (rank == owner && tid == 0) beta_out[k0 + jj] = sc.b;
        return sc;
    };
    auto exchange = [&](int jj, T acc, const T* rowsrc, int rowstride) -> Scal {
        const int buf = jj & 1;
        const int owner = (int)(jj / R);
        part[warp][lane] = acc;
        __syncthreads();
        if (warp == 0) {
            const T t = tree_sum<T, QCT / 32>(&part[0][lane], QNB);
            for (int q = 0; q < QCL; ++q) *cluster.map_shared_rank(&all_part[buf][rank][lane], q) = t;
            if (rank == owner) {
                const T rv = rowsrc[lane * rowstride];
                for (int q = 0; q < QCL; ++q) *cluster.map_shared_rank(&all_row[buf][lane], q) = rv;
            }
        }
        cluster.sync();
        Scal sc;
        if constexpr (std::is_same<T, double>::value) {
            // FP64 instructions issue at a small fraction of the FP32 rate: the
            // scalars and the columns' w_c are formed once per CTA, by warp 0
            // (every warp forming them kept the FP64 pipe 73 % busy on a panel
            // of few rows), and read by the other warps from shared memory.
            if (warp == 0) {
                sc = scalars(jj, buf, owner);
                if (lane == 0) {
                    scal_sh[0] = sc.mu;
                    scal_sh[1] = sc.b;
                    scal_sh[2] = sc.v1;
                    scal_sh[3] = sc.rv1;
                    scale_sh = sc.scale ? 1 : 0;
                }
                wc_sh[lane] = sc.wc;
            }
            __syncthreads();
            sc.mu = scal_sh[0];
            sc.b = scal_sh[1];
            sc.v1 = scal_sh[2];
            sc.rv1 = scal_sh[3];
            sc.scale = scale_sh != 0;
            sc.wc = wc_sh[lane];
            return sc;
        }
        return scalars(jj, buf, owner);
    };
    T acc;
    if (std::is_same<T, double>::value && chunk <= QRC) {
        // FP64: each thread keeps its column's QRC rows of this warp in
        // registers; per column every lane of a warp takes the raw column jj
        // from lane jj and, after the update, column jj + 1 from lane jj + 1 by
        // shuffles, and forms v, the update and the next dots itself (no
        // divergent single-lane phases, no shared-memory round trips).
        // Measured: the FP64 path 6.2 -> 23.5 solves/s; for FP32 the
        // shared-memory form below is faster (3.07 against 4.55 ms per solve).
        // The loops run over QR = 8, 16 or 32 rows per lane, the fewest that
        // hold the warp's rows: FP64 instructions issue at a small fraction of
        // the FP32 rate on this GPU, so masked rows are not free (a 32-column
        // panel of ~1000 rows took 0.53 ms with 32 rows per lane).
        auto f64_cols = [&](auto qr_tag) {
            constexpr int QR = decltype(qr_tag)::value;
            T a[QR];
#pragma unroll
            for (int q = 0; q < QR; ++q) a[q] = g0 + q < g1 ? P[lane * Rp + g0 + q] : (T)0;
            const int gr0 = r0 + g0;  // global row (from k0) of a[0]
            const int nv = g1 - g0;   // valid rows of this warp (<= 0: none)
            auto row_of = [&](int row) -> T {
                T v = (T)0;
#pragma unroll
                for (int q = 0; q < QR; ++q)
                    if (gr0 + q == row && q < nv) v = a[q];
                return v;
            };
            // column c below row `row` on this warp's rows, from lane c
            T xn[QR];
            auto column_below = [&](int c, int row) {
#pragma unroll
                for (int q = 0; q < QR; ++q) {
                    const T x = __shfl_sync(0xffffffffu, a[q], c);
                    xn[q] = (q < nv && gr0 + q > row) ? x : (T)0;
                }
            };
            column_below(0, 0);
            if (0 >= gr0 && 0 < gr0 + nv) rowbuf[lane] = row_of(0);
            {
                T s4[4] = {(T)0, (T)0, (T)0, (T)0};  // 4 chains of 8 FMAs
#pragma unroll
                for (int q = 0; q < QR; ++q) s4[q & 3] = fma(xn[q], a[q], s4[q & 3]);
                acc = lane < nb ? (s4[0] + s4[1]) + (s4[2] + s4[3]) : (T)0;
            }
            for (int jj = 0; jj < nb; ++jj) {
                const Scal sc = exchange(jj, acc, rowbuf, 1);
                // v_jj on this warp's rows: 0 above row jj, 1 on it, x / v1 below
                T v[QR];
#pragma unroll
                for (int q = 0; q < QR; ++q) {
                    const T x = __shfl_sync(0xffffffffu, a[q], jj);
                    const int gr = gr0 + q;
                    v[q] = (gr < jj || q >= nv) ? (T)0 : (gr == jj ? (T)1 : (sc.scale ? x * sc.rv1 : x));
                }
                // lane jj: its column becomes v (R diagonal mu on row jj); later
                // columns: a_c -= w_c v
                const bool own = lane == jj, upd = lane > jj && lane < nb && sc.b != (T)0;
#pragma unroll
                for (int q = 0; q < QR; ++q) {
                    const int gr = gr0 + q;
                    const T ownv = (q < nv && gr > jj) ? v[q] : ((q < nv && gr == jj) ? sc.mu : a[q]);
                    a[q] = own ? ownv : (upd ? fma(-sc.wc, v[q], a[q]) : a[q]);
                }
                const int jn = jj + 1;
                if (jn < nb) {
                    column_below(jn, jn);
                    if (jn >= gr0 && jn < gr0 + nv) rowbuf[lane] = row_of(jn);
                }
                // lanes c > jj: dots of column jj + 1; lanes i < jj: Y[i][jj]
                const bool ylane = lane < jj, dlane = lane >= jn && lane < nb && jn < nb;
                T s4[4] = {(T)0, (T)0, (T)0, (T)0};
#pragma unroll
                for (int q = 0; q < QR; ++q) s4[q & 3] = fma(ylane ? v[q] : xn[q], a[q], s4[q & 3]);
                acc = (ylane || dlane) ? (s4[0] + s4[1]) + (s4[2] + s4[3]) : (T)0;
            }
#pragma unroll
            for (int q = 0; q < QR; ++q)
                if (q < nv) P[lane * Rp + g0 + q] = a[q];
        };
        if (chunk <= 8) f64_cols(std::integral_constant<int, 8>{});
        else if (chunk <= 16) f64_cols(std::integral_constant<int, 16>{});
        else f64_cols(std::integral_constant<int, QRC>{});
    } else if (chunk <= QRC) {
        // Each thread keeps its column's QRC rows of this warp in registers
        // (rows g0 + q); per column a warp broadcasts v_jj and x_{jj+1} through
        // its own QRC-entry shared buffers, read 4 rows per load.
        T a[QRC];
#pragma unroll
        for (int q = 0; q < QRC; ++q) a[q] = g0 + q < g1 ? P[lane * Rp + g0 + q] : (T)0;
        T* bv = &bcv[warp][0];
        T* bx = &bcx[warp][0];
        const int gr0 = r0 + g0;  // global row (from k0) of a[0]
        const int nv = g1 - g0;   // valid rows of this warp (<= 0: none)
        // the diagonal row value a_lane[row] of this warp (0 when not here)
        auto row_of = [&](int row) -> T {
            T v = (T)0;
#pragma unroll
            for (int q = 0; q < QRC; ++q)
                if (gr0 + q == row && q < nv) v = a[q];
            return v;
        };
        // x_0 below row 0, then the dots of column 0
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < QRC; q += 4) {
                T o[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) o[e] = (q + e < nv && gr0 + q + e > 0) ? a[q + e] : (T)0;
                store4(bx + q, o[0], o[1], o[2], o[3]);
            }
        }
        if (0 >= gr0 && 0 < gr0 + nv) rowbuf[lane] = row_of(0);
        __syncwarp();
        acc = (T)0;
        if (lane < nb) {
            T s4[4] = {(T)0, (T)0, (T)0, (T)0};  // 4 chains of 8 FMAs
#pragma unroll
            for (int q = 0; q < QRC; q += 4) {
                T xv[4];
                load4(bx + q, xv);
#pragma unroll
                for (int e = 0; e < 4; ++e) s4[e] = fma(xv[e], a[q + e], s4[e]);
            }
            acc = (s4[0] + s4[1]) + (s4[2] + s4[3]);
        }
        for (int jj = 0; jj < nb; ++jj) {
            // rowbuf (row jj, written by the warp that owns it) is read after
            // the CTA barrier inside the exchange
            const Scal sc = exchange(jj, acc, rowbuf, 1);
            // v_jj of this warp's rows: raw column from lane jj, scaled by all lanes
            if (lane == jj) {
#pragma unroll
                for (int q = 0; q < QRC; q += 4) store4(bv + q, a[q], a[q + 1], a[q + 2], a[q + 3]);
            }
            __syncwarp();
            if (lane < QRC) {  // lane = row of this warp here
                const int gr = gr0 + lane;
                const T x = bv[lane];
                bv[lane] = (gr < jj || lane >= nv) ? (T)0 : (gr == jj ? (T)1 : (sc.scale ? x * sc.rv1 : x));
            }
            __syncwarp();
            if (lane == jj) {
#pragma unroll
                for (int q = 0; q < QRC; q += 4) {
                    T vv[4];
                    load4(bv + q, vv);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if (q + e < nv && gr0 + q + e > jj) a[q + e] = vv[e];
                        if (q + e < nv && gr0 + q + e == jj) a[q + e] = sc.mu;  // R diagonal (v there is 1)
                    }
                }
            }
            if (lane > jj && lane < nb && sc.b != (T)0) {
#pragma unroll
                for (int q = 0; q < QRC; q += 4) {
                    T vv[4];
                    load4(bv + q, vv);
#pragma unroll
                    for (int e = 0; e < 4; ++e) a[q + e] = fma(-sc.wc, vv[e], a[q + e]);
                }
            }
            // x_{jj+1} below its diagonal and row jj + 1 for the next exchange
            const int jn = jj + 1;
            if (jn < nb) {
                if (lane == jn) {
#pragma unroll
                    for (int q = 0; q < QRC; q += 4) {
                        T o[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) o[e] = (q + e < nv && gr0 + q + e > jn) ? a[q + e] : (T)0;
                        store4(bx + q, o[0], o[1], o[2], o[3]);
                    }
                }
                if (jn >= gr0 && jn < gr0 + nv) rowbuf[lane] = row_of(jn);
            }
            __syncwarp();
            // lanes c > jj: dots of column jj + 1; lanes i < jj: Y[i][jj]
            const bool ylane = lane < jj, dlane = lane >= jn && lane < nb && jn < nb;
            acc = (T)0;
            if (ylane || dlane) {
                const T* src = ylane ? bv : bx;
                T s4[4] = {(T)0, (T)0, (T)0, (T)0};  // 4 chains of 8 FMAs
#pragma unroll
                for (int q = 0; q < QRC; q += 4) {
                    T xv[4];
                    load4(src + q, xv);
#pragma unroll
                    for (int e = 0; e < 4; ++e) s4[e] = fma(xv[e], a[q + e], s4[e]);
                }
                acc = (s4[0] + s4[1]) + (s4[2] + s4[3]);
            }
        }
#pragma unroll
        for (int q = 0; q < QRC; ++q)
            if (q < nv) P[lane * Rp + g0 + q] = a[q];
    } else {
        acc = dots(0);
        for (int jj = 0; jj < nb; ++jj) {
            T* xj = P + jj * Rp;
            T* ac = P + lane * Rp;
            const int owner = (int)(jj / R);
            const Scal sc = exchange(jj, acc, P + (jj - r0), Rp);
            const T b = sc.b, wc = sc.wc;
            if (rank == owner && tid == 0) xj[jj - r0] = sc.mu;  // the diagonal entry is not read again (v there is 1)
            // v below the diagonal, this warp's rows
            const int ib = max(jj + 1 - r0, 0);
            if (sc.scale)
                for (int i = max(ib, g0) + lane; i < g1; i += 32) xj[i] = xj[i] * sc.rv1;
            __syncwarp();
            if (lane > jj && lane < nb && b != (T)0) {
                const int id = max(jj - r0, 0);  // owned rows >= the diagonal
                const int dr = jj - r0;           // local index of the diagonal row
                int i = max(id, g0);
                // blocks of 8 rows: all loads before the stores (the column of v and
                // the updated column never overlap)
                for (; i + 8 <= g1; i += 8) {
                    T v[8], av[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        v[q] = (i + q == dr) ? (T)1 : xj[i + q];
                        av[q] = ac[i + q];
                    }
#pragma unroll
                    for (int q = 0; q < 8; ++q) ac[i + q] = fma(-wc, v[q], av[q]);
                }
                for (; i < g1; ++i) {
                    const T vi = (i == dr) ? (T)1 : xj[i];
                    ac[i] = fma(-wc, vi, ac[i]);
                }
            }
            __syncwarp();
            acc = dots_y(jj);
        }
    }
    // Y[:, nb - 1] of the last column: one more reduction, into rank 0
    part[warp][lane] = acc;
    __syncthreads();
    if (warp == 0) {
        const T t = tree_sum<T, QCT / 32>(&part[0][lane], QNB);
        *cluster.map_shared_rank(&all_part[nb & 1][rank][lane], 0) = t;
    }
    cluster.sync();
    if (rank == 0 && warp == 0 && lane + 1 < nb) Ysm[lane][nb - 1] = tree_sum<T, QCL>(&all_part[nb & 1][0][lane], QNB);
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
    if (rank == 0) {
        __syncthreads();
        if (warp == 0) {
            // column by column: T[0:j, j] = -beta_j T[0:j, 0:j] Y[0:j, j]; lane = row
            T trow[QNB];
#pragma unroll
            for (int jj = 0; jj < QNB; ++jj) {
                T t = (T)0;
                if (jj < nb)
#pragma unroll
                    for (int qq = 0; qq < jj; ++qq) t = fma(trow[qq], Ysm[qq][jj], t);
                const T bj = jj < nb ? bsh[jj] : (T)0;
                trow[jj] = lane < jj ? -bj * t : (lane == jj ? bj : (T)0);
            }
#pragma unroll
            for (int c = 0; c < QNB; ++c) Tm[lane + c * QNB] = trow[c];
        }
    }
}

// ---------------------------------------------------------------------------
// Trailing update C <- (I - V T^T V^T) C in one launch.  A cluster of QUC CTAs
// owns a block of 32 columns of C; its CTAs take the 128-row sub-tiles of the
// block in turn (rank, rank + QUC, ...).  Per CTA:
//   1. W_r = V^T C over its sub-tiles (32 x 32), four row groups of 64 threads
//      with 4 x 4 register tiles, summed in a fixed order;
//   2. W = sum_r W_r over the cluster (rank order, read through distributed
//      shared memory), W2 = T^T W (T upper, so W2[p] uses T[0..p][p]);
//   3. C -= V W2 over its sub-tiles, written back coalesced.
// Sub-tiles are staged in shared memory as [32 columns][128 rows] with the
// 4-element groups of a row XOR-swizzled by (column / 4), so that both the
// transposing stores and the 4-wide reads of either phase are free of bank
// conflicts.  V columns >= nb load as zero (so do rows >= rows, columns >= nt).
// ---------------------------------------------------------------------------
constexpr int QUC = 8;    // CTAs per cluster
constexpr int QUR = 128;  // rows per sub-tile
constexpr int QUT = 256;  // threads per CTA

template <typename T>
struct alignas(4 * sizeof(T)) QuVec {
    T v[4];
};

// position of (column c, row i) in a swizzled [32][QUR] sub-tile
__device__ __forceinline__ int qu_idx(int c, int i) { return c * QUR + ((((i >> 2) ^ (c >> 2)) << 2) | (i & 3)); }

template <typename T>
static size_t qu_smem_bytes() {
    // V and C sub-tiles (the row-group partials of phase 1 reuse them), the
    // cluster-visible partial W_r, the summed W, W2 and T
    return sizeof(T) * (2 * 32 * QUR + 3 * 32 * 33 + 32 * 32);
}

// A sub-tile in registers: thread t holds row t mod QUR of columns
// t / QUR + 2 j, j < 16, of V and C (consecutive threads read consecutive rows).
template <typename T>
struct QuRegs {
    T v[16], c[16];
};

template <typename T>
__device__ __forceinline__ void qu_fetch(QuRegs<T>& rg, const T* __restrict__ V, int64_t ldv, int nb,
                                         const T* __restrict__ C, int64_t ldc, int64_t ncols, int64_t rows,
                                         int64_t r0) {
    const int i = threadIdx.x & (QUR - 1), c0 = threadIdx.x >> 7;
    const int64_t gi = r0 + i;
    const bool ok = gi < rows;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int c = c0 + 2 * j;
        rg.v[j] = (ok && c < nb) ? V[gi + c * ldv] : (T)0;
        rg.c[j] = (ok && c < ncols) ? C[gi + c * ldc] : (T)0;
    }
}

template <typename T>
__device__ __forceinline__ void qu_put(const QuRegs<T>& rg, T* __restrict__ Vs, T* __restrict__ Cs) {
    const int i = threadIdx.x & (QUR - 1), c0 = threadIdx.x >> 7;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        Vs[qu_idx(c0 + 2 * j, i)] = rg.v[j];
        Cs[qu_idx(c0 + 2 * j, i)] = rg.c[j];
    }
}

template <typename T, int CL>
__global__ void __launch_bounds__(QUT)
    k_qr_update(T* __restrict__ C, int64_t ldc, int64_t nt, const T* __restrict__ V, int64_t ldv, int nb,
                const T* __restrict__ Tm, int64_t rows) {
    extern __shared__ __align__(16) unsigned char qu_raw[];
    T* Vs = (T*)qu_raw;
    T* Cs = Vs + 32 * QUR;
    T* Wr = Cs + 32 * QUR;  // [32][33] this CTA's partial, read by the whole cluster
    T* Wf = Wr + 32 * 33;   // [32][33] the cluster sum
    T* Ts = Wf + 32 * 33;   // [32][33] T
    T* W2 = Ts + 32 * 33;   // [32][32] T^T W
    T* Wk = Vs;             // [4][32][33] row-group partials (after phase 1)
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int64_t c0 = (int64_t)(blockIdx.x / CL) * 32;
    const int64_t ncols = min64(32, nt - c0);
    T* Cb = C + c0 * ldc;
    const int tid = threadIdx.x;
    const int64_t nsub = (rows + QUR - 1) / QUR;
    for (int q = tid; q < 32 * 32; q += QUT) Ts[(q & 31) * 33 + (q >> 5)] = Tm[q];  // Ts[k][p] = T[k, p]

    // 1. W_r = V^T C over this CTA's sub-tiles (the next sub-tile is fetched
    // into registers while the current one is used)
    QuRegs<T> rg;
    if (rank < nsub) qu_fetch<T>(rg, V, ldv, nb, Cb, ldc, ncols, rows, (int64_t)rank * QUR);
    {
        const int kg = tid >> 6, tl = tid & 63, tp = tl & 7, tq = tl >> 3;
        T acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
        for (int64_t sb = rank; sb < nsub; sb += CL) {
            __syncthreads();
            qu_put<T>(rg, Vs, Cs);
            __syncthreads();
            if (sb + CL < nsub) qu_fetch<T>(rg, V, ldv, nb, Cb, ldc, ncols, rows, (sb + CL) * QUR);
#pragma unroll 2
            for (int s4 = 0; s4 < QUR / 16; ++s4) {
                const int i = kg * (QUR / 4) + 4 * s4;
                QuVec<T> va[4], cb[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) va[a] = *(const QuVec<T>*)(Vs + qu_idx(4 * tp + a, i));
#pragma unroll
                for (int b = 0; b < 4; ++b) cb[b] = *(const QuVec<T>*)(Cs + qu_idx(4 * tq + b, i));
#pragma unroll
                for (int w = 0; w < 4; ++w)
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) acc[a][b] = fma(va[a].v[w], cb[b].v[w], acc[a][b]);
            }
        }
        __syncthreads();
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) Wk[(kg * 32 + 4 * tp + a) * 33 + 4 * tq + b] = acc[a][b];
        __syncthreads();
        for (int q = tid; q < 32 * 32; q += QUT) {
            const int p = q >> 5, c = q & 31;
            Wr[p * 33 + c] = ((Wk[p * 33 + c] + Wk[(32 + p) * 33 + c]) + Wk[(64 + p) * 33 + c]) + Wk[(96 + p) * 33 + c];
        }
    }
    // the first sub-tile of step 3 (C is not written before step 3)
    if (rank < nsub) qu_fetch<T>(rg, V, ldv, nb, Cb, ldc, ncols, rows, (int64_t)rank * QUR);
    // 2. W = sum over the cluster, W2 = T^T W
    cluster.sync();
    for (int q = tid; q < 32 * 32; q += QUT) {
        const int p = q >> 5, c = q & 31;
        T w = (T)0;
        for (int r = 0; r < CL; ++r) w += cluster.map_shared_rank(Wr, r)[p * 33 + c];
        Wf[p * 33 + c] = w;
    }
    // this CTA's reads of the other CTAs' partials are done; they may exit
    // once every CTA has arrived (waited for at the end)
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    __syncthreads();
    for (int q = tid; q < 32 * 32; q += QUT) {
        const int p = q >> 5, c = q & 31;
        T w = (T)0;
        for (int k = 0; k <= p; ++k) w = fma(Ts[k * 33 + p], Wf[k * 33 + c], w);
        W2[p * 32 + c] = w;
    }
    // 3. C -= V W2 over this CTA's sub-tiles
    {
        const int ti = tid & 31, tq = tid >> 5;  // rows 4 ti .. 4 ti + 3, columns 4 tq .. 4 tq + 3
        for (int64_t sb = rank; sb < nsub; sb += CL) {
            __syncthreads();
            qu_put<T>(rg, Vs, Cs);
            __syncthreads();
            if (sb + CL < nsub) qu_fetch<T>(rg, V, ldv, nb, Cb, ldc, ncols, rows, (sb + CL) * QUR);
            QuVec<T> cv[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) cv[b] = *(const QuVec<T>*)(Cs + qu_idx(4 * tq + b, 4 * ti));
#pragma unroll 4
            for (int p = 0; p < 32; ++p) {
                const QuVec<T> v = *(const QuVec<T>*)(Vs + qu_idx(p, 4 * ti));
                const QuVec<T> w = *(const QuVec<T>*)(W2 + p * 32 + 4 * tq);
#pragma unroll
                for (int b = 0; b < 4; ++b)
#pragma unroll
                    for (int a = 0; a < 4; ++a) cv[b].v[a] = fma(-v.v[a], w.v[b], cv[b].v[a]);
            }
#pragma unroll
            for (int b = 0; b < 4; ++b) *(QuVec<T>*)(Cs + qu_idx(4 * tq + b, 4 * ti)) = cv[b];
            __syncthreads();
            const int64_t r0 = sb * QUR;
            for (int e = tid; e < 32 * QUR; e += QUT) {
                const int i = e & (QUR - 1), c = e >> 7;
                if (r0 + i < rows && c < ncols) Cb[(r0 + i) + c * ldc] = Cs[qu_idx(c, i)];
            }
        }
    }
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
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

// Dynamic shared memory of the cluster panel: the local panel and, after it,
// rank 0's V^T V partials of every rank or (fused: the previous panel's
// update applied first) the local rows of V_p and the row-group partials.
template <typename T>
static size_t qr_cluster_smem(int64_t rows, int qcl, bool fused) {
    const size_t Rp = (size_t)(ceil_div(rows, qcl) | 1);
    // the fused form also stages the previous panel's V rows and the W
    // partials (Vl, Wk, Ct, Vt behind the local panel)
    const size_t pre = Rp * QNB + (size_t)(QKG + 2) * QNB * (QNB + 1);
    return sizeof(T) * (Rp * QNB + (fused ? pre : 0));
}

struct QrCluster {
    int qcl = 0;         // CTAs per cluster, 0: single-CTA panel kernel
    bool fused = false;  // each panel applies the previous panel's update to its own columns
};

// 16 CTAs per cluster where the device can schedule that with the panel's
// shared memory (non-portable size), else 8; 0 if neither fits (the
// single-CTA panel kernel then runs).  The fused form (each panel applies the
// previous panel's update to its own columns) is preferred where its shared
// memory fits.  Decided once per precision and size.
template <typename T>
static QrCluster qr_cluster_query(int64_t s) {
    const size_t lim = 200 * 1024;
    for (bool fused : {true, false})
        for (int qcl : {16, 8}) {
            const size_t sm = qr_cluster_smem<T>(s, qcl, fused);
            if (sm > lim) continue;
            auto kern = qcl == 16 ? k_qr_panel_cl<T, 16> : k_qr_panel_cl<T, 8>;
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess ||
                (qcl > 8 &&
                 cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
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
            if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) == cudaSuccess && nclusters >= 1) {
                QrCluster q;
                q.qcl = qcl;
                q.fused = fused;
                return q;
            }
            cudaGetLastError();
        }
    return QrCluster();
}

template <typename T>
static QrCluster qr_cluster_size(int64_t s) {
    static std::mutex mu;
    static int64_t last_s = -1;
    static int last_dev = -1;
    static QrCluster last_q;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (s != last_s || dev != last_dev) {
        last_q = qr_cluster_query<T>(s);
        last_s = s;
        last_dev = dev;
    }
    return last_q;
}

template <typename T>
static cudaError_t qr_launch_cluster(int qcl, size_t smem, cudaStream_t st, T* W, int64_t s, int64_t k0, int nb,
                                     T* beta, T* Tm, T* V, int64_t rows, const T* Vp, int64_t ldvp, const T* Tp) {
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
    return cudaLaunchKernelEx(&cfg, kern, W, s, s, k0, nb, beta, Tm, V, rows, Vp, ldvp, Tp);
}

// V and T are double-buffered by panel parity (a panel's V and T are read by
// its trailing update and by the next panel while the next panel writes the
// other buffer).
struct QrLayout {
    size_t w, beta, tm[2], v[2];
    size_t total;
};

static QrLayout qr_layout(int64_t s, int64_t n, int es) {
    QrLayout L;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    L.w = take((size_t)s * n * es);
    L.beta = take((size_t)n * es);
    for (int b = 0; b < 2; ++b) {
        L.tm[b] = take((size_t)QNB * QNB * es);
        L.v[b] = take((size_t)s * QNB * es);
    }
    L.total = off;
    return L;
}

// Whether clusters of 16 update CTAs (non-portable size) can be scheduled
// with the update's shared memory; decided once per device.
template <typename T>
static bool qu_cluster16_ok() {
    static std::mutex mu;
    static int known[64] = {};  // 0 unknown, 1 yes, 2 no
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    std::lock_guard<std::mutex> lk(mu);
    if (known[dev] == 0) {
        const size_t sm = qu_smem_bytes<T>();
        auto kern = k_qr_update<T, 16>;
        bool ok = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) == cudaSuccess &&
                  cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
        if (ok) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = 16;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(16);
            cfg.blockDim = dim3(QUT);
            cfg.dynamicSmemBytes = sm;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int nclusters = 0;
            ok = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) == cudaSuccess && nclusters >= 1;
        }
        cudaGetLastError();
        known[dev] = ok ? 1 : 2;
    }
    return known[dev] == 1;
}

// C (rows x nt, ld s) <- (I - V T^T V^T) C.  A cluster per 32 columns; FP64
// updates of few columns (the in-block updates of the blocked FP64 QR: at
// most 7 column tiles, 56 CTAs with 8 per cluster) take 16 CTAs per cluster
// when there are rows for 16 (2048 or more), so that twice the SMs share
// them.
template <typename T>
static lsq_status qr_apply(const T* V, const T* Tm, int nb, int64_t rows, T* C, int64_t s, int64_t nt,
                           cudaStream_t st) {
    if (nt <= 0) return LSQ_OK;
    const size_t sm = qu_smem_bytes<T>();
    const int64_t ctiles = ceil_div(nt, 32);
    const bool wide = std::is_same<T, double>::value && ctiles * 16 <= device_sm_count() &&
                      ceil_div(rows, QUR) >= 16 && qu_cluster16_ok<T>();
    const int cl = wide ? 16 : 8;
    auto kern = wide ? k_qr_update<T, 16> : k_qr_update<T, 8>;
    LSQ_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(ctiles * cl));
    cfg.blockDim = dim3(QUT);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    LSQ_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, C, s, nt, V, rows, nb, Tm, rows));
    note_launch();
    return LSQ_OK;
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

// ---------------------------------------------------------------------------
// FP64 QR with the trailing updates on the tensor cores.  The columns are
// taken in blocks of QTB: inside a block, 32-column panels and their
// rank-32 updates as above (restricted to the block); then the block's
// reflectors H_1 ... H_b = I - V T V^T update every later column at once,
//   W = V^T C,  X = T^T W,  C <- C - V X,
// each an FP64-accurate digit-sliced product (csrc/oz_trsm.cu; K chunks of
// at most 512).  T is formed from S = T^{-1} = striu(V^T V) + diag(1/beta)
// (Puglisi 1992; Joffrain et al. 2006: the triangular factor of the compact
// WY form is the inverse of that matrix), column by column with the betas
// as factors (a zero beta, H = I, gives a zero row and column of T).
// ---------------------------------------------------------------------------
constexpr int QTB = 256;  // columns per block of the tensor-core form
constexpr int QTK = 512;  // K chunk of one digit-sliced product

static bool qr_tc_blocked(int es, int64_t n) { return es == 8 && n > QTB && fp64_emulation_enabled() && ot_trsm_supported(); }

struct QrTcLayout {
    size_t vx, vt, g, tt, wn, xp, err, ot, ot_bytes, total;
};

static QrTcLayout qr_tc_layout(int64_t s, int64_t n) {
    QrTcLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    L.vx = take(sizeof(double) * (size_t)s * QTB);
    L.vt = take(sizeof(double) * (size_t)s * QTB);
    L.g = take(sizeof(double) * QTB * QTB);
    L.tt = take(sizeof(double) * QTB * QTB);
    L.wn = take(sizeof(double) * QTB * (size_t)n);
    L.xp = take(sizeof(double) * QTB * (size_t)n);
    L.err = take(sizeof(int32_t));
    L.ot_bytes = ot_update_ws_bytes(std::max<int64_t>(s, QTB), std::max<int64_t>(n, QTB), QTK);
    L.ot = take(L.ot_bytes);
    L.total = off;
    return L;
}

// The block's reflectors as explicit V (rows x nb, ld rows) and V^T (nb x
// rows, ld nb): unit diagonal, zero above, Householder vectors below (the
// lower part of W's columns j0 .. j0 + nb - 1 from row j0).
__global__ void k_qr_vblock(const double* __restrict__ W, int64_t ld, int64_t j0, int64_t rows, int nb,
                            double* __restrict__ Vx, double* __restrict__ Vt) {
    const int64_t total = rows * nb;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = q % rows, c = q / rows;
        const double v = r < c ? 0.0 : (r == c ? 1.0 : W[(j0 + r) + (j0 + c) * ld]);
        Vx[q] = v;
        Vt[c + r * nb] = v;
    }
}

// T^T (ld nb) from Gn = -V^T V and the betas: column j of T by back
// substitution, t_j = beta_j, t_i = -beta_i sum_{i < p <= j} S[i][p] t_p with
// S[i][p] = (V^T V)[i][p]; one warp per column, the sums over lanes in a
// fixed order.
__global__ void __launch_bounds__(32) k_qr_tinv(const double* __restrict__ Gn, const double* __restrict__ beta,
                                                 int nb, double* __restrict__ Tt) {
    __shared__ double t[QTB];
    const int j = blockIdx.x, lane = threadIdx.x;
    for (int i = lane; i < nb; i += 32) t[i] = 0.0;
    __syncwarp();
    if (lane == 0) t[j] = beta[j];
    __syncwarp();
    for (int i = j - 1; i >= 0; --i) {
        double acc = 0.0;
        for (int p = i + 1 + lane; p <= j; p += 32) acc = fma(-Gn[i + (int64_t)p * nb], t[p], acc);
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) t[i] = -beta[i] * acc;
        __syncwarp();
    }
    for (int i = lane; i < nb; i += 32) Tt[j + (int64_t)i * nb] = t[i];
}

__global__ void k_qr_err_to_info(const int32_t* __restrict__ err, int32_t* __restrict__ info) {
    if (*err != 0 && *info == 0) *info = -2;
}

// C (rows x nt, ld s) <- (I - V T^T V^T) C for the block of nb reflectors
// stored in W's columns j0 .. j0 + nb - 1 (C: W's rows j0.., columns j0 + nb..).
static lsq_status qr_tc_trailing(double* W, int64_t s, int64_t j0, int nb, int64_t n, const double* beta, char* base,
                                 const QrTcLayout& L, cudaStream_t st) {
    const int64_t rows = s - j0, nt = n - j0 - nb;
    if (nt <= 0) return LSQ_OK;
    double* Vx = (double*)(base + L.vx);
    double* Vt = (double*)(base + L.vt);
    double* Gn = (double*)(base + L.g);
    double* Tt = (double*)(base + L.tt);
    double* Wn = (double*)(base + L.wn);
    double* Xp = (double*)(base + L.xp);
    int32_t* err = (int32_t*)(base + L.err);
    char* ows = base + L.ot;
    double* C = W + j0 + (j0 + nb) * s;
    lsq_status r;
    k_qr_vblock<<<(unsigned)std::min<int64_t>(ceil_div(rows * nb, 256), 8192), 256, 0, st>>>(W, s, j0, rows, nb, Vx,
                                                                                              Vt);
    LSQ_LAUNCH_CHECK();
    // Gn = -V^T V and Wn = -V^T C, accumulated over K chunks of the rows
    LSQ_CUDA_TRY(cudaMemsetAsync(Gn, 0, sizeof(double) * nb * nb, st));
    LSQ_CUDA_TRY(cudaMemsetAsync(Wn, 0, sizeof(double) * nb * (size_t)nt, st));
    for (int64_t k = 0; k < rows; k += QTK) {
        const int64_t kc = std::min<int64_t>(QTK, rows - k);
        if ((r = ot_gemm_update(Vt + k * nb, nb, Vx + k, 1, rows, Gn, nb, Gn, nb, nb, nb, kc, ows, L.ot_bytes, err,
                                st)) != LSQ_OK)
            return r;
        if ((r = ot_gemm_update(Vt + k * nb, nb, C + k, 1, s, Wn, nb, Wn, nb, nb, nt, kc, ows, L.ot_bytes, err, st)) !=
            LSQ_OK)
            return r;
    }
    k_qr_tinv<<<(unsigned)nb, 32, 0, st>>>(Gn, beta + j0, nb, Tt);
    LSQ_LAUNCH_CHECK();
    // Xp = 0 - T^T Wn = T^T (V^T C)
    LSQ_CUDA_TRY(cudaMemsetAsync(Xp, 0, sizeof(double) * nb * (size_t)nt, st));
    if ((r = ot_gemm_update(Tt, nb, Wn, 1, nb, Xp, nb, Xp, nb, nb, nt, nb, ows, L.ot_bytes, err, st)) != LSQ_OK)
        return r;
    // C <- C - V Xp
    return ot_gemm_update(Vx, rows, Xp, 1, nb, C, s, C, s, rows, nt, nb, ows, L.ot_bytes, err, st);
}

size_t qr_ws_bytes(int64_t s, int64_t n, int prec) {
    int es = prec == LSQ_FP64 ? 8 : 4;
    size_t b = qr_layout(s, n, es).total + 256;
    if (qr_tc_blocked(es, n)) b += qr_tc_layout(s, n).total + 256;
    return b;
}

// FP64 QR by blocks of QTB columns (see qr_tc_trailing): the panels and
// rank-32 updates inside a block on the panel stream as in qr_run, the
// block's update of every later column on the tensor cores.  W holds A_s.
static lsq_status qr_blocked_f64(double* W, double* beta, int64_t s, int64_t n, const int32_t* colexp, double* Rs,
                                 int64_t ldr, int32_t* info, char* base, const QrLayout& L, char* tcb,
                                 cudaStream_t st) {
    const QrTcLayout TL = qr_tc_layout(s, n);
    int32_t* err = (int32_t*)(tcb + TL.err);
    LSQ_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int32_t), st));
    const QrCluster qc = qr_cluster_size<double>(s);
    const int qcl = qc.qcl;
    int k = 0;  // panel counter: the parity of the V and T buffers
    lsq_status r = LSQ_OK;
    for (int64_t j0 = 0; j0 < n && r == LSQ_OK; j0 += QTB) {
        const int64_t j1 = std::min<int64_t>(n, j0 + QTB);
        const double* Vprev = nullptr;
        const double* Tprev = nullptr;
        int64_t ldvprev = 0;
        for (int64_t k0 = j0; k0 < j1; k0 += QNB, ++k) {
            const int b = k & 1;
            const int nb = (int)std::min<int64_t>(QNB, j1 - k0);
            const int64_t rows = s - k0;
            double* Tm = (double*)(base + L.tm[b]);
            double* V = (double*)(base + L.v[b]);
            if (qcl > 0) {
                const size_t clsm = qr_cluster_smem<double>(rows, qcl, qc.fused);
                if (qr_launch_cluster<double>(qcl, clsm, st, W, s, k0, nb, beta, Tm, V, rows, Vprev, ldvprev, Tprev) !=
                    cudaSuccess)
                    return LSQ_ERR_CUDA;
            } else {
                k_qr_panel<double><<<1, QPT, 0, st>>>(W, s, s, k0, nb, beta, Tm, V, rows);
            }
            note_launch();
            if (cudaGetLastError() != cudaSuccess) return LSQ_ERR_CUDA;
            // the rest of the block's columns
            const int64_t nt = j1 - k0 - nb;
            if (nt <= 0) {
                ++k;
                break;
            }
            const int64_t nn = std::min<int64_t>(QNB, nt), nw = nt - nn;
            double* C = W + k0 + (k0 + nb) * s;
            const bool fuse_next = qcl > 0 && qc.fused && nb == QNB;
            r = fuse_next ? qr_apply<double>(V, Tm, nb, rows, C + nn * s, s, nw, st)
                          : qr_apply<double>(V, Tm, nb, rows, C, s, nt, st);
            if (r != LSQ_OK) return r;
            Vprev = fuse_next ? V : nullptr;
            Tprev = fuse_next ? Tm : nullptr;
            ldvprev = rows;
        }
        // the block's reflectors on every later column
        r = qr_tc_trailing(W, s, j0, (int)(j1 - j0), n, beta, tcb, TL, st);
    }
    if (r != LSQ_OK) return r;
    k_qr_extract<double><<<(unsigned)std::min<int64_t>(ceil_div(n * n, 256), 4096), 256, 0, st>>>(W, s, n, colexp, Rs,
                                                                                                ldr);
    LSQ_LAUNCH_CHECK();
    if (info) {
        k_check_diag<<<(unsigned)ceil_div(n, 128), 128, 0, st>>>(Rs, n, ldr, info);
        LSQ_LAUNCH_CHECK();
        k_qr_err_to_info<<<1, 1, 0, st>>>(err, info);
        LSQ_LAUNCH_CHECK();
    }
    return LSQ_OK;
}

template <typename T>
static lsq_status qr_run(const void* As, int64_t s, int64_t n, int64_t ldas, int as_prec, const int32_t* colexp,
                         double* Rs, int64_t ldr, int32_t* info, void* ws, size_t ws_bytes, cudaStream_t st) {
    int es = sizeof(T);
    QrLayout L = qr_layout(s, n, es);
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
    if constexpr (std::is_same<T, double>::value) {
        if (qr_tc_blocked(es, n)) {
            char* tcb = base + align_up(L.total, 256);
            if (L.total + 256 + qr_tc_layout(s, n).total + ((char*)base - (char*)ws) > ws_bytes) return LSQ_ERR_NOMEM;
            return qr_blocked_f64(W, beta, s, n, colexp, Rs, ldr, info, base, L, tcb, st);
        }
    }
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
    const QrCluster qc = qr_cluster_size<T>(s);
    const int qcl = qc.qcl;
    // the previous panel's V and T when this panel applies its update itself
    const T* Vprev = nullptr;
    const T* Tprev = nullptr;
    int64_t ldvprev = 0;
    int k = 0;
    for (int64_t k0 = 0; k0 < n && r == LSQ_OK; k0 += QNB, ++k) {
        const int b = k & 1;
        int nb = (int)std::min<int64_t>(QNB, n - k0);
        int64_t rows = s - k0;
        T* Tm = (T*)(base + L.tm[b]);
        T* V = (T*)(base + L.v[b]);
        const size_t clsm = qcl > 0 ? qr_cluster_smem<T>(rows, qcl, qc.fused) : 0;
        // Householder panel: sum over its columns of 4 (rows - j)(nb - j) flops
        double pflops = 0.0;
        for (int j = 0; j < nb; ++j) pflops += 4.0 * (double)(rows - j) * (double)(nb - j);
        stage_mark(ST_K_QRPANEL, true, sh);
        if (qcl > 0) {
            if (qr_launch_cluster<T>(qcl, clsm, sh, W, s, k0, nb, beta, Tm, V, rows, Vprev, ldvprev, Tprev) !=
                cudaSuccess) {
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
        // the next panel's columns (narrow part): by the next panel kernel
        // itself when fused (a full panel only: V then has QNB columns), else
        // a separate update on the panel stream
        const bool fuse_next = qcl > 0 && qc.fused && nb == QNB;
        if (qs) {
            // the wide part on the low-priority stream, after this panel
            if (cudaEventRecord(ev_p, sh) != cudaSuccess || cudaStreamWaitEvent(sl, ev_p, 0) != cudaSuccess) {
                r = LSQ_ERR_CUDA;
                break;
            }
            r = qr_apply<T>(V, Tm, nb, rows, C + nn * s, s, nw, sl);
            if (r != LSQ_OK || cudaEventRecord(ev_w[b], sl) != cudaSuccess) {
                r = r != LSQ_OK ? r : LSQ_ERR_CUDA;
                break;
            }
            // the next panel's columns also hold the previous panel's wide
            // update, and the next panel overwrites that update's V and T
            if (k >= 1 && cudaStreamWaitEvent(sh, ev_w[b ^ 1], 0) != cudaSuccess) {
                r = LSQ_ERR_CUDA;
                break;
            }
            if (!fuse_next) r = qr_apply<T>(V, Tm, nb, rows, C, s, nn, sh);
        } else {
            r = fuse_next ? qr_apply<T>(V, Tm, nb, rows, C + nn * s, s, nw, st)
                          : qr_apply<T>(V, Tm, nb, rows, C, s, nt, st);
        }
        Vprev = fuse_next ? V : nullptr;
        Tprev = fuse_next ? Tm : nullptr;
        ldvprev = rows;
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
