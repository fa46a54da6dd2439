// Block-level triangular solve on a vector held in shared memory, used by
// the vector solves of Eqs. e_pne / e_hpne and by the Hager iterations of the
// condition estimate.  Diagonal 32x32 blocks are solved by warp 0 with
// shuffles; the off-diagonal updates are spread over the whole block.
#pragma once
#include "common.cuh"

namespace lsq {

// TB_UPPER_T: U^T y = c for upper U (a forward solve reading U by rows).
enum TrsvKindB { TB_LOWER = 0, TB_LOWER_T = 1, TB_UPPER = 2, TB_UNIT_LOWER = 3, TB_UPPER_T = 4 };

template <typename T>
__device__ void block_trsv(int kind, const T* __restrict__ M, int64_t n, int64_t ld, T* ys) {
    __shared__ T dblk[32][33];
    int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nth = blockDim.x;
    bool forward = (kind == TB_LOWER || kind == TB_UNIT_LOWER || kind == TB_UPPER_T);
    bool unit = (kind == TB_UNIT_LOWER);
    int64_t nblk = (n + 31) / 32;
    __syncthreads();
    for (int64_t bq = 0; bq < nblk; ++bq) {
        int64_t b = forward ? bq : nblk - 1 - bq;
        int64_t b0 = b * 32;
        int bs = (int)min64(32, n - b0);
        // the diagonal block, staged by the whole block in one pass
        for (int q = tid; q < 32 * 32; q += nth) {
            int r = q & 31, c = q >> 5;
            dblk[r][c] = (r < bs && c < bs) ? M[(b0 + r) + (b0 + c) * ld] : (T)0;
        }
        __syncthreads();
        if (warp == 0) {
            T v = lane < bs ? ys[b0 + lane] : (T)0;
            if (forward) {
                for (int jj = 0; jj < bs; ++jj) {
                    if (lane == jj && !unit) v = v / dblk[jj][jj];
                    T vj = __shfl_sync(0xffffffffu, v, jj);
                    if (lane > jj && lane < bs) {
                        T mv = kind == TB_UPPER_T ? dblk[jj][lane] : dblk[lane][jj];
                        v = fma(-mv, vj, v);
                    }
                }
            } else {
                for (int jj = bs - 1; jj >= 0; --jj) {
                    if (lane == jj) v = v / dblk[jj][jj];
                    T vj = __shfl_sync(0xffffffffu, v, jj);
                    if (lane < jj) {
                        T mv = kind == TB_UPPER ? dblk[lane][jj] : dblk[jj][lane];
                        v = fma(-mv, vj, v);
                    }
                }
            }
            if (lane < bs) ys[b0 + lane] = v;
        }
        __syncthreads();
        if (forward) {
            for (int64_t i = b0 + bs + tid; i < n; i += nth) {
                T t = ys[i];
                if (kind == TB_UPPER_T)
                    for (int k = 0; k < bs; ++k) t = fma(-M[(b0 + k) + i * ld], ys[b0 + k], t);
                else
                    for (int k = 0; k < bs; ++k) t = fma(-M[i + (b0 + k) * ld], ys[b0 + k], t);
                ys[i] = t;
            }
        } else {
            for (int64_t i = tid; i < b0; i += nth) {
                T t = ys[i];
                if (kind == TB_UPPER)
                    for (int k = 0; k < bs; ++k) t = fma(-M[i + (b0 + k) * ld], ys[b0 + k], t);
                else
                    for (int k = 0; k < bs; ++k) t = fma(-M[(b0 + k) + i * ld], ys[b0 + k], t);
                ys[i] = t;
            }
        }
        __syncthreads();
    }
}

}  // namespace lsq
