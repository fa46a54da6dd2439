// Hager's estimate of ||M^{-1}||_1 in FP32 (Sec. 6.1's estimator; Higham's
// form: the stopping test, at most five iterations and the alternating-sign
// extra vector) for the condition estimates: M^{-1} = (L L^T)^{-1} with L
// lower triangular (a Cholesky factor of the Gram, or R_e^T), or R^{-1} with
// R upper triangular (the judge of a preconditioner).
//
// Every application of M^{-1} (or M^{-T}) runs as the wavefront triangular
// solves of csrc/factor.cu across many CTAs; the reductions, the argmax and
// the decisions run in single-block kernels.  The launch sequence is fixed
// (four iterations of the loop are always launched): once the test ends the
// iterations a device flag makes the remaining kernels and solves return at
// once, so the host never waits on the device.
#include "common.cuh"
#include "kernels.cuh"

#include <algorithm>

namespace lsq {

struct HagerState {
    float est;      // current estimate of ||M^{-1}||_1
    int32_t jlast;  // index of the last unit vector
    int32_t done;   // the iterations are over: their kernels and solves skip
    int32_t fail;   // the factor is unusable: every solve skips
};

struct HagerLayout {
    size_t st, x, y, xi, z, sync, total;
};

static HagerLayout hager_layout(int64_t n) {
    HagerLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    L.st = take(sizeof(HagerState));
    L.x = take(sizeof(float) * (size_t)n);
    L.y = take(sizeof(float) * (size_t)n);
    L.xi = take(sizeof(float) * (size_t)n);
    L.z = take(sizeof(float) * (size_t)n);
    L.sync = take(sizeof(int32_t) * trsv_sync_ints(n));
    L.total = off;
    return L;
}

size_t hager_ws_bytes(int64_t n) { return hager_layout(n).total + 256; }

constexpr int HG_THREADS = 1024;

// Block sum and max (all threads get the result).
__device__ float hg_sum(float v, float* red) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = 0.0f;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    return t;
}

__global__ void __launch_bounds__(HG_THREADS) k_hg_init(float* __restrict__ x, float* __restrict__ y, int64_t n,
                                                        const int32_t* __restrict__ fail, HagerState* st) {
    const float v = 1.0f / (float)n;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) x[i] = y[i] = v;
    if (threadIdx.x == 0) {
        const int32_t f = fail ? *fail : 0;
        st->est = 0.0f;
        st->jlast = -1;
        st->fail = f != 0;
        st->done = f != 0;
    }
}

// est = ||y||_1, xi = z = sign(y)
__global__ void __launch_bounds__(HG_THREADS) k_hg_first(const float* __restrict__ y, float* __restrict__ xi,
                                                         float* __restrict__ z, int64_t n, HagerState* st) {
    __shared__ float red[32];
    float p = 0.0f;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        p += fabsf(y[i]);
        xi[i] = z[i] = y[i] >= 0.0f ? 1.0f : -1.0f;
    }
    const float est = hg_sum(p, red);
    if (threadIdx.x == 0) st->est = est;
}

// j = argmax |z_i| (the first of equal maxima); stop if |z_j| <= z^T x or j
// repeats; else x = y = e_j.
__global__ void __launch_bounds__(HG_THREADS) k_hg_pick(const float* __restrict__ z, float* __restrict__ x,
                                                        float* __restrict__ y, int64_t n, HagerState* st) {
    // the state is read once, before any thread of the block writes it
    __shared__ float red[32], rv[32];
    __shared__ int ri[32];
    __shared__ int stop, jsel, s_done, s_jlast;
    if (threadIdx.x == 0) {
        s_done = st->done;
        s_jlast = st->jlast;
    }
    __syncthreads();
    if (s_done) return;
    float best = -1.0f, pz = 0.0f;
    int bi = 0x7fffffff;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const float a = fabsf(z[i]);
        if (a > best) {
            best = a;
            bi = (int)i;
        }
        pz += z[i] * x[i];
    }
    for (int off = 16; off > 0; off >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, best, off);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (ov > best || (ov == best && oi < bi)) {
            best = ov;
            bi = oi;
        }
    }
    if ((threadIdx.x & 31) == 0) {
        rv[threadIdx.x >> 5] = best;
        ri[threadIdx.x >> 5] = bi;
    }
    const float ztx = hg_sum(pz, red);  // synchronises the block
    if (threadIdx.x == 0) {
        float zmax = -1.0f;
        int j = 0x7fffffff;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q)
            if (rv[q] > zmax || (rv[q] == zmax && ri[q] < j)) {
                zmax = rv[q];
                j = ri[q];
            }
        stop = (zmax <= ztx || j == s_jlast || j < 0 || (int64_t)j >= n) ? 1 : 0;
        jsel = j;
        if (stop) st->done = 1;
        else st->jlast = j;
    }
    __syncthreads();
    if (stop) return;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) x[i] = y[i] = (i == jsel) ? 1.0f : 0.0f;
}

// est_new = ||y||_1; stop if sign(y) == xi or est_new <= est (keeping the
// larger); else est = est_new, xi = z = sign(y).
__global__ void __launch_bounds__(HG_THREADS) k_hg_update(const float* __restrict__ y, float* __restrict__ xi,
                                                          float* __restrict__ z, int64_t n, HagerState* st) {
    // the state is read once, before any thread of the block writes it
    __shared__ float red[32], s_est;
    __shared__ int differ, s_done;
    if (threadIdx.x == 0) {
        differ = 0;
        s_done = st->done;
        s_est = st->est;
    }
    __syncthreads();
    if (s_done) return;
    float p = 0.0f;
    int d = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        p += fabsf(y[i]);
        d |= ((y[i] >= 0.0f ? 1.0f : -1.0f) != xi[i]);
    }
    const float est_new = hg_sum(p, red);  // synchronises the block
    if (d) differ = 1;
    __syncthreads();
    const float est = s_est;
    if (!differ || est_new <= est) {
        if (threadIdx.x == 0) {
            if (est_new > est) st->est = est_new;
            st->done = 1;
        }
        return;
    }
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) xi[i] = z[i] = y[i] >= 0.0f ? 1.0f : -1.0f;
    if (threadIdx.x == 0) st->est = est_new;
}

// The extra vector (-1)^i (1 + i / (n - 1)).
__global__ void k_hg_alt(float* __restrict__ y, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float mag = n > 1 ? 1.0f + (float)i / (float)(n - 1) : 1.0f;
        y[i] = (i % 2 == 0) ? mag : -mag;
    }
}

// out = max(est, 2 ||y||_1 / (3 n)); +inf when the factor was unusable.
__global__ void __launch_bounds__(HG_THREADS) k_hg_final(const float* __restrict__ y, int64_t n,
                                                         const HagerState* st, float* __restrict__ out) {
    __shared__ float red[32];
    float p = 0.0f;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) p += fabsf(y[i]);
    const float alt = 2.0f * hg_sum(p, red) / (3.0f * (float)n);
    if (threadIdx.x == 0) *out = st->fail ? __int_as_float(0x7f800000) : fmaxf(st->est, alt);
}

// ||M||_1 (largest column sum of |M|; the upper triangle only when upper),
// one warp per column, into *out as the bit pattern of a non-negative float
// (atomicMax orders those like the values; NaN lands above +inf).  *out must
// be zero before the launch.
__global__ void k_colnorm1_max(const float* __restrict__ M, int64_t n, int64_t ld, int upper,
                               unsigned int* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t wpb = blockDim.x >> 5;
    for (int64_t c = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); c < n; c += (int64_t)gridDim.x * wpb) {
        const int64_t rows = upper ? c + 1 : n;
        float s = 0.0f;
        for (int64_t i = lane; i < rows; i += 32) s += fabsf(M[i + c * ld]);
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) atomicMax(out, __float_as_uint(s));
    }
}

lsq_status launch_colnorm1_max(const float* M, int64_t n, int64_t ld, bool upper, float* out, cudaStream_t st) {
    LSQ_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(float), st));
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(n, 8), 1024);
    k_colnorm1_max<<<grid, 256, 0, st>>>(M, n, ld, upper ? 1 : 0, (unsigned int*)out);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

lsq_status hager_inv_norm1(const float* M, int64_t n, int64_t ld, bool upper, const int32_t* fail, float* est_out,
                           int32_t* err, void* ws, size_t ws_bytes, cudaStream_t st) {
    const HagerLayout L = hager_layout(n);
    char* base = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    if (!ws || n <= 0 || L.total + (size_t)(base - (char*)ws) > ws_bytes) return LSQ_ERR_NOMEM;
    HagerState* hs = (HagerState*)(base + L.st);
    float* x = (float*)(base + L.x);
    float* y = (float*)(base + L.y);
    float* xi = (float*)(base + L.xi);
    float* z = (float*)(base + L.z);
    int32_t* sync = (int32_t*)(base + L.sync);
    const int32_t* always = &hs->fail;  // solves that run unless the factor failed
    const int32_t* loop = &hs->done;    // solves of the iterations
    // v <- M^{-1} v, or M^{-T} v (the same for the symmetric (L L^T)^{-1})
    auto apply = [&](float* v, bool transpose, const int32_t* skip) -> lsq_status {
        lsq_status r;
        if (upper) return launch_trsv<float>(transpose ? TRSV_UPPER_T : TRSV_UPPER, M, n, ld, v, skip, sync, err, st);
        if ((r = launch_trsv<float>(TRSV_LOWER, M, n, ld, v, skip, sync, err, st)) != LSQ_OK) return r;
        return launch_trsv<float>(TRSV_LOWER_T, M, n, ld, v, skip, sync, err, st);
    };
    lsq_status r;
    k_hg_init<<<1, HG_THREADS, 0, st>>>(x, y, n, fail, hs);
    LSQ_LAUNCH_CHECK();
    if ((r = apply(y, false, always)) != LSQ_OK) return r;
    k_hg_first<<<1, HG_THREADS, 0, st>>>(y, xi, z, n, hs);
    LSQ_LAUNCH_CHECK();
    if ((r = apply(z, true, always)) != LSQ_OK) return r;
    for (int it = 1; it < 5; ++it) {
        k_hg_pick<<<1, HG_THREADS, 0, st>>>(z, x, y, n, hs);
        LSQ_LAUNCH_CHECK();
        if ((r = apply(y, false, loop)) != LSQ_OK) return r;
        k_hg_update<<<1, HG_THREADS, 0, st>>>(y, xi, z, n, hs);
        LSQ_LAUNCH_CHECK();
        if ((r = apply(z, true, loop)) != LSQ_OK) return r;
    }
    k_hg_alt<<<(unsigned)std::min<int64_t>(ceil_div(n, 256), 1024), 256, 0, st>>>(y, n);
    LSQ_LAUNCH_CHECK();
    if ((r = apply(y, false, always)) != LSQ_OK) return r;
    k_hg_final<<<1, HG_THREADS, 0, st>>>(y, n, hs, est_out);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

}  // namespace lsq
