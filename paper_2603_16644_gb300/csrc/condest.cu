// Low-precision condition estimate of Sec. 6.1 (first line of Alg. 1):
//   G = fl32(A^T A) (A rounded to FP32; the products as six BF16 piece
//   products on the tensor cores with FP32 accumulation, or an FP32 split-K
//   CUDA-core GEMM when the tensor-core sketch GEMM is switched off),
//   ||G||_1, FP32 Cholesky of G, and Hager's estimate of ||G^{-1}||_1 with
//   Higham's stopping test and alternating-sign extra vector (at most 5
//   iterations, every application of G^{-1} = two triangular solves), then
//   kappa0 = 0.5 log10(n ||G||_1 gamma) in FP64 from the FP32 values, since
//   kappa(A)^2 = kappa(A^T A) <= n ||A^T A||_1 ||(A^T A)^{-1}||_1.
// A Cholesky breakdown or a non-finite value is the "overflow" case: kappa0
// = +inf and double precision.  The whole decision stays on the device.
#include "common.cuh"
#include "kernels.cuh"
#include "trsv_block.cuh"

#include <algorithm>

namespace lsq {

__device__ __forceinline__ int prec_from_kappa0(double k0) {
    if (!(k0 == k0) || isinf(k0)) return LSQ_FP64;
    if (k0 < 2.0) return LSQ_FP8_E4M3;
    if (k0 < 3.0) return LSQ_BF16;
    if (k0 < 4.0) return LSQ_FP16;
    if (k0 <= 8.0) return LSQ_FP32;
    return LSQ_FP64;
}

// ||G||_1 of the symmetric FP32 matrix: column sums in row order, max.
__global__ void k_norm1(const float* __restrict__ G, int64_t n, int64_t ld, float* __restrict__ out) {
    float mx = 0.0f;
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
        float s = 0.0f;
        for (int64_t i = 0; i < n; ++i) s += fabsf(G[i + c * ld]);
        mx = fmaxf(mx, s);
    }
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    __shared__ float w[32];
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t = fmaxf(t, w[q]);
        *out = t;
    }
}

__device__ float blk_sum(float v, float* red) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = 0.0f;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    return t;
}

__device__ int blk_argmax_abs(const float* z, int64_t n, float* redv, int* redi, float* outmax) {
    float best = -1.0f;
    int bi = 0x7fffffff;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        float v = fabsf(z[i]);
        if (v > best) { best = v; bi = (int)i; }
    }
    for (int off = 16; off > 0; off >>= 1) {
        float ov = __shfl_xor_sync(0xffffffffu, best, off);
        int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) { redv[threadIdx.x >> 5] = best; redi[threadIdx.x >> 5] = bi; }
    __syncthreads();
    float b = -1.0f;
    int ix = 0x7fffffff;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q)
        if (redv[q] > b || (redv[q] == b && redi[q] < ix)) { b = redv[q]; ix = redi[q]; }
    *outmax = b;
    return ix;
}

// Hager / Higham loop, one block; vectors in dynamic shared memory.
__global__ void __launch_bounds__(512) k_hager(const float* __restrict__ L, int64_t n, int64_t ld,
                                               const float* __restrict__ norm1, const int32_t* __restrict__ chol_info,
                                               double* __restrict__ kappa0, int32_t* __restrict__ chosen) {
    extern __shared__ __align__(16) unsigned char hraw[];
    float* x = reinterpret_cast<float*>(hraw);
    float* y = x + n;
    float* xi = y + n;
    float* z = xi + n;
    __shared__ float redv[32];
    __shared__ int redi[32];
    __shared__ int flag;
    int tid = threadIdx.x;
    if (*chol_info != 0 || !isfinite(*norm1)) {
        if (tid == 0) {
            *kappa0 = __longlong_as_double(0x7ff0000000000000ll);
            *chosen = LSQ_FP64;
        }
        return;
    }
    float fn = (float)n;
    for (int64_t i = tid; i < n; i += blockDim.x) { x[i] = 1.0f / fn; y[i] = 1.0f / fn; }
    block_trsv<float>(TB_LOWER, L, n, ld, y);
    block_trsv<float>(TB_LOWER_T, L, n, ld, y);
    float ps = 0.0f;
    for (int64_t i = tid; i < n; i += blockDim.x) ps += fabsf(y[i]);
    float est = blk_sum(ps, redv);
    for (int64_t i = tid; i < n; i += blockDim.x) { xi[i] = y[i] >= 0.0f ? 1.0f : -1.0f; z[i] = xi[i]; }
    block_trsv<float>(TB_LOWER, L, n, ld, z);
    block_trsv<float>(TB_LOWER_T, L, n, ld, z);
    int jlast = -1;
    for (int it = 1; it < 5; ++it) {
        float zmax;
        int j = blk_argmax_abs(z, n, redv, redi, &zmax);
        float pz = 0.0f;
        for (int64_t i = tid; i < n; i += blockDim.x) pz += z[i] * x[i];
        float ztx = blk_sum(pz, redv);
        if (zmax <= ztx || j == jlast) break;
        jlast = j;
        for (int64_t i = tid; i < n; i += blockDim.x) { x[i] = (i == j) ? 1.0f : 0.0f; y[i] = x[i]; }
        block_trsv<float>(TB_LOWER, L, n, ld, y);
        block_trsv<float>(TB_LOWER_T, L, n, ld, y);
        float py = 0.0f;
        int differ = 0;
        for (int64_t i = tid; i < n; i += blockDim.x) {
            py += fabsf(y[i]);
            differ |= ((y[i] >= 0.0f ? 1.0f : -1.0f) != xi[i]);
        }
        float est_new = blk_sum(py, redv);
        if (tid == 0) flag = 0;
        __syncthreads();
        if (differ) flag = 1;
        __syncthreads();
        if (!flag || est_new <= est) {
            if (est_new > est) est = est_new;
            break;
        }
        est = est_new;
        for (int64_t i = tid; i < n; i += blockDim.x) { xi[i] = y[i] >= 0.0f ? 1.0f : -1.0f; z[i] = xi[i]; }
        block_trsv<float>(TB_LOWER, L, n, ld, z);
        block_trsv<float>(TB_LOWER_T, L, n, ld, z);
    }
    for (int64_t i = tid; i < n; i += blockDim.x) {
        float mag = n > 1 ? 1.0f + (float)i / (float)(n - 1) : 1.0f;
        y[i] = (i % 2 == 0) ? mag : -mag;
    }
    block_trsv<float>(TB_LOWER, L, n, ld, y);
    block_trsv<float>(TB_LOWER_T, L, n, ld, y);
    float pa = 0.0f;
    for (int64_t i = tid; i < n; i += blockDim.x) pa += fabsf(y[i]);
    float alt = 2.0f * blk_sum(pa, redv) / (3.0f * fn);
    if (alt > est) est = alt;
    if (tid == 0) {
        double prod = (double)n * (double)(*norm1) * (double)est;
        double k0 = (isfinite(prod) && prod > 0.0) ? 0.5 * log10(prod) : __longlong_as_double(0x7ff0000000000000ll);
        *kappa0 = k0;
        *chosen = prec_from_kappa0(k0);
    }
}

__global__ void k_err_to_info(const int32_t* __restrict__ err, int32_t* __restrict__ info) {
    if (*err != 0 && *info == 0) *info = -2;
}

struct CondLayout {
    size_t g, norm, info, err, gemm, gemm_bytes, z, total;
    bool tc;
    int64_t ldz;
};

// G on the tensor cores (BF16 pieces of the FP32-rounded columns, one GEMM)
// where the sketch GEMM is enabled, else the FP32 CUDA-core split-K GEMM.
static CondLayout cond_layout(int64_t m, int64_t n, int num_sms) {
    CondLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    L.tc = tensor_core_sketch_enabled() && sketch_tc_supported(LSQ_BF16);
    L.g = take(sizeof(float) * (size_t)n * n);
    L.norm = take(sizeof(float));
    L.info = take(sizeof(int32_t));
    L.err = take(sizeof(int32_t));
    if (L.tc) {
        L.ldz = align_up((size_t)m, 16);
        L.z = take(sizeof(uint16_t) * 7 * (size_t)L.ldz * n);
        L.gemm_bytes = sketch_tc_ws_bytes(n, n, 6 * L.ldz, LSQ_BF16, num_sms);
    } else {
        L.gemm_bytes = gemm_kmajor_ws_bytes(plan_gemm_kmajor(n, n, m, true, LSQ_FP32, num_sms));
    }
    L.gemm = take(L.gemm_bytes);
    L.total = off + 256;
    return L;
}

size_t condest_ws_bytes(int64_t m, int64_t n, int num_sms) { return cond_layout(m, n, num_sms).total; }

lsq_status launch_condest(const double* A, int64_t m, int64_t n, int64_t lda, double* kappa0, int32_t* chosen,
                          void* ws, size_t ws_bytes, int num_sms, cudaStream_t st) {
    CondLayout L = cond_layout(m, n, num_sms);
    char* base = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    if (!ws || L.total > ws_bytes) return LSQ_ERR_NOMEM;
    float* G = (float*)(base + L.g);
    float* nrm = (float*)(base + L.norm);
    int32_t* cinfo = (int32_t*)(base + L.info);
    lsq_status r;
    if (L.tc) {
        uint16_t* Z = (uint16_t*)(base + L.z);
        int32_t* err = (int32_t*)(base + L.err);
        LSQ_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int32_t), st));
        if ((r = launch_gram_split3<double>(A, m, n, lda, L.ldz, Z, st)) != LSQ_OK) return r;
        r = launch_sketch_tc(Z, 7 * L.ldz, Z + L.ldz, 7 * L.ldz, LSQ_BF16, n, n, 6 * L.ldz, G, n, base + L.gemm,
                             L.gemm_bytes, err, st);
    } else {
        GemmPlan gp = plan_gemm_kmajor(n, n, m, true, LSQ_FP32, num_sms);
        r = launch_gemm_kmajor(gp, A, LSQ_FP64, lda, A, LSQ_FP64, lda, G, n, base + L.gemm, st);
    }
    if (r != LSQ_OK) return r;
    // row-sharded A: A^T A summed over the shards
    if ((r = reduce_partial(G, n * n, LSQ_REDUCE_SUM_F32, st)) != LSQ_OK) return r;
    k_norm1<<<1, 1024, 0, st>>>(G, n, n, nrm);
    LSQ_LAUNCH_CHECK();
    LSQ_CUDA_TRY(cudaMemsetAsync(cinfo, 0, sizeof(int32_t), st));
    r = launch_cholesky<float>(G, n, n, cinfo, st);
    if (r != LSQ_OK) return r;
    if (L.tc) {
        // a timed-out tensor-core pipeline leaves no estimate: the overflow case (FP64)
        k_err_to_info<<<1, 1, 0, st>>>((const int32_t*)(base + L.err), cinfo);
        LSQ_LAUNCH_CHECK();
    }
    size_t smem = sizeof(float) * 4 * (size_t)n;
    if (smem > 200 * 1024) return LSQ_ERR_ARG;
    if (smem > 48 * 1024) LSQ_CUDA_TRY(cudaFuncSetAttribute(k_hager, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_hager<<<1, 512, smem, st>>>(G, n, n, nrm, cinfo, kappa0, chosen);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

// ---------------------------------------------------------------------------
// Estimate on the sketch (precision code LSQ_AUTO_SKETCH): the estimator
// above applied to G_s = A_e^T A_e of an FP32 sketch A_e = Omega_e A, with
// G_s^{-1} applied through L = R_e^T from the FP32 QR of A_e (R_e^T R_e =
// G_s) instead of an FP32 Cholesky of G_s, which breaks down once
// kappa(A)^2 > 1/u32.  The caller has computed A_e, R_e (unscaled), the
// FP32 judge of R_e (accept = u32 kappa_1(R_e) <= 1, Lemma rscond for the
// FP32 factor itself) and G_s of the scaled sketch.
// ---------------------------------------------------------------------------
// G_s of the scaled sketch -> G_s of A: entry (p, q) times 2^-(e_p + e_q) (exact)
__global__ void k_unscale_gram(float* __restrict__ G, int64_t n, const int32_t* __restrict__ e) {
    const int64_t total = n * n;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q % n, j = q / n;
        G[q] = ldexpf(G[q], -(e[i] + e[j]));
    }
}

// L = R^T in FP32 (lower, ld n), zero above the diagonal
__global__ void k_lower_from_upper(const double* __restrict__ R, int64_t n, int64_t ldr, float* __restrict__ L) {
    const int64_t total = n * n;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q % n, j = q / n;
        L[q] = i >= j ? (float)R[j + i * ldr] : 0.0f;
    }
}

// An FP32 factor that does not resolve A gives no estimate: kappa0 = +inf (FP64).
__global__ void k_sketch_guard(const int32_t* __restrict__ accept, double* __restrict__ kappa0,
                               int32_t* __restrict__ chosen) {
    if (!*accept) {
        *kappa0 = __longlong_as_double(0x7ff0000000000000ll);
        *chosen = LSQ_FP64;
    }
}

size_t condest_sketch_finish_ws_bytes(int64_t n) {
    return align_up(sizeof(float) * (size_t)n * n, 256) + 512;
}

lsq_status launch_condest_sketch_finish(float* G, const int32_t* colexp, const double* Re, int64_t n, int64_t ldr,
                                        const int32_t* accept, double* kappa0, int32_t* chosen, void* ws,
                                        size_t ws_bytes, cudaStream_t st) {
    if (!ws || ws_bytes < condest_sketch_finish_ws_bytes(n)) return LSQ_ERR_NOMEM;
    char* base = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    float* L = (float*)base;
    float* nrm = (float*)(base + align_up(sizeof(float) * (size_t)n * n, 256));
    int32_t* cinfo = (int32_t*)(nrm + 1);
    const unsigned g = (unsigned)std::min<int64_t>(ceil_div(n * n, 256), 8192);
    if (colexp) {
        k_unscale_gram<<<g, 256, 0, st>>>(G, n, colexp);
        LSQ_LAUNCH_CHECK();
    }
    k_norm1<<<1, 1024, 0, st>>>(G, n, n, nrm);
    LSQ_LAUNCH_CHECK();
    k_lower_from_upper<<<g, 256, 0, st>>>(Re, n, ldr, L);
    LSQ_LAUNCH_CHECK();
    LSQ_CUDA_TRY(cudaMemsetAsync(cinfo, 0, sizeof(int32_t), st));
    size_t smem = sizeof(float) * 4 * (size_t)n;
    if (smem > 200 * 1024) return LSQ_ERR_ARG;
    if (smem > 48 * 1024) LSQ_CUDA_TRY(cudaFuncSetAttribute(k_hager, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_hager<<<1, 512, smem, st>>>(L, n, n, nrm, cinfo, kappa0, chosen);
    LSQ_LAUNCH_CHECK();
    k_sketch_guard<<<1, 1, 0, st>>>(accept, kappa0, chosen);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

}  // namespace lsq
