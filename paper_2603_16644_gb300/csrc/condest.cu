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

// kappa0 = 0.5 log10(n ||G||_1 gamma) in FP64 from the FP32 norm and estimate
// gamma of ||G^{-1}||_1, and the precision; the overflow case (a failed
// factorization, a timed-out wait, a non-finite value) gives +inf and FP64.
__global__ void k_condest_final(int64_t n, const float* __restrict__ norm1, const float* __restrict__ gamma,
                                const int32_t* __restrict__ fail, const int32_t* __restrict__ err,
                                double* __restrict__ kappa0, int32_t* __restrict__ chosen) {
    const double inf = __longlong_as_double(0x7ff0000000000000ll);
    double k0 = inf;
    if (*fail == 0 && (!err || *err == 0) && isfinite(*norm1) && isfinite(*gamma)) {
        const double prod = (double)n * (double)(*norm1) * (double)(*gamma);
        k0 = (isfinite(prod) && prod > 0.0) ? 0.5 * log10(prod) : inf;
    }
    *kappa0 = k0;
    *chosen = prec_from_kappa0(k0);
}

__global__ void k_err_to_info(const int32_t* __restrict__ err, int32_t* __restrict__ info) {
    if (*err != 0 && *info == 0) *info = -2;
}

struct CondLayout {
    size_t g, norm, info, err, gemm, gemm_bytes, z, gam, herr, hg, hg_bytes, total;
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
    L.gam = take(sizeof(float));
    L.herr = take(sizeof(int32_t));
    L.hg_bytes = hager_ws_bytes(n);
    L.hg = take(L.hg_bytes);
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
    if ((r = launch_colnorm1_max(G, n, n, false, nrm, st)) != LSQ_OK) return r;
    LSQ_CUDA_TRY(cudaMemsetAsync(cinfo, 0, sizeof(int32_t), st));
    r = launch_cholesky<float>(G, n, n, cinfo, st);
    if (r != LSQ_OK) return r;
    if (L.tc) {
        // a timed-out tensor-core pipeline leaves no estimate: the overflow case (FP64)
        k_err_to_info<<<1, 1, 0, st>>>((const int32_t*)(base + L.err), cinfo);
        LSQ_LAUNCH_CHECK();
    }
    // gamma ~ ||G^{-1}||_1 through the Cholesky factor (lower triangle of G)
    float* gam = (float*)(base + L.gam);
    int32_t* herr = (int32_t*)(base + L.herr);
    LSQ_CUDA_TRY(cudaMemsetAsync(herr, 0, sizeof(int32_t), st));
    if ((r = hager_inv_norm1(G, n, n, false, cinfo, gam, herr, base + L.hg, L.hg_bytes, st)) != LSQ_OK) return r;
    k_condest_final<<<1, 1, 0, st>>>(n, nrm, gam, cinfo, herr, kappa0, chosen);
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
    return align_up(sizeof(float) * (size_t)n * n, 256) + 256 + hager_ws_bytes(n) + 256;
}

lsq_status launch_condest_sketch_finish(float* G, const int32_t* colexp, const double* Re, int64_t n, int64_t ldr,
                                        const int32_t* accept, double* kappa0, int32_t* chosen, void* ws,
                                        size_t ws_bytes, cudaStream_t st) {
    if (!ws || ws_bytes < condest_sketch_finish_ws_bytes(n)) return LSQ_ERR_NOMEM;
    char* base = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    float* L = (float*)base;
    char* small = base + align_up(sizeof(float) * (size_t)n * n, 256);
    float* nrm = (float*)small;
    int32_t* cinfo = (int32_t*)(small + 4);
    float* gam = (float*)(small + 8);
    int32_t* herr = (int32_t*)(small + 12);
    char* hg = small + 256;
    const unsigned g = (unsigned)std::min<int64_t>(ceil_div(n * n, 256), 8192);
    if (colexp) {
        k_unscale_gram<<<g, 256, 0, st>>>(G, n, colexp);
        LSQ_LAUNCH_CHECK();
    }
    lsq_status r;
    if ((r = launch_colnorm1_max(G, n, n, false, nrm, st)) != LSQ_OK) return r;
    k_lower_from_upper<<<g, 256, 0, st>>>(Re, n, ldr, L);
    LSQ_LAUNCH_CHECK();
    LSQ_CUDA_TRY(cudaMemsetAsync(small + 4, 0, 12, st));  // cinfo, gamma, herr
    if ((r = hager_inv_norm1(L, n, n, false, cinfo, gam, herr, hg, hager_ws_bytes(n), st)) != LSQ_OK) return r;
    k_condest_final<<<1, 1, 0, st>>>(n, nrm, gam, cinfo, herr, kappa0, chosen);
    LSQ_LAUNCH_CHECK();
    k_sketch_guard<<<1, 1, 0, st>>>(accept, kappa0, chosen);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

}  // namespace lsq
