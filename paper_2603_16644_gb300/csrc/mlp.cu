// Learned precision proposal (not part of the paper's method; it proposes the
// u_p of Alg. 1 and is checked by a condition estimate):
//   - features of A: column-norm statistics and the diagonal of the
//     preconditioner from an FP8-e4m3 sparse-sign sketch with an FP32 QR;
//   - an MLP d -> 64 -> 64 -> 64 -> 4 (ReLU, softmax cross-entropy) in FP32:
//     forward, backward (per-sample deltas, then per-parameter sums over the
//     batch in sample order: deterministic) and Adam;
//   - the judge: Hager's 1-norm estimate (Sec. 6.1's estimator, single
//     precision, csrc/hager.cu) of kappa_1(R_s) for a computed
//     preconditioner; a precision
//     u_p is accepted when u_p * kappa_1(R_s) <= 1, the regime of Lemma
//     rscond (eps * kappa(R_s) < 1).
#include "common.cuh"
#include "kernels.cuh"

#include <algorithm>

namespace lsq {

constexpr int MH = 64;   // hidden width
constexpr int MC = 4;    // classes: FP8-e4m3, BF16, FP32, FP64
constexpr int NFEAT = 10;

__host__ __device__ inline int64_t mlp_params(int d) { return (int64_t)MH * d + MH + 2 * ((int64_t)MH * MH + MH) + (int64_t)MC * MH + MC; }

struct MlpPtrs {
    const float *W1, *b1, *W2, *b2, *W3, *b3, *W4, *b4;
};

__device__ inline MlpPtrs mlp_ptrs(const float* p, int d) {
    MlpPtrs q;
    q.W1 = p;
    q.b1 = q.W1 + MH * d;
    q.W2 = q.b1 + MH;
    q.b2 = q.W2 + MH * MH;
    q.W3 = q.b2 + MH;
    q.b3 = q.W3 + MH * MH;
    q.W4 = q.b3 + MH;
    q.b4 = q.W4 + MC * MH;
    return q;
}

// Forward for one sample; z1..z3 are the pre-activations (kept for backward).
__device__ void mlp_fwd1(const MlpPtrs& P, int d, const float* x, float* z1, float* z2, float* z3, float* z4) {
    for (int o = 0; o < MH; ++o) {
        float a = P.b1[o];
        for (int i = 0; i < d; ++i) a = fmaf(P.W1[o * d + i], x[i], a);
        z1[o] = a;
    }
    for (int o = 0; o < MH; ++o) {
        float a = P.b2[o];
        for (int i = 0; i < MH; ++i) a = fmaf(P.W2[o * MH + i], fmaxf(z1[i], 0.0f), a);
        z2[o] = a;
    }
    for (int o = 0; o < MH; ++o) {
        float a = P.b3[o];
        for (int i = 0; i < MH; ++i) a = fmaf(P.W3[o * MH + i], fmaxf(z2[i], 0.0f), a);
        z3[o] = a;
    }
    for (int c = 0; c < MC; ++c) {
        float a = P.b4[c];
        for (int i = 0; i < MH; ++i) a = fmaf(P.W4[c * MH + i], fmaxf(z3[i], 0.0f), a);
        z4[c] = a;
    }
}

__global__ void k_mlp_forward(const float* __restrict__ params, int d, int batch, const float* __restrict__ X,
                              float* __restrict__ logits) {
    extern __shared__ float sp[];
    int64_t np = mlp_params(d);
    for (int64_t q = threadIdx.x; q < np; q += blockDim.x) sp[q] = params[q];
    __syncthreads();
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= batch) return;
    MlpPtrs P = mlp_ptrs(sp, d);
    float z1[MH], z2[MH], z3[MH], z4[MC];
    mlp_fwd1(P, d, X + (int64_t)s * d, z1, z2, z3, z4);
    for (int c = 0; c < MC; ++c) logits[(int64_t)s * MC + c] = z4[c];
}

// Per-sample deltas and activations for the gradient; per-sample loss.
// Row s of `act` holds h1 | h2 | h3 (3 x 64) and of `del` d1 | d2 | d3 | d4.
__global__ void k_mlp_delta(const float* __restrict__ params, int d, int batch, const float* __restrict__ X,
                            const int32_t* __restrict__ labels, float* __restrict__ act, float* __restrict__ del,
                            float* __restrict__ loss_s) {
    extern __shared__ float sp[];
    int64_t np = mlp_params(d);
    for (int64_t q = threadIdx.x; q < np; q += blockDim.x) sp[q] = params[q];
    __syncthreads();
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= batch) return;
    MlpPtrs P = mlp_ptrs(sp, d);
    float z1[MH], z2[MH], z3[MH], z4[MC];
    mlp_fwd1(P, d, X + (int64_t)s * d, z1, z2, z3, z4);
    float mx = z4[0];
    for (int c = 1; c < MC; ++c) mx = fmaxf(mx, z4[c]);
    float se = 0.0f;
    for (int c = 0; c < MC; ++c) se += expf(z4[c] - mx);
    int y = labels[s];
    loss_s[s] = -(z4[y] - mx - logf(se));
    float* A = act + (int64_t)s * 3 * MH;
    float* D = del + (int64_t)s * (3 * MH + MC);
    float d4[MC];
    for (int c = 0; c < MC; ++c) {
        d4[c] = (expf(z4[c] - mx) / se - (c == y ? 1.0f : 0.0f)) / (float)batch;
        D[3 * MH + c] = d4[c];
    }
    float d3[MH], d2[MH];
    for (int i = 0; i < MH; ++i) {
        float t = 0.0f;
        for (int c = 0; c < MC; ++c) t = fmaf(P.W4[c * MH + i], d4[c], t);
        d3[i] = z3[i] > 0.0f ? t : 0.0f;
    }
    for (int i = 0; i < MH; ++i) {
        float t = 0.0f;
        for (int o = 0; o < MH; ++o) t = fmaf(P.W3[o * MH + i], d3[o], t);
        d2[i] = z2[i] > 0.0f ? t : 0.0f;
    }
    for (int i = 0; i < MH; ++i) {
        float t = 0.0f;
        for (int o = 0; o < MH; ++o) t = fmaf(P.W2[o * MH + i], d2[o], t);
        D[i] = z1[i] > 0.0f ? t : 0.0f;  // d1
        D[MH + i] = d2[i];
        D[2 * MH + i] = d3[i];
        A[i] = fmaxf(z1[i], 0.0f);
        A[MH + i] = fmaxf(z2[i], 0.0f);
        A[2 * MH + i] = fmaxf(z3[i], 0.0f);
    }
}

// One thread per parameter: sum of delta x activation over the batch in order.
__global__ void k_mlp_grad(int d, int batch, const float* __restrict__ X, const float* __restrict__ act,
                           const float* __restrict__ del, const float* __restrict__ loss_s, float* __restrict__ grad,
                           float* __restrict__ loss) {
    int64_t np = mlp_params(d);
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q == 0 && loss) {
        float t = 0.0f;
        for (int s = 0; s < batch; ++s) t += loss_s[s];
        *loss = t / (float)batch;
    }
    if (q >= np) return;
    const int DS = 3 * MH + MC, AS = 3 * MH;
    // locate q in the packing: W1 b1 W2 b2 W3 b3 W4 b4
    int64_t off = q;
    int layer, o, i;
    bool bias;
    int64_t sizes[8] = {(int64_t)MH * d, MH, MH * MH, MH, MH * MH, MH, MC * MH, MC};
    int blk = 0;
    while (off >= sizes[blk]) { off -= sizes[blk]; ++blk; }
    layer = blk / 2;
    bias = (blk % 2) == 1;
    int in = layer == 0 ? d : MH;
    if (bias) { o = (int)off; i = -1; } else { o = (int)(off / in); i = (int)(off % in); }
    float t = 0.0f;
    for (int s = 0; s < batch; ++s) {
        const float* D = del + (int64_t)s * DS;
        float dl = layer < 3 ? D[layer * MH + o] : D[3 * MH + o];
        float a;
        if (bias) a = 1.0f;
        else if (layer == 0) a = X[(int64_t)s * d + i];
        else a = act[(int64_t)s * AS + (layer - 1) * MH + i];
        t = fmaf(dl, a, t);
    }
    grad[q] = t;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, int64_t count, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= count) return;
    float gq = g[q];
    float a = b1 * m1[q] + (1.0f - b1) * gq;
    float v = b2 * m2[q] + (1.0f - b2) * gq * gq;
    m1[q] = a;
    m2[q] = v;
    p[q] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
}

// ---------------------------------------------------------------------------
// Features (see the oracle for the definitions), one block.
// ---------------------------------------------------------------------------
__global__ void k_colnorm2(const double* __restrict__ A, int64_t m, int64_t lda, double* __restrict__ out) {
    int64_t c = blockIdx.x;
    const double* col = A + c * lda;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) s = fma(col[i], col[i], s);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    __shared__ double w[32];
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += w[q];
        out[c] = t;
    }
}

__global__ void k_features(const double* __restrict__ cn2, const double* __restrict__ Rs, int64_t ldr, int64_t m,
                           int64_t n, float* __restrict__ f) {
    if (threadIdx.x != 0) return;
    double cmax = -1e300, cmin = 1e300, cmean = 0, dmax = -1e300, dmin = 1e300, dmean = 0, fro = 0;
    for (int64_t j = 0; j < n; ++j) {
        double cn = log10(fmax(sqrt(cn2[j]), 1e-300));
        double dj = log10(fmax(fabs(Rs[j + j * ldr]), 1e-300));
        fro += cn2[j];
        cmax = fmax(cmax, cn); cmin = fmin(cmin, cn); cmean += cn;
        dmax = fmax(dmax, dj); dmin = fmin(dmin, dj); dmean += dj;
    }
    cmean /= n;
    dmean /= n;
    double cvar = 0, dvar = 0, sxy = 0, sxx = 0;
    int64_t q0 = n - (n + 3) / 4;
    double tmax = -1e300, tmin = 1e300;
    int64_t small = 0;
    for (int64_t j = 0; j < n; ++j) {
        double cn = log10(fmax(sqrt(cn2[j]), 1e-300));
        double dj = log10(fmax(fabs(Rs[j + j * ldr]), 1e-300));
        double t = (double)j / (double)n - 0.5 * (double)(n - 1) / (double)n;
        cvar += (cn - cmean) * (cn - cmean);
        dvar += (dj - dmean) * (dj - dmean);
        sxy += t * (dj - dmean);
        sxx += t * t;
        if (j >= q0) { tmax = fmax(tmax, dj); tmin = fmin(tmin, dj); }
        small += (dj < dmax - 2.0);
    }
    f[0] = (float)(log2((double)m) / 16.0);
    f[1] = (float)(log2((double)n) / 10.0);
    f[2] = (float)(cmax - cmin);
    f[3] = (float)sqrt(cvar / n);
    f[4] = (float)(dmax - dmin);
    f[5] = (float)sqrt(dvar / n);
    f[6] = (float)(sxx > 0 ? sxy / sxx : 0.0);
    f[7] = (float)(tmax - tmin);
    f[8] = (float)((double)small / (double)n);
    f[9] = (float)(dmin - log10(fmax(sqrt(fro / (double)n), 1e-300)));
}

// Proposal: logits of one feature vector -> class -> precision code.
__global__ void k_propose(const float* __restrict__ logits, int32_t* __restrict__ prec, float* __restrict__ probs) {
    if (threadIdx.x != 0) return;
    int best = 0;
    float mx = logits[0];
    for (int c = 1; c < MC; ++c)
        if (logits[c] > mx) { mx = logits[c]; best = c; }
    const int32_t map[MC] = {LSQ_FP8_E4M3, LSQ_BF16, LSQ_FP32, LSQ_FP64};
    *prec = map[best];
    if (probs) {
        float se = 0.0f;
        for (int c = 0; c < MC; ++c) se += expf(logits[c] - mx);
        for (int c = 0; c < MC; ++c) probs[c] = expf(logits[c] - mx) / se;
    }
}

// ---------------------------------------------------------------------------
// Judge: Hager's estimate of ||R^{-1}||_1 (R upper, FP32 copy), times ||R||_1.
// ---------------------------------------------------------------------------
__global__ void k_to_f32_upper(const double* __restrict__ R, int64_t n, int64_t ldr, float* __restrict__ Rf) {
    int64_t total = n * n;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = q % n, j = q / n;
        Rf[q] = i <= j ? __double2float_rn(R[i + j * ldr]) : 0.0f;
    }
}

// kappa_1(R) = ||R||_1 gamma (gamma ~ ||R^{-1}||_1) and the judgement
// u_p kappa_1(R) <= 1; a non-finite value or a timed-out solve rejects.
__global__ void k_judge_final(const float* __restrict__ rnorm, const float* __restrict__ gamma,
                              const int32_t* __restrict__ err, int prec, int32_t* __restrict__ accept,
                              double* __restrict__ kappa1) {
    const double k1 = (double)(*rnorm) * (double)(*gamma);
    const double u = prec == LSQ_FP8_E4M3 ? 0x1p-4 : prec == LSQ_BF16 ? 0x1p-8 : prec == LSQ_FP16 ? 0x1p-11
                   : prec == LSQ_FP32 ? 0x1p-24 : 0x1p-53;
    const bool finite = isfinite(k1) && k1 > 0.0 && *err == 0;
    *kappa1 = finite ? k1 : __longlong_as_double(0x7ff0000000000000ll);
    *accept = (finite && u * k1 <= 1.0) ? 1 : 0;
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
lsq_status launch_mlp_forward(const float* params, int d, int batch, const float* X, float* logits, cudaStream_t st) {
    size_t smem = sizeof(float) * (size_t)mlp_params(d);
    if (smem > 200 * 1024) return LSQ_ERR_ARG;
    if (smem > 48 * 1024) LSQ_CUDA_TRY(cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_mlp_forward<<<(unsigned)ceil_div(batch, 64), 64, smem, st>>>(params, d, batch, X, logits);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

size_t mlp_backward_ws_bytes(int d, int batch) {
    return align_up(sizeof(float) * (size_t)batch * (3 * MH), 256) + align_up(sizeof(float) * (size_t)batch * (3 * MH + MC), 256) +
           align_up(sizeof(float) * (size_t)batch, 256) + 256;
}

lsq_status launch_mlp_backward(const float* params, int d, int batch, const float* X, const int32_t* labels,
                               float* grad, float* loss, void* ws, size_t ws_bytes, cudaStream_t st) {
    if (ws_bytes < mlp_backward_ws_bytes(d, batch) || !ws) return LSQ_ERR_NOMEM;
    char* base = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    float* act = (float*)base;
    float* del = (float*)(base + align_up(sizeof(float) * (size_t)batch * (3 * MH), 256));
    float* ls = (float*)((char*)del + align_up(sizeof(float) * (size_t)batch * (3 * MH + MC), 256));
    size_t smem = sizeof(float) * (size_t)mlp_params(d);
    if (smem > 200 * 1024) return LSQ_ERR_ARG;
    if (smem > 48 * 1024) LSQ_CUDA_TRY(cudaFuncSetAttribute(k_mlp_delta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_mlp_delta<<<(unsigned)ceil_div(batch, 64), 64, smem, st>>>(params, d, batch, X, labels, act, del, ls);
    LSQ_LAUNCH_CHECK();
    int64_t np = mlp_params(d);
    k_mlp_grad<<<(unsigned)ceil_div(np, 128), 128, 0, st>>>(d, batch, X, act, del, ls, grad, loss);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

lsq_status launch_adam(float* p, const float* g, float* m1, float* m2, int64_t count, float lr, float b1, float b2,
                       float eps, int step, cudaStream_t st) {
    float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    k_adam<<<(unsigned)ceil_div(count, 256), 256, 0, st>>>(p, g, m1, m2, count, lr, b1, b2, eps, c1, c2);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

lsq_status launch_colnorm2(const double* A, int64_t m, int64_t n, int64_t lda, double* out, cudaStream_t st) {
    k_colnorm2<<<(unsigned)n, 256, 0, st>>>(A, m, lda, out);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

lsq_status launch_features_finish(const double* cn2, const double* Rs, int64_t ldr, int64_t m, int64_t n, float* f,
                                  cudaStream_t st) {
    k_features<<<1, 32, 0, st>>>(cn2, Rs, ldr, m, n, f);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

lsq_status launch_propose(const float* logits, int32_t* prec, float* probs, cudaStream_t st) {
    k_propose<<<1, 32, 0, st>>>(logits, prec, probs);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

size_t judge_ws_bytes(int64_t n) { return align_up(sizeof(float) * (size_t)n * n, 256) + 256 + hager_ws_bytes(n) + 256; }

lsq_status launch_judge(const double* Rs, int64_t n, int64_t ldr, int prec, int32_t* accept, double* kappa1, void* ws,
                        size_t ws_bytes, cudaStream_t st) {
    if (!ws || ws_bytes < judge_ws_bytes(n)) return LSQ_ERR_NOMEM;
    float* Rf = (float*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    char* small = (char*)Rf + align_up(sizeof(float) * (size_t)n * n, 256);
    float* rnorm = (float*)small;
    float* gam = (float*)(small + 4);
    int32_t* herr = (int32_t*)(small + 8);
    k_to_f32_upper<<<(unsigned)std::min<int64_t>(ceil_div(n * n, 256), 4096), 256, 0, st>>>(Rs, n, ldr, Rf);
    LSQ_LAUNCH_CHECK();
    lsq_status r;
    if ((r = launch_colnorm1_max(Rf, n, n, true, rnorm, st)) != LSQ_OK) return r;
    LSQ_CUDA_TRY(cudaMemsetAsync(herr, 0, sizeof(int32_t), st));
    if ((r = hager_inv_norm1(Rf, n, n, true, nullptr, gam, herr, small + 256, hager_ws_bytes(n), st)) != LSQ_OK)
        return r;
    k_judge_final<<<1, 1, 0, st>>>(rnorm, gam, herr, prec, accept, kappa1);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

int64_t mlp_param_count_host(int d) { return mlp_params(d); }
int mlp_num_features() { return NFEAT; }

}  // namespace lsq
