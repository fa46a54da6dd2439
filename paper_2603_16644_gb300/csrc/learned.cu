// C-ABI of the learned precision proposal and its judges (not in the
// paper), and of the PNE solve that uses them.  The paper's own estimator of
// Sec. 6.1 (here on the Gram of a sketch, lsq_condest_sketch) judges every
// proposal that could lose accuracy (any precision below FP64) and is the
// fallback when it rejects one; the FP32 Hager estimate of kappa_1(R_s) of
// the computed preconditioner (Lemma rscond) is a second opinion.
#include "common.cuh"
#include "kernels.cuh"

#include <algorithm>

namespace lsq {
lsq_status launch_mlp_forward(const float* params, int d, int batch, const float* X, float* logits, cudaStream_t st);
size_t mlp_backward_ws_bytes(int d, int batch);
lsq_status launch_mlp_backward(const float* params, int d, int batch, const float* X, const int32_t* labels,
                               float* grad, float* loss, void* ws, size_t ws_bytes, cudaStream_t st);
lsq_status launch_adam(float* p, const float* g, float* m1, float* m2, int64_t count, float lr, float b1, float b2,
                       float eps, int step, cudaStream_t st);
lsq_status launch_colnorm2(const double* A, int64_t m, int64_t n, int64_t lda, double* out, cudaStream_t st);
lsq_status launch_features_finish(const double* cn2, const double* Rs, int64_t ldr, int64_t m, int64_t n, float* f,
                                  cudaStream_t st);
lsq_status launch_propose(const float* logits, int32_t* prec, float* probs, cudaStream_t st);
size_t judge_ws_bytes(int64_t n);
lsq_status launch_judge(const double* Rs, int64_t n, int64_t ldr, int prec, int32_t* accept, double* kappa1, void* ws,
                        size_t ws_bytes, cudaStream_t st);
int64_t mlp_param_count_host(int d);
int mlp_num_features();
lsq_status solve_impl_ext(bool hpne, const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
                          const lsq_opts* o, double* x, double* Rs_out, int32_t* info, void* ws, size_t ws_bytes,
                          cudaStream_t st, const double* Rs_in);
size_t solve_ws_bytes_ext(int64_t m, int64_t n, const lsq_opts* o, bool hpne);
}  // namespace lsq

using namespace lsq;

namespace {

struct Off {
    size_t off = 0;
    size_t take(size_t bytes) {
        size_t o = off;
        off = align_up(off + std::max<size_t>(bytes, 1), 256);
        return o;
    }
};

lsq_opts feature_opts(int64_t m, int64_t n, uint64_t seed) {
    lsq_opts o{};
    o.kind = LSQ_SPARSE_SIGN;
    o.s = std::min<int64_t>(2 * n, m);
    o.zeta = (int32_t)std::min<int64_t>(8, o.s);
    o.seed = seed;
    o.sketch_prec = LSQ_FP8_E4M3;
    o.qr_prec = LSQ_FP32;
    return o;
}

struct FeatLayout {
    size_t sk, as_, ce, qr, rs, cn2, info, f, logits, total;
    size_t sk_bytes, qr_bytes;
};

FeatLayout feat_layout(int64_t m, int64_t n, uint64_t seed) {
    FeatLayout L{};
    Off q;
    lsq_opts o = feature_opts(m, n, seed);
    L.sk_bytes = lsq_workspace_size(LSQ_OP_SKETCH, m, n, &o);
    L.qr_bytes = lsq_workspace_size(LSQ_OP_PRECOND_QR, o.s, n, nullptr);
    L.sk = q.take(L.sk_bytes);
    L.as_ = q.take(sizeof(float) * (size_t)o.s * n);
    L.ce = q.take(sizeof(int32_t) * n);
    L.qr = q.take(L.qr_bytes);
    L.rs = q.take(sizeof(double) * (size_t)n * n);
    L.cn2 = q.take(sizeof(double) * n);
    L.info = q.take(sizeof(int32_t));
    L.f = q.take(sizeof(float) * 16);
    L.logits = q.take(sizeof(float) * 8);
    L.total = q.off + 256;
    return L;
}

char* aligned(void* p) { return (char*)(((uintptr_t)p + 255) & ~(uintptr_t)255); }

lsq_status features_impl(const double* A, int64_t m, int64_t n, int64_t lda, uint64_t seed, float* f, char* base,
                         const FeatLayout& L, cudaStream_t st) {
    lsq_opts o = feature_opts(m, n, seed);
    float* As = (float*)(base + L.as_);
    int32_t* ce = (int32_t*)(base + L.ce);
    double* Rs = (double*)(base + L.rs);
    int32_t* info = (int32_t*)(base + L.info);
    lsq_status r = lsq_sketch(A, m, n, lda, &o, As, o.s, ce, nullptr, base + L.sk, L.sk_bytes, st);
    if (r != LSQ_OK) return r;
    r = lsq_precond_qr(As, o.s, n, o.s, LSQ_FP32, LSQ_FP32, ce, Rs, n, info, base + L.qr, L.qr_bytes, st);
    if (r != LSQ_OK) return r;
    if ((r = launch_colnorm2(A, m, n, lda, (double*)(base + L.cn2), st)) != LSQ_OK) return r;
    return launch_features_finish((double*)(base + L.cn2), Rs, n, m, n, f, st);
}

struct LearnLayout {
    FeatLayout F;
    size_t feat, judge, small, as_, ce, sk, qr, rs, est, solve, total;
    size_t judge_bytes, sk_bytes, qr_bytes, est_bytes, solve_bytes;
};

LearnLayout learn_layout(int64_t m, int64_t n, const lsq_opts* o) {
    LearnLayout L{};
    Off q;
    L.F = feat_layout(m, n, o->seed);
    L.feat = q.take(L.F.total);
    L.judge_bytes = judge_ws_bytes(n);
    L.judge = q.take(L.judge_bytes);
    L.small = q.take(256);
    lsq_opts o64 = *o;
    o64.sketch_prec = LSQ_FP32;  // the judged preconditioners are at most FP32
    o64.qr_prec = LSQ_FP32;
    L.sk_bytes = lsq_workspace_size(LSQ_OP_SKETCH, m, n, &o64);
    L.sk = q.take(L.sk_bytes);
    L.as_ = q.take(sizeof(float) * (size_t)o->s * n);
    L.ce = q.take(sizeof(int32_t) * n);
    L.qr_bytes = lsq_workspace_size(LSQ_OP_PRECOND_QR, o->s, n, nullptr);
    L.qr = q.take(L.qr_bytes);
    L.rs = q.take(sizeof(double) * (size_t)n * n);
    L.est_bytes = lsq_workspace_size(LSQ_OP_CONDEST_SKETCH, m, n, nullptr);
    L.est = q.take(L.est_bytes);
    lsq_opts oa = *o;
    oa.sketch_prec = LSQ_AUTO;  // widest layout
    L.solve_bytes = solve_ws_bytes_ext(m, n, &oa, false);
    L.solve = q.take(L.solve_bytes);
    L.total = q.off + 256;
    return L;
}

int next_precision(int p) {
    switch (p) {
    case LSQ_FP8_E4M3: return LSQ_BF16;
    case LSQ_BF16: return LSQ_FP32;
    case LSQ_FP16: return LSQ_FP32;
    default: return LSQ_FP64;
    }
}

}  // namespace

extern "C" {

int64_t lsq_mlp_param_count(int32_t d) { return d > 0 ? mlp_param_count_host(d) : 0; }

int32_t lsq_mlp_num_features(void) { return mlp_num_features(); }

size_t lsq_features_workspace_size(int64_t m, int64_t n) {
    if (m <= 0 || n <= 0) return 0;
    return feat_layout(m, n, 0).total + 256;
}

lsq_status lsq_features(const double* A, int64_t m, int64_t n, int64_t lda, uint64_t seed, float* f, void* ws,
                        size_t ws_bytes, void* stream) {
    if (!A || !f || m <= 0 || n <= 0 || lda < m || m < n) return LSQ_ERR_ARG;
    FeatLayout L = feat_layout(m, n, seed);
    if (!ws || L.total + 256 > ws_bytes) return LSQ_ERR_NOMEM;
    return features_impl(A, m, n, lda, seed, f, aligned(ws), L, (cudaStream_t)stream);
}

lsq_status lsq_mlp_forward(const float* params, int32_t d, int32_t batch, const float* X, float* logits,
                           void* stream) {
    if (!params || !X || !logits || d <= 0 || batch <= 0) return LSQ_ERR_ARG;
    return launch_mlp_forward(params, d, batch, X, logits, (cudaStream_t)stream);
}

size_t lsq_mlp_backward_workspace_size(int32_t d, int32_t batch) {
    return d > 0 && batch > 0 ? mlp_backward_ws_bytes(d, batch) : 0;
}

lsq_status lsq_mlp_backward(const float* params, int32_t d, int32_t batch, const float* X, const int32_t* labels,
                            float* grad, float* loss, void* ws, size_t ws_bytes, void* stream) {
    if (!params || !X || !labels || !grad || d <= 0 || batch <= 0) return LSQ_ERR_ARG;
    return launch_mlp_backward(params, d, batch, X, labels, grad, loss, ws, ws_bytes, (cudaStream_t)stream);
}

lsq_status lsq_mlp_adam(float* params, const float* grad, float* m1, float* m2, int64_t count, float lr, float beta1,
                        float beta2, float eps, int32_t step, void* stream) {
    if (!params || !grad || !m1 || !m2 || count <= 0 || step < 1) return LSQ_ERR_ARG;
    return launch_adam(params, grad, m1, m2, count, lr, beta1, beta2, eps, step, (cudaStream_t)stream);
}

lsq_status lsq_propose_precision(const double* A, int64_t m, int64_t n, int64_t lda, uint64_t seed,
                                 const float* params, int32_t d, int32_t* prec, float* probs, void* ws,
                                 size_t ws_bytes, void* stream) {
    if (!A || !params || !prec || d != mlp_num_features() || m <= 0 || n <= 0 || lda < m || m < n) return LSQ_ERR_ARG;
    FeatLayout L = feat_layout(m, n, seed);
    if (!ws || L.total + 256 > ws_bytes) return LSQ_ERR_NOMEM;
    char* base = aligned(ws);
    cudaStream_t st = (cudaStream_t)stream;
    float* f = (float*)(base + L.f);
    float* logits = (float*)(base + L.logits);
    lsq_status r = features_impl(A, m, n, lda, seed, f, base, L, st);
    if (r != LSQ_OK) return r;
    if ((r = launch_mlp_forward(params, d, 1, f, logits, st)) != LSQ_OK) return r;
    return launch_propose(logits, prec, probs, st);
}

size_t lsq_judge_workspace_size(int64_t n) { return n > 0 ? judge_ws_bytes(n) + 256 : 0; }

lsq_status lsq_judge_preconditioner(const double* Rs, int64_t n, int64_t ldr, int32_t prec, int32_t* accept,
                                    double* kappa1, void* ws, size_t ws_bytes, void* stream) {
    if (!Rs || !accept || !kappa1 || n <= 0 || ldr < n || prec < LSQ_FP8_E4M3 || prec > LSQ_FP64) return LSQ_ERR_ARG;
    return launch_judge(Rs, n, ldr, prec, accept, kappa1, ws, ws_bytes, (cudaStream_t)stream);
}

size_t lsq_learned_workspace_size(int64_t m, int64_t n, const lsq_opts* opts) {
    if (!opts || m <= 0 || n <= 0 || opts->s < n || opts->s > m) return 0;
    return learn_layout(m, n, opts).total + 256;
}

lsq_status lsq_pne_solve_learned(const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
                                 const lsq_opts* opts, const float* params, int32_t d, double* x, int32_t* info,
                                 int32_t* used_prec, int32_t* escalations, void* ws, size_t ws_bytes, void* stream) {
    if (!A || !b || !opts || !params || !x || !info || !used_prec || !escalations || m <= 0 || n <= 0 || lda < m ||
        opts->s < n || opts->s > m || d != mlp_num_features())
        return LSQ_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    LearnLayout L = learn_layout(m, n, opts);
    if (!ws || L.total + 256 > ws_bytes) return LSQ_ERR_NOMEM;
    char* base = aligned(ws);
    char* fb = base + L.feat;
    int32_t* dprec = (int32_t*)(base + L.small);
    float* probs = (float*)(base + L.small + 16);
    int32_t* daccept = (int32_t*)(base + L.small + 64);
    double* dk1 = (double*)(base + L.small + 128);
    lsq_status r = lsq_propose_precision(A, m, n, lda, opts->seed, params, d, dprec, probs, fb, L.F.total + 256, st);
    if (r != LSQ_OK) return r;
    int32_t p = LSQ_FP64;
    LSQ_CUDA_TRY(cudaMemcpyAsync(&p, dprec, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    LSQ_CUDA_TRY(cudaStreamSynchronize(st));
    int esc = 0;
    float* As = (float*)(base + L.as_);
    int32_t* ce = (int32_t*)(base + L.ce);
    double* Rs = (double*)(base + L.rs);
    bool have_rs = false;
    lsq_opts o2 = *opts;
    if (p != LSQ_FP64) {
        // a proposal below FP64 could lose accuracy: the paper's estimator
        // judges it, and its own choice replaces a proposal below it
        double* dk0 = (double*)(base + L.small + 160);
        int32_t* dch = (int32_t*)(base + L.small + 192);
        if ((r = lsq_condest_sketch(A, m, n, lda, opts->seed, dk0, dch, base + L.est, L.est_bytes, st)) != LSQ_OK)
            return r;
        int32_t pe = LSQ_FP64;
        LSQ_CUDA_TRY(cudaMemcpyAsync(&pe, dch, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        LSQ_CUDA_TRY(cudaStreamSynchronize(st));
        if (pe < LSQ_FP8_E4M3 || pe > LSQ_FP64) pe = LSQ_FP64;
        if (pe > p) {  // precision codes rise with the precision
            p = pe;
            ++esc;
        }
    }
    while (p != LSQ_FP64) {
        // second opinion on the computed preconditioner: u_p kappa_1(R_s) <= 1
        o2.sketch_prec = p;
        o2.qr_prec = LSQ_FP32;
        if ((r = lsq_sketch(A, m, n, lda, &o2, As, o2.s, ce, nullptr, base + L.sk, L.sk_bytes, st)) != LSQ_OK) return r;
        if ((r = lsq_precond_qr(As, o2.s, n, o2.s, LSQ_FP32, LSQ_FP32, ce, Rs, n, info, base + L.qr, L.qr_bytes,
                                st)) != LSQ_OK)
            return r;
        if ((r = launch_judge(Rs, n, n, p, daccept, dk1, base + L.judge, L.judge_bytes, st)) != LSQ_OK) return r;
        int32_t acc = 0;
        LSQ_CUDA_TRY(cudaMemcpyAsync(&acc, daccept, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        LSQ_CUDA_TRY(cudaStreamSynchronize(st));
        if (acc) { have_rs = true; break; }
        p = next_precision(p);
        ++esc;
    }
    *used_prec = p;
    *escalations = esc;
    o2.sketch_prec = p;
    o2.qr_prec = p == LSQ_FP64 ? LSQ_FP64 : LSQ_FP32;
    return solve_impl_ext(false, A, m, n, lda, b, &o2, x, nullptr, info, base + L.solve, L.solve_bytes, st,
                          have_rs ? Rs : nullptr);
}

}  // extern "C"
