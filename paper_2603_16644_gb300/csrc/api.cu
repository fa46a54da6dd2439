// C-ABI entry points of liblsq (declared in include/lsq.h): argument checks,
// workspace layout and the sequence of kernels that implements Alg. 1.
#include "common.cuh"
#include "kernels.cuh"

#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

using namespace lsq;

namespace lsq {

static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// Pool of event pairs, one pair per (solve, stage) while profiling is on.
struct StageProf {
    std::mutex mu;
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t next = 0;
    struct Rec { int stage; size_t ev_begin, ev_end; double work; };
    std::vector<Rec> recs;
    size_t open_begin[ST_COUNT] = {};
    bool open[ST_COUNT] = {};
};
static StageProf g_prof;

static size_t prof_event() {
    if (g_prof.next >= g_prof.pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return (size_t)-1;
        g_prof.pool.push_back(e);
    }
    return g_prof.next++;
}

static std::atomic<int> g_last_cuda_error{0};

// Row-sharded solves: the caller's reduction of partial sums (none by default).
static lsq_reduce_fn g_reduce_fn = nullptr;
static void* g_reduce_user = nullptr;

lsq_status reduce_partial(void* buf, int64_t count, int kind, cudaStream_t st) {
    if (!g_reduce_fn) return LSQ_OK;
    int32_t r = g_reduce_fn(buf, count, kind, (void*)st, g_reduce_user);
    return r == LSQ_OK ? LSQ_OK : LSQ_ERR_CUDA;
}
void note_cuda_error(cudaError_t e) { g_last_cuda_error.store((int)e); }

void stage_mark(int stage, bool begin, cudaStream_t st, double work) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    if (!g_prof.on) return;
    size_t e = prof_event();
    if (e == (size_t)-1) return;
    cudaEventRecord(g_prof.pool[e], st);
    if (begin) {
        g_prof.open_begin[stage] = e;
        g_prof.open[stage] = true;
    } else if (g_prof.open[stage]) {
        g_prof.recs.push_back({stage, g_prof.open_begin[stage], e, work});
        g_prof.open[stage] = false;
    }
}

}  // namespace lsq

namespace {

// Gaussian sketches in FP8/BF16/FP16 run on the tensor cores unless switched
// off (lsq_set_tensor_core_sketch), which routes them to the CUDA-core GEMM.
bool g_tensor_core_sketch = true;
}  // namespace

namespace lsq {
bool tensor_core_sketch_enabled() { return g_tensor_core_sketch; }
}  // namespace lsq

namespace {

// The symmetric FP64 Gram of PNE (csrc/ozaki.cu) and the off-diagonal
// products of A_p = A R^{-1} (csrc/oz_trsm.cu) run as digit-sliced
// tensor-core products unless switched off (lsq_set_fp64_emulation).
bool g_fp64_emulation = true;

inline cudaStream_t S(void* p) { return reinterpret_cast<cudaStream_t>(p); }

}  // namespace

namespace lsq {
bool fp64_emulation_enabled() { return g_fp64_emulation; }
}  // namespace lsq

namespace {

bool valid_sketch_prec(int p) { return p >= LSQ_FP8_E4M3 && p <= LSQ_FP64; }
bool is_auto(int p) { return p == LSQ_AUTO || p == LSQ_AUTO_SKETCH; }

// Solution methods (Sec. 1, Sec. 5): PNE (Eq. e_pne), HPNE with LU or QR
// (Eq. e_hpne), seminormal equations (Eq. e_sne), not-normal equations with
// B = A U_s^{-1} (Eq. e_nne).
enum { M_PNE = 0, M_HPNE = 1, M_HPNE_QR = 2, M_SNE = 3, M_NNE = 4 };
// methods whose n x n system is A_p^T A (nonsymmetric) rather than A_p^T A_p
bool method_nonsym(int m) { return m == M_HPNE || m == M_HPNE_QR || m == M_NNE; }
// Workspaces of AUTO solves are laid out for the widest precision (FP64).
int layout_prec(int p) { return is_auto(p) ? LSQ_FP64 : p; }

lsq_status check_opts(const lsq_opts* o, int64_t m, int64_t n, bool allow_auto) {
    if (!o) return LSQ_ERR_ARG;
    if (o->kind != LSQ_GAUSSIAN && o->kind != LSQ_SPARSE_SIGN && o->kind != LSQ_SRFT) return LSQ_ERR_ARG;
    if (o->s < n || o->s > m || o->s > 0x7fffffff) return LSQ_ERR_ARG;
    if (o->kind == LSQ_SPARSE_SIGN && (o->zeta < 1 || o->zeta > 32 || o->zeta > o->s)) return LSQ_ERR_ARG;
    if (!valid_sketch_prec(o->sketch_prec) && !(allow_auto && is_auto(o->sketch_prec))) return LSQ_ERR_ARG;
    if (o->qr_prec != LSQ_FP32 && o->qr_prec != LSQ_FP64) return LSQ_ERR_ARG;
    if (o->refine_steps < 0 || o->refine_steps > 1) return LSQ_ERR_ARG;
    if (o->row_offset < 0 || (o->row_offset != 0 && o->kind == LSQ_SRFT)) return LSQ_ERR_ARG;
    return LSQ_OK;
}

// Byte offsets of every piece of scratch, from one routine so that the size
// query and the solver agree.
struct Off {
    size_t off = 0;
    size_t take(size_t bytes) {
        size_t o = off;
        off = align_up(off + std::max<size_t>(bytes, 1), 256);
        return o;
    }
};

struct SketchLayout {
    size_t colmax, colexp, ahat, idx, sgn, counts, rowptr, cursor, col, maxcount, err, om, gemm, total, gemm_bytes;
    int64_t ldq, ldo;
};

// Columns of Omega per digit-sliced product of the FP64 Gaussian sketch (the
// largest K whose digit-pair sums stay exact in FP32).
constexpr int64_t kSketchChunk = 1024;  // K chunk of the FP64 sketch (three-digit Omega)

// The Gaussian sketch on the tensor cores: FP64 by digit slicing (switch
// lsq_set_fp64_emulation), FP32 as BF16 pieces (lsq_set_tensor_core_sketch).
bool gauss_fp64_tc(int prec) { return prec == LSQ_FP64 && g_fp64_emulation && ot_trsm_supported(); }
bool gauss_fp32_tc(int prec) { return prec == LSQ_FP32 && g_tensor_core_sketch && sketch_tc_supported(LSQ_BF16); }

SketchLayout sketch_layout(int64_t m, int64_t n, int64_t s, int kind, int zeta, int prec, int sms) {
    SketchLayout L{};
    Off o;
    int es = prec_bytes(prec);
    L.ldq = align_up((size_t)m, 16);
    L.ldo = L.ldq;
    L.colmax = o.take(sizeof(unsigned long long) * n);
    L.colexp = o.take(sizeof(int32_t) * n);
    L.err = o.take(sizeof(int32_t));
    if (kind == LSQ_SPARSE_SIGN) {
        L.ahat = o.take((size_t)m * n * es);
        L.idx = o.take(sizeof(int32_t) * (size_t)m * zeta);
        L.sgn = o.take((size_t)m * zeta);
        L.counts = o.take(sizeof(int32_t) * (size_t)s);
        L.rowptr = o.take(sizeof(int32_t) * (size_t)(s + 1));
        L.cursor = o.take(sizeof(int32_t) * (size_t)s);
        L.col = o.take(sizeof(uint32_t) * (size_t)m * zeta);
        L.maxcount = o.take(sizeof(int32_t));
    } else if (kind == LSQ_SRFT) {
        // signed, zero-padded and transformed columns (m' x n)
        L.ahat = o.take(srft_ws_bytes(m, n, prec));
    } else if (gauss_fp64_tc(prec)) {
        // FP64: K chunks of Omega generated one at a time as the digit planes
        // of tensor-core products accumulated into A_s (A is read in place)
        L.gemm = o.take(ot_update_ws_bytes(s, n, kSketchChunk));
    } else if (gauss_fp32_tc(prec)) {
        // FP32: three BF16 pieces per value, six K segments of length ldq (a
        // multiple of 64: the operands are K-blocked in slices of 64)
        L.ldq = L.ldo = align_up((size_t)m, 64);
        L.ahat = o.take(sizeof(uint16_t) * 6 * (size_t)L.ldq * n);
        L.om = o.take(sizeof(uint16_t) * 6 * (size_t)L.ldo * s);
        L.gemm = o.take(sketch_tc_ws_bytes(s, n, 6 * L.ldq, LSQ_BF16, sms));
    } else {
        L.ahat = o.take((size_t)L.ldq * n * es);
        L.om = o.take((size_t)L.ldo * s * es);
        GemmPlan gp = plan_gemm_kmajor(s, n, m, false, prec == LSQ_FP64 ? LSQ_FP64 : LSQ_FP32, sms);
        L.gemm = o.take(std::max(gemm_kmajor_ws_bytes(gp), sketch_tc_ws_bytes(s, n, m, prec, sms)));
    }
    L.total = o.off;
    L.gemm_bytes = L.total - L.gemm;
    return L;
}

// Condition estimate on a sketch (lsq_condest_sketch): its options and scratch.
lsq_opts est_opts(int64_t m, int64_t n, uint64_t seed, int32_t row_offset = 0) {
    lsq_opts e{};
    e.row_offset = row_offset;
    e.kind = LSQ_SPARSE_SIGN;
    e.s = std::min<int64_t>(2 * n, m);
    e.zeta = (int32_t)std::min<int64_t>(8, e.s);
    e.seed = seed;
    e.sketch_prec = LSQ_FP32;
    e.qr_prec = LSQ_FP32;
    return e;
}

struct EstLayout {
    SketchLayout sk;
    size_t sk_base, ae, re, qr, qr_bytes, judge, judge_bytes, g, gemm, gemm_bytes, z, fin, fin_bytes, acc, k1, qinfo,
        gerr, total;
    bool tc;
    int64_t ldz;
};

EstLayout est_layout(int64_t m, int64_t n, int sms) {
    EstLayout L{};
    Off q;
    const lsq_opts e = est_opts(m, n, 0);
    L.sk = sketch_layout(m, n, e.s, e.kind, e.zeta, LSQ_FP32, sms);
    L.sk_base = q.take(L.sk.total);
    L.ae = q.take(sizeof(float) * (size_t)e.s * n);
    L.re = q.take(sizeof(double) * (size_t)n * n);
    L.qr_bytes = qr_ws_bytes(e.s, n, LSQ_FP32);
    L.qr = q.take(L.qr_bytes);
    L.judge_bytes = judge_ws_bytes(n);
    L.judge = q.take(L.judge_bytes);
    L.g = q.take(sizeof(float) * (size_t)n * n);
    // G_s on the tensor cores (BF16 pieces, one GEMM) or the FP32 CUDA-core GEMM
    L.tc = tensor_core_sketch_enabled() && sketch_tc_supported(LSQ_BF16);
    if (L.tc) {
        L.ldz = align_up((size_t)e.s, 16);
        L.z = q.take(sizeof(uint16_t) * 7 * (size_t)L.ldz * n);
        L.gemm_bytes = sketch_tc_ws_bytes(n, n, 6 * L.ldz, LSQ_BF16, sms);
    } else {
        L.gemm_bytes = gemm_kmajor_ws_bytes(plan_gemm_kmajor(n, n, e.s, true, LSQ_FP32, sms));
    }
    L.gemm = q.take(L.gemm_bytes);
    L.gerr = q.take(sizeof(int32_t));
    L.fin_bytes = condest_sketch_finish_ws_bytes(n);
    L.fin = q.take(L.fin_bytes);
    L.acc = q.take(sizeof(int32_t));
    L.k1 = q.take(sizeof(double));
    L.qinfo = q.take(sizeof(int32_t));
    L.total = q.off;
    return L;
}

lsq_status run_sketch(const double* A, int64_t m, int64_t n, int64_t lda, const lsq_opts* o, int prec, void* As,
                      int64_t ldas, int32_t* colexp_out, char* base, const SketchLayout& L, int32_t* err,
                      cudaStream_t st);

__global__ void k_reject_on_err(const int32_t* __restrict__ err, int32_t* __restrict__ accept) {
    if (*err != 0) *accept = 0;
}

// FP32 sparse-sign sketch, its FP32 R_e, the judge of R_e and the estimator
// of Sec. 6.1 on the sketch's Gram (csrc/condest.cu); base: EstLayout.
lsq_status run_condest_sketch(const double* A, int64_t m, int64_t n, int64_t lda, uint64_t seed, double* kappa0,
                              int32_t* chosen, char* base, const EstLayout& L, int sms, cudaStream_t st,
                              int32_t row_offset = 0) {
    const lsq_opts e = est_opts(m, n, seed, row_offset);
    char* skb = base + L.sk_base;
    int32_t* err = (int32_t*)(skb + L.sk.err);
    int32_t* ce = (int32_t*)(skb + L.sk.colexp);
    float* Ae = (float*)(base + L.ae);
    double* Re = (double*)(base + L.re);
    int32_t* acc = (int32_t*)(base + L.acc);
    double* k1 = (double*)(base + L.k1);
    int32_t* qinfo = (int32_t*)(base + L.qinfo);
    LSQ_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int32_t), st));
    LSQ_CUDA_TRY(cudaMemsetAsync(qinfo, 0, sizeof(int32_t), st));
    lsq_status r = run_sketch(A, m, n, lda, &e, LSQ_FP32, Ae, e.s, ce, skb, L.sk, err, st);
    if (r != LSQ_OK) return r;
    if ((r = reduce_partial(Ae, e.s * n, LSQ_REDUCE_SUM_F32, st)) != LSQ_OK) return r;
    if ((r = launch_precond_qr(Ae, e.s, n, e.s, LSQ_FP32, LSQ_FP32, ce, Re, n, qinfo, base + L.qr, L.qr_bytes, st)) !=
        LSQ_OK)
        return r;
    if ((r = launch_judge(Re, n, n, LSQ_FP32, acc, k1, base + L.judge, L.judge_bytes, st)) != LSQ_OK) return r;
    float* G = (float*)(base + L.g);
    if (L.tc) {
        uint16_t* Z = (uint16_t*)(base + L.z);
        int32_t* gerr = (int32_t*)(base + L.gerr);
        LSQ_CUDA_TRY(cudaMemsetAsync(gerr, 0, sizeof(int32_t), st));
        if ((r = launch_gram_split3<float>(Ae, e.s, n, e.s, L.ldz, Z, st)) != LSQ_OK) return r;
        r = launch_sketch_tc(Z, 7 * L.ldz, Z + L.ldz, 7 * L.ldz, LSQ_BF16, n, n, 6 * L.ldz, G, n, base + L.gemm,
                             L.gemm_bytes, gerr, st);
        if (r != LSQ_OK) return r;
        // a timed-out pipeline leaves no Gram: reject the factor (the overflow case, FP64)
        k_reject_on_err<<<1, 1, 0, st>>>(gerr, acc);
        LSQ_LAUNCH_CHECK();
    } else {
        GemmPlan gp = plan_gemm_kmajor(n, n, e.s, true, LSQ_FP32, sms);
        if ((r = launch_gemm_kmajor(gp, Ae, LSQ_FP32, e.s, Ae, LSQ_FP32, e.s, G, n, base + L.gemm, st)) != LSQ_OK)
            return r;
    }
    return launch_condest_sketch_finish(G, ce, Re, n, n, acc, kappa0, chosen, base + L.fin, L.fin_bytes, st);
}

struct SolveLayout {
    SketchLayout sk;
    size_t sk_base, as_, rs, qr, ap, g, c, x, r, gv, piv, gemm, gemv, cond, k0, ch, err, tsync, oz, est, total;
    size_t hq_m, hq_r, hq_qr, hq_qr_bytes;  // HPNE through QR: [[H, c], [0, 1]], its R, QR scratch
    size_t oz_bytes;
    size_t qr_bytes, cond_bytes;
};

SolveLayout solve_layout(int64_t m, int64_t n, const lsq_opts* o, int prec, int method, int sms) {
    const bool hpne = method_nonsym(method);
    SolveLayout L{};
    Off q;
    L.sk = sketch_layout(m, n, o->s, o->kind, o->zeta, prec, sms);
    // reserve for the widest sketch precision, so that a workspace sized with
    // the layout of one precision (AUTO sizes with FP64) fits whichever runs
    size_t sk_bytes = L.sk.total;
    for (int p = LSQ_FP8_E4M3; p <= LSQ_FP64; ++p)
        sk_bytes = std::max(sk_bytes, sketch_layout(m, n, o->s, o->kind, o->zeta, p, sms).total);
    L.sk_base = q.take(sk_bytes);
    int as_es = prec == LSQ_FP64 ? 8 : 4;
    L.as_ = q.take((size_t)o->s * n * as_es);
    L.rs = q.take(sizeof(double) * (size_t)n * n);
    int qp = prec == LSQ_FP64 ? LSQ_FP64 : o->qr_prec;
    L.qr_bytes = qr_ws_bytes(o->s, n, qp);
    if (method == M_NNE) L.qr_bytes = std::max(L.qr_bytes, lu_precond_ws_bytes(o->s, n, qp));
    L.qr = q.take(L.qr_bytes);
    L.ap = q.take(sizeof(double) * (size_t)m * n);
    L.g = q.take(sizeof(double) * (size_t)n * n);
    L.c = q.take(sizeof(double) * n);
    L.x = q.take(sizeof(double) * n);
    L.r = q.take(sizeof(double) * m);
    L.gv = q.take(sizeof(double) * n);
    L.piv = q.take(sizeof(int32_t) * n);
    GemmPlan gp = plan_gemm_kmajor(n, n, m, !hpne, LSQ_FP64, sms);
    L.gemm = q.take(gemm_kmajor_ws_bytes(gp));
    L.gemv = q.take(gemv_t_ws_bytes(m, n));
    L.cond_bytes = condest_ws_bytes(m, n, sms);
    L.cond = q.take(L.cond_bytes);
    L.k0 = q.take(sizeof(double));
    L.ch = q.take(sizeof(int32_t));
    L.err = q.take(sizeof(int32_t));
    L.tsync = q.take(sizeof(int32_t) * trsv_sync_ints(n));
    // shared by the tensor-core A_p (first) and the tensor-core Gram of PNE
    L.oz_bytes = std::max(ot_trsm_ws_bytes(m, n), hpne ? oz_gemm_tn_ws_bytes(m, n) : oz_gram_ws_bytes(m, n));
    L.oz = q.take(L.oz_bytes);
    L.est = o->sketch_prec == LSQ_AUTO_SKETCH ? q.take(est_layout(m, n, sms).total) : 0;
    if (method == M_HPNE_QR) {
        L.hq_m = q.take(sizeof(double) * (size_t)(n + 1) * (n + 1));
        L.hq_r = q.take(sizeof(double) * (size_t)(n + 1) * (n + 1));
        L.hq_qr_bytes = qr_ws_bytes(n + 1, n + 1, LSQ_FP64);
        L.hq_qr = q.take(L.hq_qr_bytes);
    }
    L.total = q.off + 256;
    return L;
}

char* aligned(void* ws) { return (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255); }

__global__ void k_merge_err(const int32_t* __restrict__ err, int32_t* __restrict__ info) {
    if (*err != 0) atomicCAS(info, 0, *err);
}

lsq_status run_sketch(const double* A, int64_t m, int64_t n, int64_t lda, const lsq_opts* o, int prec, void* As,
                      int64_t ldas, int32_t* colexp_out, char* base, const SketchLayout& L, int32_t* err,
                      cudaStream_t st) {
    unsigned long long* colmax = (unsigned long long*)(base + L.colmax);
    int32_t* colexp = colexp_out ? colexp_out : (int32_t*)(base + L.colexp);
    lsq_status r = launch_colexp(A, m, n, lda, prec, colmax, colexp, st);
    if (r != LSQ_OK) return r;
    if (o->kind == LSQ_SRFT)
        return launch_srft(A, m, n, lda, colexp, prec, o->seed, o->s, base + L.ahat, As, ldas, st);
    if (o->kind == LSQ_SPARSE_SIGN) {
        int32_t* idx = (int32_t*)(base + L.idx);
        int8_t* sgn = (int8_t*)(base + L.sgn);
        if ((r = launch_sparse_gen(o->seed, m, o->s, o->zeta, idx, sgn, err, o->row_offset, st)) != LSQ_OK) return r;
        if ((r = launch_sparse_csr(idx, sgn, m, o->s, o->zeta, (int32_t*)(base + L.counts), (int32_t*)(base + L.rowptr),
                                   (int32_t*)(base + L.cursor), (uint32_t*)(base + L.col),
                                   (int32_t*)(base + L.maxcount), err, st)) != LSQ_OK)
            return r;
        if ((r = launch_quantize_rm(A, m, n, lda, colexp, prec, base + L.ahat, st)) != LSQ_OK) return r;
        return launch_sparse_gather((int32_t*)(base + L.rowptr), (uint32_t*)(base + L.col), base + L.ahat, prec,
                                    o->s, n, As, ldas, st);
    }
    if (gauss_fp64_tc(prec)) {
        // A_s = sum over K chunks of Omega[:, chunk] A[chunk, :], each chunk an
        // FP64-accurate product (C - (-Omega) A), accumulated in FP64.  The
        // chunk of -Omega is generated straight into the product's X digit
        // planes: its entries lie on the 2^-17 grid below 8, three digits.
        double* As64 = (double*)As;
        LSQ_CUDA_TRY(cudaMemset2DAsync(As64, sizeof(double) * ldas, 0, sizeof(double) * o->s, n, st));
        for (int64_t k0 = 0; k0 < m; k0 += kSketchChunk) {
            const int64_t kc = std::min<int64_t>(kSketchChunk, m - k0);
            if ((r = ot_gauss_digits(o->seed, o->s, o->row_offset + k0, kc, n, base + L.gemm, L.gemm_bytes, st)) !=
                LSQ_OK)
                return r;
            if ((r = ot_gemm_update(nullptr, o->s, A + k0, 1, lda, As64, ldas, As64, ldas, o->s, n, kc,
                                    base + L.gemm, L.gemm_bytes, err, st, 2, nullptr, 0, 0, 3)) != LSQ_OK)
                return r;
        }
        return LSQ_OK;
    }
    if (gauss_fp32_tc(prec)) {
        const int64_t K6 = 6 * L.ldq;
        if ((r = launch_gauss_split3(o->seed, o->s, m, L.ldq, (uint16_t*)(base + L.om), o->row_offset, st)) != LSQ_OK)
            return r;
        if ((r = launch_quantize_split3(A, m, n, lda, colexp, L.ldq, (uint16_t*)(base + L.ahat), st)) != LSQ_OK)
            return r;
        return launch_sketch_tc(base + L.om, K6, base + L.ahat, K6, LSQ_BF16, o->s, n, K6, (float*)As, ldas,
                                base + L.gemm, L.gemm_bytes, err, st, true);
    }
    if ((r = launch_gauss_gen(o->seed, o->s, m, prec, base + L.om, L.ldo, o->row_offset, st)) != LSQ_OK) return r;
    if ((r = launch_quantize_cm(A, m, n, lda, colexp, prec, base + L.ahat, L.ldq, st)) != LSQ_OK) return r;
    if (g_tensor_core_sketch && sketch_tc_supported(prec))
        return launch_sketch_tc(base + L.om, L.ldo, base + L.ahat, L.ldq, prec, o->s, n, m, (float*)As, ldas,
                                base + L.gemm, L.total - L.gemm, err, st);
    GemmPlan gp = plan_gemm_kmajor(o->s, n, m, false, prec == LSQ_FP64 ? LSQ_FP64 : LSQ_FP32, device_sm_count());
    return launch_gemm_kmajor(gp, base + L.om, prec, L.ldo, base + L.ahat, prec, L.ldq, As, ldas, base + L.gemm, st);
}

// HPNE through QR: M = [[H, v], [0, g]] ((n+1) x (n+1), ld n+1); the
// Householder R of M holds R_H and Q_H^T v, so H x = v gives x = R_H^{-1}
// (Q_H^T v).  The corner g (the power of two at or above max |v|, 1 for a
// zero or non-finite v) changes neither R_H nor Q_H^T v (the reflectors of
// the first n columns have no component in the last row); a unit corner
// would set the scale of the last column to 1 and with it the columnwise
// error of the QR's products, whatever the size of v.
__global__ void k_hq_gamma(const double* __restrict__ v, int64_t n, double* __restrict__ g) {
    __shared__ double red[32];
    double mx = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, fabs(v[i]));
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t = fmax(t, red[q]);
        *g = (t > 0.0 && isfinite(t)) ? ldexp(1.0, ilogb(t) + 1) : 1.0;
    }
}

__global__ void k_hq_augment(const double* __restrict__ H, int64_t n, int64_t ldh, const double* __restrict__ v,
                             const double* __restrict__ g, double* __restrict__ M) {
    const int64_t n1 = n + 1, total = n1 * n1;
    const double corner = *g;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q % n1, j = q / n1;
        M[q] = (i < n && j < n) ? H[i + j * ldh] : (j == n ? (i < n ? v[i] : corner) : 0.0);
    }
}

lsq_status hq_solve(const double* H, int64_t n, double* v, char* base, const SolveLayout& L, int32_t* info,
                    int32_t* sync, int32_t* err, cudaStream_t st) {
    double* M = (double*)(base + L.hq_m);
    double* Ra = (double*)(base + L.hq_r);
    const int64_t n1 = n + 1;
    double* g = Ra + n1 * n1 - 1;  // scratch until the QR writes R
    k_hq_gamma<<<1, 1024, 0, st>>>(v, n, g);
    LSQ_LAUNCH_CHECK();
    k_hq_augment<<<(unsigned)std::min<int64_t>(ceil_div(n1 * n1, 256), 8192), 256, 0, st>>>(H, n, n, v, g, M);
    LSQ_LAUNCH_CHECK();
    lsq_status r = launch_precond_qr(M, n1, n1, n1, LSQ_FP64, LSQ_FP64, nullptr, Ra, n1, info, base + L.hq_qr,
                                     L.hq_qr_bytes, st);
    if (r != LSQ_OK) return r;
    LSQ_CUDA_TRY(cudaMemcpyAsync(v, Ra + n * n1, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    return launch_trsv<double>(TRSV_UPPER, Ra, n, n1, v, info, sync, err, st);
}

// Solve with the factors already in G (and piv / Rs): PNE: L L^T y = v, x = Rs^{-1} y;
// HPNE: P, unit L, U.
// sync: trsv_sync_ints(n) int32 of scratch; err: status word for a timed-out wait.
lsq_status solve_factored(bool hpne, const double* G, int64_t n, int64_t ldg, const int32_t* piv, const double* Rs,
                          int64_t ldr, double* v, const int32_t* info, int32_t* sync, int32_t* err,
                          cudaStream_t st) {
    lsq_status r;
    if (hpne) {
        if ((r = launch_apply_piv(piv, n, v, info, st)) != LSQ_OK) return r;
        if ((r = launch_trsv<double>(TRSV_UNIT_LOWER, G, n, ldg, v, info, sync, err, st)) != LSQ_OK) return r;
        return launch_trsv<double>(TRSV_UPPER, G, n, ldg, v, info, sync, err, st);
    }
    if ((r = launch_trsv<double>(TRSV_LOWER, G, n, ldg, v, info, sync, err, st)) != LSQ_OK) return r;
    if ((r = launch_trsv<double>(TRSV_LOWER_T, G, n, ldg, v, info, sync, err, st)) != LSQ_OK) return r;
    if (Rs) return launch_trsv<double>(TRSV_UPPER, Rs, n, ldr, v, info, sync, err, st);
    return LSQ_OK;
}

lsq_status trsm_gram(const double* A, int64_t m, int64_t n, int64_t lda, const double* Rs, int64_t ldr,
                     const double* b, bool hpne, double* Ap, int64_t ldap, double* G, int64_t ldg, double* c,
                     void* gemm_ws, double* gemv_ws, int64_t gemv_cap, int sms, cudaStream_t st,
                     void* oz_ws = nullptr, size_t oz_bytes = 0, int32_t* err = nullptr) {
    stage_mark(ST_TRSM, true, st);
    lsq_status r;
    if (g_fp64_emulation && oz_ws && oz_bytes >= ot_trsm_ws_bytes(m, n) && ot_trsm_supported())
        r = ot_trsm(A, m, n, lda, Rs, ldr, Ap, ldap, oz_ws, oz_bytes, err, st);
    else
        r = launch_trsm_right_upper(A, m, n, lda, Rs, ldr, Ap, ldap, st);
    if (r != LSQ_OK) return r;
    stage_mark(ST_TRSM, false, st);
    stage_mark(ST_GRAM, true, st);
    GemmPlan gp = plan_gemm_kmajor(n, n, m, !hpne, LSQ_FP64, sms);
    if (hpne) {
        if (g_fp64_emulation && oz_ws && oz_bytes >= oz_gemm_tn_ws_bytes(m, n))
            r = oz_gemm_tn(Ap, ldap, A, lda, m, n, G, ldg, oz_ws, oz_bytes, err, st);
        else
            r = launch_gemm_kmajor(gp, Ap, LSQ_FP64, ldap, A, LSQ_FP64, lda, G, ldg, gemm_ws, st);
    } else if (g_fp64_emulation && oz_ws && oz_bytes >= oz_gram_ws_bytes(m, n)) {
        r = oz_gram(Ap, m, n, ldap, G, ldg, oz_ws, oz_bytes, err, st);
    } else {
        r = launch_gemm_kmajor(gp, Ap, LSQ_FP64, ldap, Ap, LSQ_FP64, ldap, G, ldg, gemm_ws, st);
    }
    if (r != LSQ_OK) return r;
    r = launch_gemv_t(Ap, m, n, ldap, b, c, gemv_ws, gemv_cap, st);
    stage_mark(ST_GRAM, false, st);
    return r;
}

lsq_status solve_impl(int method, const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
                      const lsq_opts* o, double* x, double* Rs_out, int32_t* info, void* ws, size_t ws_bytes,
                      cudaStream_t st, const double* Rs_in = nullptr) {
    if (method < M_PNE || method > M_NNE) return LSQ_ERR_ARG;
    const bool hpne = method_nonsym(method);
    if (!A || !b || !x || !info || m <= 0 || n <= 0 || lda < m) return LSQ_ERR_ARG;
    lsq_status r = check_opts(o, m, n, true);
    if (r != LSQ_OK) return r;
    int sms = device_sm_count();
    // Layout with the widest sketch precision when AUTO, so one workspace
    // serves whatever precision the estimate picks.
    SolveLayout L = solve_layout(m, n, o, layout_prec(o->sketch_prec), method, sms);
    if (!ws || L.total > ws_bytes) return LSQ_ERR_NOMEM;
    char* base = aligned(ws);
    int32_t* err = (int32_t*)(base + L.err);
    LSQ_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int32_t), st));
    LSQ_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int32_t), st));
    int prec = o->sketch_prec;
    if (is_auto(prec)) {
        double* k0 = (double*)(base + L.k0);
        int32_t* ch = (int32_t*)(base + L.ch);
        stage_mark(ST_CONDEST, true, st);
        if (prec == LSQ_AUTO)
            r = launch_condest(A, m, n, lda, k0, ch, base + L.cond, L.cond_bytes, sms, st);
        else
            r = run_condest_sketch(A, m, n, lda, o->seed, k0, ch, base + L.est, est_layout(m, n, sms), sms, st,
                                   o->row_offset);
        if (r != LSQ_OK) return r;
        stage_mark(ST_CONDEST, false, st);
        int32_t host_ch = LSQ_FP64;
        LSQ_CUDA_TRY(cudaMemcpyAsync(&host_ch, ch, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        LSQ_CUDA_TRY(cudaStreamSynchronize(st));
        prec = host_ch;
        if (!valid_sketch_prec(prec)) prec = LSQ_FP64;
    }
    int qp = prec == LSQ_FP64 ? LSQ_FP64 : o->qr_prec;
    SketchLayout SK = sketch_layout(m, n, o->s, o->kind, o->zeta, prec, sms);
    char* skb = base + L.sk_base;
    void* As = base + L.as_;
    int64_t s = o->s;
    double* Rs = (double*)(base + L.rs);
    double* Ap = (double*)(base + L.ap);
    double* G = (double*)(base + L.g);
    double* c = (double*)(base + L.c);
    double* r_ = (double*)(base + L.r);
    double* gv = (double*)(base + L.gv);
    int32_t* piv = (int32_t*)(base + L.piv);
    int32_t* colexp = (int32_t*)(skb + SK.colexp);
    if (Rs_in) {
        // preconditioner already computed (and accepted) by the caller
        LSQ_CUDA_TRY(cudaMemcpyAsync(Rs, Rs_in, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, st));
    } else {
        stage_mark(ST_SKETCH, true, st);
        if ((r = run_sketch(A, m, n, lda, o, prec, As, s, colexp, skb, SK, err, st)) != LSQ_OK) return r;
        if ((r = reduce_partial(As, s * n, prec == LSQ_FP64 ? LSQ_REDUCE_SUM_F64 : LSQ_REDUCE_SUM_F32, st)) != LSQ_OK)
            return r;
        stage_mark(ST_SKETCH, false, st);
        stage_mark(ST_QR, true, st);
        const int as_prec = prec == LSQ_FP64 ? LSQ_FP64 : LSQ_FP32;
        if (method == M_NNE)
            r = launch_lu_precond(As, s, n, s, as_prec, qp, colexp, Rs, n, info, base + L.qr, L.qr_bytes, st);
        else
            r = launch_precond_qr(As, s, n, s, as_prec, qp, colexp, Rs, n, info, base + L.qr, L.qr_bytes, st);
        if (r != LSQ_OK) return r;
        stage_mark(ST_QR, false, st);
    }
    if ((r = trsm_gram(A, m, n, lda, Rs, n, b, hpne, Ap, m, G, n, c, base + L.gemm, (double*)(base + L.gemv),
                       (int64_t)(gemv_t_ws_bytes(m, n) / sizeof(double)), sms, st, base + L.oz, L.oz_bytes, err)) !=
        LSQ_OK)
        return r;
    int32_t* tsync = (int32_t*)(base + L.tsync);
    double* gemv_ws = (double*)(base + L.gemv);
    const int64_t gemv_cap = (int64_t)(gemv_t_ws_bytes(m, n) / sizeof(double));
    if (method == M_SNE && (r = launch_gemv_t(A, m, n, lda, b, c, gemv_ws, gemv_cap, st)) != LSQ_OK) return r;
    // row-sharded A: the Gram and the right-hand side summed over the shards
    if ((r = reduce_partial(G, n * n, LSQ_REDUCE_SUM_F64, st)) != LSQ_OK) return r;
    if ((r = reduce_partial(c, n, LSQ_REDUCE_SUM_F64, st)) != LSQ_OK) return r;
    if (method == M_SNE) {
        // right-hand side of Eq. e_sne in factored form: R_s^{-T} (A^T b)
        if ((r = launch_trsv<double>(TRSV_UPPER_T, Rs, n, n, c, info, tsync, err, st)) != LSQ_OK) return r;
    }
    stage_mark(ST_FACTOR, true, st);
    if (method == M_HPNE || method == M_NNE)
        r = launch_lu(G, n, n, piv, info, st);
    else if (method != M_HPNE_QR)
        r = launch_cholesky<double>(G, n, n, info, st, base + L.oz, L.oz_bytes);
    if (r != LSQ_OK) return r;
    stage_mark(ST_FACTOR, false, st);
    stage_mark(ST_SOLVE, true, st);
    LSQ_CUDA_TRY(cudaMemcpyAsync(x, c, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    if (method == M_HPNE_QR)
        r = hq_solve(G, n, x, base, L, info, tsync, err, st);
    else
        r = solve_factored(hpne, G, n, n, piv, Rs, n, x, info, tsync, err, st);
    if (r != LSQ_OK) return r;
    stage_mark(ST_SOLVE, false, st);
    if (o->refine_steps > 0) stage_mark(ST_REFINE, true, st);
    for (int step = 0; step < o->refine_steps; ++step) {
        if ((r = launch_residual(A, m, n, lda, x, b, r_, st)) != LSQ_OK) return r;
        // A_p^T r, or A^T r for the corrected seminormal equations (R^T R d = A^T r),
        // summed over the shards of a row-sharded A
        if (method == M_SNE)
            r = launch_gemv_t(A, m, n, lda, r_, gv, gemv_ws, gemv_cap, st);
        else
            r = launch_gemv_t(Ap, m, n, m, r_, gv, gemv_ws, gemv_cap, st);
        if (r != LSQ_OK) return r;
        if ((r = reduce_partial(gv, n, LSQ_REDUCE_SUM_F64, st)) != LSQ_OK) return r;
        if (method == M_SNE && (r = launch_trsv<double>(TRSV_UPPER_T, Rs, n, n, gv, info, tsync, err, st)) != LSQ_OK)
            return r;
        if (method == M_HPNE_QR)
            r = hq_solve(G, n, gv, base, L, info, tsync, err, st);
        else
            r = solve_factored(hpne, G, n, n, piv, Rs, n, gv, info, tsync, err, st);
        if (r != LSQ_OK) return r;
        if ((r = launch_axpy1(x, gv, n, st)) != LSQ_OK) return r;
    }
    if (o->refine_steps > 0) stage_mark(ST_REFINE, false, st);
    if (Rs_out) LSQ_CUDA_TRY(cudaMemcpyAsync(Rs_out, Rs, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, st));
    k_merge_err<<<1, 1, 0, st>>>(err, info);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

struct HostLayout {
    size_t a, b, x, info, solve, total;
};

HostLayout host_layout(int64_t m, int64_t n, const lsq_opts* o, bool hpne, int sms) {
    HostLayout H{};
    Off q;
    H.a = q.take(sizeof(double) * (size_t)m * n);
    H.b = q.take(sizeof(double) * m);
    H.x = q.take(sizeof(double) * n);
    H.info = q.take(sizeof(int32_t));
    int p = layout_prec(o->sketch_prec);
    H.solve = q.take(solve_layout(m, n, o, p, hpne, sms).total);
    H.total = q.off + 256;
    return H;
}

lsq_status solve_host_impl(bool hpne, const double* A_host, int64_t m, int64_t n, int64_t lda, const double* b_host,
                           const lsq_opts* o, double* x_host, int32_t* info_host, void* ws, size_t ws_bytes,
                           cudaStream_t st) {
    if (!A_host || !b_host || !x_host || !info_host || m <= 0 || n <= 0 || lda < m) return LSQ_ERR_ARG;
    lsq_status r = check_opts(o, m, n, true);
    if (r != LSQ_OK) return r;
    int sms = device_sm_count();
    HostLayout H = host_layout(m, n, o, hpne, sms);
    if (!ws || H.total > ws_bytes) return LSQ_ERR_NOMEM;
    char* base = aligned(ws);
    double* A = (double*)(base + H.a);
    double* b = (double*)(base + H.b);
    double* x = (double*)(base + H.x);
    int32_t* info = (int32_t*)(base + H.info);
    if (lda == m) {
        LSQ_CUDA_TRY(cudaMemcpyAsync(A, A_host, sizeof(double) * (size_t)m * n, cudaMemcpyHostToDevice, st));
    } else {
        LSQ_CUDA_TRY(cudaMemcpy2DAsync(A, sizeof(double) * m, A_host, sizeof(double) * lda, sizeof(double) * m, n,
                                       cudaMemcpyHostToDevice, st));
    }
    LSQ_CUDA_TRY(cudaMemcpyAsync(b, b_host, sizeof(double) * m, cudaMemcpyHostToDevice, st));
    size_t solve_cap = ws_bytes - (size_t)((base + H.solve) - (char*)ws);
    r = solve_impl(hpne, A, m, n, m, b, o, x, nullptr, info, base + H.solve, solve_cap, st);
    if (r != LSQ_OK) return r;
    LSQ_CUDA_TRY(cudaMemcpyAsync(x_host, x, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    LSQ_CUDA_TRY(cudaMemcpyAsync(info_host, info, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    LSQ_CUDA_TRY(cudaStreamSynchronize(st));
    return LSQ_OK;
}

}  // namespace

extern "C" {

int32_t lsq_version(void) { return 100; }

lsq_reduce_fn lsq_set_reduce_hook(lsq_reduce_fn fn, void* user) {
    lsq_reduce_fn prev = g_reduce_fn;
    g_reduce_fn = fn;
    g_reduce_user = user;
    return prev;
}

const char* lsq_last_cuda_error(void) { return cudaGetErrorString((cudaError_t)g_last_cuda_error.load()); }

int64_t lsq_launch_count(void) { return (int64_t)g_launches.load(); }

int64_t lsq_test_set_solve_wait_ns(int64_t ns) {
    if (ns <= 0) return -1;
    return (int64_t)lsq::set_trsv_wait_ns((uint64_t)ns);
}

int32_t lsq_set_fp64_emulation(int32_t enable) {
    int32_t prev = g_fp64_emulation ? 1 : 0;
    g_fp64_emulation = enable != 0;
    return prev;
}

size_t lsq_trsm_tc_workspace_size(int64_t m, int64_t n) { return m > 0 && n > 0 ? ot_trsm_ws_bytes(m, n) + 256 : 0; }

lsq_status lsq_trsm_tc(const double* A, int64_t m, int64_t n, int64_t lda, const double* R, int64_t ldr, double* Ap,
                       int64_t ldap, int32_t* info, void* ws, size_t ws_bytes, void* stream) {
    if (!A || !R || !Ap || m <= 0 || n <= 0 || lda < m || ldap < m || ldr < n) return LSQ_ERR_ARG;
    if (A != Ap) {
        // reject partial overlap of the input and output column ranges
        const char* a0 = (const char*)A;
        const char* a1 = (const char*)(A + (n - 1) * lda + m);
        const char* p0 = (const char*)Ap;
        const char* p1 = (const char*)(Ap + (n - 1) * ldap + m);
        if (a0 < p1 && p0 < a1) return LSQ_ERR_ARG;
    } else if (ldap != lda) {
        return LSQ_ERR_ARG;
    }
    if (info) LSQ_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int32_t), S(stream)));
    return ot_trsm(A, m, n, lda, R, ldr, Ap, ldap, ws, ws_bytes, info, S(stream));
}

size_t lsq_gemm_tn_tc_workspace_size(int64_t m, int64_t n) {
    return m > 0 && n > 0 ? oz_gemm_tn_ws_bytes(m, n) + 256 : 0;
}

lsq_status lsq_gemm_tn_tc(const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t m, int64_t n,
                          double* G, int64_t ldg, int32_t* info, void* ws, size_t ws_bytes, void* stream) {
    if (!X || !Y || !G || m <= 0 || n <= 0 || ldx < m || ldy < m || ldg < n) return LSQ_ERR_ARG;
    if (info) LSQ_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int32_t), S(stream)));
    return oz_gemm_tn(X, ldx, Y, ldy, m, n, G, ldg, ws, ws_bytes, info, S(stream));
}

size_t lsq_gram_tc_workspace_size(int64_t m, int64_t n) { return m > 0 && n > 0 ? oz_gram_ws_bytes(m, n) + 256 : 0; }

lsq_status lsq_gram_tc(const double* X, int64_t m, int64_t n, int64_t ld, double* G, int64_t ldg, int32_t* info,
                       void* ws, size_t ws_bytes, void* stream) {
    if (!X || !G || m <= 0 || n <= 0 || ld < m || ldg < n) return LSQ_ERR_ARG;
    if (info) LSQ_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int32_t), S(stream)));
    return oz_gram(X, m, n, ld, G, ldg, ws, ws_bytes, info, S(stream));
}

int32_t lsq_set_tensor_core_sketch(int32_t enable) {
    int32_t prev = g_tensor_core_sketch ? 1 : 0;
    g_tensor_core_sketch = enable != 0;
    return prev;
}

int32_t lsq_profile(int32_t enable) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    g_prof.on = enable != 0;
    g_prof.next = 0;
    g_prof.recs.clear();
    for (int i = 0; i < ST_COUNT; ++i) g_prof.open[i] = false;
    return LSQ_OK;
}

int32_t lsq_profile_collect(double* ms_by_stage, int32_t* count_by_stage, int32_t nstages) {
    return lsq_profile_collect_work(ms_by_stage, count_by_stage, nullptr, nstages);
}

int32_t lsq_profile_collect_work(double* ms_by_stage, int32_t* count_by_stage, double* work_by_stage,
                                 int32_t nstages) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    if (!ms_by_stage || !count_by_stage || nstages < 8) return LSQ_ERR_ARG;
    for (int i = 0; i < nstages; ++i) {
        ms_by_stage[i] = 0.0;
        count_by_stage[i] = 0;
        if (work_by_stage) work_by_stage[i] = 0.0;
    }
    for (auto& rec : g_prof.recs) {
        if (cudaEventSynchronize(g_prof.pool[rec.ev_end]) != cudaSuccess) return LSQ_ERR_CUDA;
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, g_prof.pool[rec.ev_begin], g_prof.pool[rec.ev_end]) != cudaSuccess)
            return LSQ_ERR_CUDA;
        if (rec.stage >= nstages) continue;
        ms_by_stage[rec.stage] += ms;
        count_by_stage[rec.stage] += 1;
        if (work_by_stage) work_by_stage[rec.stage] += rec.work;
    }
    g_prof.recs.clear();
    g_prof.next = 0;
    return LSQ_OK;
}

int32_t lsq_profile_records(int32_t stage, double* ms, double* work, int32_t cap) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    if (!ms || !work || cap < 0) return -LSQ_ERR_ARG;
    int32_t k = 0;
    for (auto& rec : g_prof.recs) {
        if (rec.stage != stage) continue;
        if (k < cap) {
            if (cudaEventSynchronize(g_prof.pool[rec.ev_end]) != cudaSuccess) return -LSQ_ERR_CUDA;
            float t = 0.0f;
            if (cudaEventElapsedTime(&t, g_prof.pool[rec.ev_begin], g_prof.pool[rec.ev_end]) != cudaSuccess)
                return -LSQ_ERR_CUDA;
            ms[k] = t;
            work[k] = rec.work;
        }
        ++k;
    }
    return k;
}

const char* lsq_status_string(int32_t s) {
    switch (s) {
    case LSQ_OK: return "LSQ_OK";
    case LSQ_ERR_ARG: return "LSQ_ERR_ARG";
    case LSQ_ERR_BREAKDOWN: return "LSQ_ERR_BREAKDOWN";
    case LSQ_ERR_NONFINITE: return "LSQ_ERR_NONFINITE";
    case LSQ_ERR_TIMEOUT: return "LSQ_ERR_TIMEOUT";
    case LSQ_ERR_CUDA: return "LSQ_ERR_CUDA";
    case LSQ_ERR_NOMEM: return "LSQ_ERR_NOMEM";
    default: return "LSQ_UNKNOWN";
    }
}

int32_t lsq_precision_from_kappa0(double k0) {
    if (!(k0 == k0) || k0 > 1.0e308) return LSQ_FP64;
    if (k0 < 2.0) return LSQ_FP8_E4M3;
    if (k0 < 3.0) return LSQ_BF16;
    if (k0 < 4.0) return LSQ_FP16;
    if (k0 <= 8.0) return LSQ_FP32;
    return LSQ_FP64;
}

size_t lsq_workspace_size(int32_t op, int64_t m, int64_t n, const lsq_opts* o) {
    if (m <= 0 || n <= 0) return 0;
    int sms = device_sm_count();
    switch (op) {
    case LSQ_OP_SKETCH:
        if (check_opts(o, m, n, false) != LSQ_OK) return 0;
        return sketch_layout(m, n, o->s, o->kind, o->zeta, o->sketch_prec, sms).total + 256;
    case LSQ_OP_PRECOND_QR:  // m is s here
        return qr_ws_bytes(m, n, LSQ_FP64) + 256;
    case LSQ_OP_CONDEST:
        return condest_ws_bytes(m, n, sms) + 256;
    case LSQ_OP_CONDEST_SKETCH:
        return est_layout(m, n, sms).total + 256;
    case LSQ_OP_PNE:
    case LSQ_OP_HPNE:
    case LSQ_OP_HPNE_QR:
    case LSQ_OP_SNE:
    case LSQ_OP_NNE: {
        if (check_opts(o, m, n, true) != LSQ_OK) return 0;
        const int method = op == LSQ_OP_PNE    ? M_PNE
                           : op == LSQ_OP_HPNE ? M_HPNE
                           : op == LSQ_OP_HPNE_QR ? M_HPNE_QR
                           : op == LSQ_OP_SNE  ? M_SNE
                                               : M_NNE;
        return solve_layout(m, n, o, layout_prec(o->sketch_prec), method, sms).total + 256;
    }
    case LSQ_OP_TRSM_GRAM: {
        GemmPlan gp = plan_gemm_kmajor(n, n, m, false, LSQ_FP64, sms);
        GemmPlan gs = plan_gemm_kmajor(n, n, m, true, LSQ_FP64, sms);
        return std::max(gemm_kmajor_ws_bytes(gp), gemm_kmajor_ws_bytes(gs)) + gemv_t_ws_bytes(m, n) +
               std::max(std::max(oz_gram_ws_bytes(m, n), oz_gemm_tn_ws_bytes(m, n)), ot_trsm_ws_bytes(m, n)) + 2048;
    }
    case LSQ_OP_FACTOR_SOLVE:
        return align_up(sizeof(int32_t) * trsv_sync_ints(n), 256) + cholesky_ws_bytes(n) + 512;
    case LSQ_OP_PNE_HOST:
    case LSQ_OP_HPNE_HOST:
        if (check_opts(o, m, n, true) != LSQ_OK) return 0;
        return host_layout(m, n, o, op == LSQ_OP_HPNE_HOST, sms).total + 256;
    default:
        return 0;
    }
}

lsq_status lsq_sparse_sign_operator(uint64_t seed, int64_t m, int64_t s, int32_t zeta, int32_t* idx, int8_t* sgn,
                                    void* stream) {
    if (m <= 0 || s <= 0 || s > 0x7fffffff || zeta < 1 || zeta > 32 || zeta > s || !idx || !sgn) return LSQ_ERR_ARG;
    return launch_sparse_gen(seed, m, s, zeta, idx, sgn, nullptr, 0, S(stream));
}

lsq_status lsq_gaussian_operator(uint64_t seed, int64_t s, int64_t m, int32_t prec, double* Om, void* stream) {
    if (m <= 0 || s <= 0 || !Om || !valid_sketch_prec(prec)) return LSQ_ERR_ARG;
    return launch_gauss_inspect(seed, s, m, prec, Om, S(stream));
}

lsq_status lsq_sketch(const double* A, int64_t m, int64_t n, int64_t lda, const lsq_opts* o, void* As, int64_t ldas,
                      int32_t* colexp, int32_t* info, void* ws, size_t ws_bytes, void* stream) {
    if (!A || !As || m <= 0 || n <= 0 || lda < m) return LSQ_ERR_ARG;
    lsq_status r = check_opts(o, m, n, false);
    if (r != LSQ_OK) return r;
    if (ldas < o->s) return LSQ_ERR_ARG;
    int sms = device_sm_count();
    SketchLayout L = sketch_layout(m, n, o->s, o->kind, o->zeta, o->sketch_prec, sms);
    if (!ws || L.total + 256 > ws_bytes) return LSQ_ERR_NOMEM;
    char* base = aligned(ws);
    int32_t* err = (int32_t*)(base + L.err);
    LSQ_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int32_t), S(stream)));
    if (info) LSQ_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int32_t), S(stream)));
    r = run_sketch(A, m, n, lda, o, o->sketch_prec, As, ldas, colexp, base, L, err, S(stream));
    if (r != LSQ_OK) return r;
    if (info) {
        k_merge_err<<<1, 1, 0, S(stream)>>>(err, info);
        LSQ_LAUNCH_CHECK();
    }
    return LSQ_OK;
}

lsq_status lsq_precond_qr(const void* As, int64_t s, int64_t n, int64_t ldas, int32_t as_prec, int32_t qr_prec,
                          const int32_t* colexp, double* Rs, int64_t ldr, int32_t* info, void* ws, size_t ws_bytes,
                          void* stream) {
    if (!As || !Rs || n <= 0 || s < n || ldas < s || ldr < n) return LSQ_ERR_ARG;
    if ((as_prec != LSQ_FP32 && as_prec != LSQ_FP64) || (qr_prec != LSQ_FP32 && qr_prec != LSQ_FP64)) return LSQ_ERR_ARG;
    if (info) LSQ_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int32_t), S(stream)));
    return launch_precond_qr(As, s, n, ldas, as_prec, qr_prec, colexp, Rs, ldr, info, ws, ws_bytes, S(stream));
}

lsq_status lsq_condest(const double* A, int64_t m, int64_t n, int64_t lda, double* kappa0, int32_t* chosen, void* ws,
                       size_t ws_bytes, void* stream) {
    if (!A || !kappa0 || !chosen || m <= 0 || n <= 0 || lda < m) return LSQ_ERR_ARG;
    return launch_condest(A, m, n, lda, kappa0, chosen, ws, ws_bytes, device_sm_count(), S(stream));
}

lsq_status lsq_condest_sketch(const double* A, int64_t m, int64_t n, int64_t lda, uint64_t seed, double* kappa0,
                              int32_t* chosen, void* ws, size_t ws_bytes, void* stream) {
    if (!A || !kappa0 || !chosen || m <= 0 || n <= 0 || lda < m) return LSQ_ERR_ARG;
    int sms = device_sm_count();
    EstLayout L = est_layout(m, n, sms);
    if (!ws || L.total + 256 > ws_bytes) return LSQ_ERR_NOMEM;
    return run_condest_sketch(A, m, n, lda, seed, kappa0, chosen, aligned(ws), L, sms, S(stream));
}

lsq_status lsq_trsm_gram(const double* A, int64_t m, int64_t n, int64_t lda, const double* Rs, int64_t ldr,
                         const double* b, int32_t hpne, double* Ap, int64_t ldap, double* G, int64_t ldg, double* c,
                         void* ws, size_t ws_bytes, void* stream) {
    if (!A || !Rs || !b || !Ap || !G || !c || m <= 0 || n <= 0 || lda < m || ldr < n || ldap < m || ldg < n)
        return LSQ_ERR_ARG;
    int sms = device_sm_count();
    size_t need = lsq_workspace_size(LSQ_OP_TRSM_GRAM, m, n, nullptr);
    if (!ws || ws_bytes < need) return LSQ_ERR_NOMEM;
    char* base = aligned(ws);
    size_t gemv_bytes = gemv_t_ws_bytes(m, n);
    double* gemv_ws = (double*)base;
    char* gemm_ws = base + align_up(gemv_bytes, 256);
    GemmPlan gp = plan_gemm_kmajor(n, n, m, false, LSQ_FP64, sms);
    GemmPlan gs = plan_gemm_kmajor(n, n, m, true, LSQ_FP64, sms);
    char* oz_ws = gemm_ws + align_up(std::max(gemm_kmajor_ws_bytes(gp), gemm_kmajor_ws_bytes(gs)), 256);
    size_t oz_cap = ws_bytes - (size_t)(oz_ws - (char*)ws);
    return trsm_gram(A, m, n, lda, Rs, ldr, b, hpne != 0, Ap, ldap, G, ldg, c, gemm_ws, gemv_ws,
                     (int64_t)(gemv_bytes / sizeof(double)), sms, S(stream), oz_ws, oz_cap, nullptr);
}

lsq_status lsq_factor_solve(int32_t hpne, double* G, int64_t n, int64_t ldg, const double* c, const double* Rs,
                            int64_t ldr, double* x, int32_t* piv, int32_t* info, void* ws, size_t ws_bytes,
                            void* stream) {
    if (!G || !c || !x || !info || n <= 0 || ldg < n || (hpne && !piv) || (Rs && ldr < n)) return LSQ_ERR_ARG;
    if (!ws || ws_bytes < lsq_workspace_size(LSQ_OP_FACTOR_SOLVE, 1, n, nullptr)) return LSQ_ERR_NOMEM;
    int32_t* tsync = (int32_t*)aligned(ws);
    char* cws = (char*)tsync + align_up(sizeof(int32_t) * trsv_sync_ints(n), 256);
    size_t cws_bytes = ws_bytes - (size_t)(cws - (char*)ws);
    cudaStream_t st = S(stream);
    LSQ_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int32_t), st));
    lsq_status r = hpne ? launch_lu(G, n, ldg, piv, info, st)
                        : launch_cholesky<double>(G, n, ldg, info, st, cws, cws_bytes);
    if (r != LSQ_OK) return r;
    LSQ_CUDA_TRY(cudaMemcpyAsync(x, c, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    return solve_factored(hpne != 0, G, n, ldg, piv, Rs, ldr, x, info, tsync, info, st);
}

lsq_status lsq_pne_solve(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, const lsq_opts* opts,
                         double* x, double* Rs_out, int32_t* info, void* ws, size_t ws_bytes, void* stream) {
    return solve_impl(false, A, m, n, lda, b, opts, x, Rs_out, info, ws, ws_bytes, S(stream));
}

lsq_status lsq_hpne_solve(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, const lsq_opts* opts,
                          double* x, double* Rs_out, int32_t* info, void* ws, size_t ws_bytes, void* stream) {
    return solve_impl(true, A, m, n, lda, b, opts, x, Rs_out, info, ws, ws_bytes, S(stream));
}

lsq_status lsq_hpne_qr_solve(const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
                             const lsq_opts* opts, double* x, double* Rs_out, int32_t* info, void* ws, size_t ws_bytes,
                             void* stream) {
    return solve_impl(M_HPNE_QR, A, m, n, lda, b, opts, x, Rs_out, info, ws, ws_bytes, S(stream));
}

lsq_status lsq_sne_solve(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, const lsq_opts* opts,
                         double* x, double* Rs_out, int32_t* info, void* ws, size_t ws_bytes, void* stream) {
    return solve_impl(M_SNE, A, m, n, lda, b, opts, x, Rs_out, info, ws, ws_bytes, S(stream));
}

lsq_status lsq_nne_solve(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, const lsq_opts* opts,
                         double* x, double* Us_out, int32_t* info, void* ws, size_t ws_bytes, void* stream) {
    return solve_impl(M_NNE, A, m, n, lda, b, opts, x, Us_out, info, ws, ws_bytes, S(stream));
}

lsq_status lsq_pne_solve_host(const double* A_host, int64_t m, int64_t n, int64_t lda, const double* b_host,
                              const lsq_opts* opts, double* x_host, int32_t* info_host, void* ws, size_t ws_bytes,
                              void* stream) {
    return solve_host_impl(false, A_host, m, n, lda, b_host, opts, x_host, info_host, ws, ws_bytes, S(stream));
}

lsq_status lsq_hpne_solve_host(const double* A_host, int64_t m, int64_t n, int64_t lda, const double* b_host,
                               const lsq_opts* opts, double* x_host, int32_t* info_host, void* ws, size_t ws_bytes,
                               void* stream) {
    return solve_host_impl(true, A_host, m, n, lda, b_host, opts, x_host, info_host, ws, ws_bytes, S(stream));
}

}  // extern "C"

namespace lsq {

// Entry points for the batched driver (csrc/batched.cu).
lsq_status solve_impl_ext(bool hpne, const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
                          const lsq_opts* o, double* x, double* Rs_out, int32_t* info, void* ws, size_t ws_bytes,
                          cudaStream_t st, const double* Rs_in) {
    return solve_impl(hpne, A, m, n, lda, b, o, x, Rs_out, info, ws, ws_bytes, st, Rs_in);
}

size_t solve_ws_bytes_ext(int64_t m, int64_t n, const lsq_opts* o, bool hpne) {
    return solve_layout(m, n, o, layout_prec(o->sketch_prec), hpne, device_sm_count()).total + 256;
}

}  // namespace lsq
