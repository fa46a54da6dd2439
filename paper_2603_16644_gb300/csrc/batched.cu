// Batched PNE / HPNE (Alg. 1 on many independent problems of uneven shape).
//
// The problems are spread over a fixed set of internal streams (heaviest
// first, each to the least-loaded stream), and the whole fan-out -- every
// kernel of every problem plus the fork/join events -- is captured into one
// CUDA graph that is launched on the caller's stream.  The executable graph
// is cached and replayed while the batch description is unchanged, so a
// repeated batched call is one graph launch.  Problems asking for the AUTO
// precision first get one batched condition-estimate pass (Sec. 6.1; on A^T A
// for AUTO, on a sketch for AUTO_SKETCH) and a single readback of the chosen
// precisions, because kernel selection in the captured graph needs them on
// the host.  The batched sketch and preconditioner QR (lsq_sketch_batched,
// lsq_precond_qr_batched) use the same captured fan-out.
#include "common.cuh"
#include "kernels.cuh"

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

namespace lsq {
lsq_status solve_impl_ext(bool hpne, const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
                          const lsq_opts* o, double* x, double* Rs_out, int32_t* info, void* ws, size_t ws_bytes,
                          cudaStream_t st, const double* Rs_in);
size_t solve_ws_bytes_ext(int64_t m, int64_t n, const lsq_opts* o, bool hpne);
}  // namespace lsq

namespace {

using namespace lsq;

constexpr int kMaxStreams = 64;

// Internal streams of the fan-out: 16, or $LSQ_BATCH_STREAMS (1 .. 64), read
// once per process.
int n_streams() {
    static const int ns = [] {
        const char* e = std::getenv("LSQ_BATCH_STREAMS");
        const int v = e ? std::atoi(e) : 16;
        return v < 1 ? 1 : (v > kMaxStreams ? kMaxStreams : v);
    }();
    return ns;
}

struct BatchState {
    std::mutex mu;
    int dev = -1;
    cudaStream_t sub[kMaxStreams] = {};
    cudaStream_t cap = nullptr;  // the graph is captured here, never on the caller stream
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kMaxStreams] = {};
};
BatchState g_batch;

// A cached executable graph and the description it was built from: one for
// the solves (or the batched sketch / QR steps), one for the estimate pass.
struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    std::vector<unsigned char> key;
    void drop() {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        key.clear();
    }
};
GraphCache g_main, g_est;
lsq_status ensure_streams() {
    int dev = 0;
    LSQ_CUDA_TRY(cudaGetDevice(&dev));
    if (g_batch.dev == dev && g_batch.fork) return LSQ_OK;
    for (int k = 0; k < n_streams(); ++k) {
        LSQ_CUDA_TRY(cudaStreamCreateWithFlags(&g_batch.sub[k], cudaStreamNonBlocking));
        LSQ_CUDA_TRY(cudaEventCreateWithFlags(&g_batch.join[k], cudaEventDisableTiming));
    }
    LSQ_CUDA_TRY(cudaEventCreateWithFlags(&g_batch.fork, cudaEventDisableTiming));
    LSQ_CUDA_TRY(cudaStreamCreateWithFlags(&g_batch.cap, cudaStreamNonBlocking));
    g_batch.dev = dev;
    g_main.drop();
    g_est.drop();
    return LSQ_OK;
}

struct Plan {
    std::vector<int> stream_of;   // problem -> internal stream
    std::vector<int> order;       // launch order (heaviest first)
    size_t slot_bytes = 0;        // workspace per internal stream
    size_t head_bytes = 0;        // chosen-precision scratch at the front
};

double work_of(const lsq_batch_problem& p) { return 2.0 * (double)p.m * (double)p.n * (double)p.n; }

Plan make_plan(bool hpne, int32_t count, const lsq_batch_problem* probs) {
    Plan P;
    P.stream_of.assign(count, 0);
    P.order.resize(count);
    for (int i = 0; i < count; ++i) P.order[i] = i;
    std::stable_sort(P.order.begin(), P.order.end(),
                     [&](int a, int b) { return work_of(probs[a]) > work_of(probs[b]); });
    double load[kMaxStreams] = {};
    for (int i : P.order) {
        int best = 0;
        for (int k = 1; k < n_streams(); ++k)
            if (load[k] < load[best]) best = k;
        P.stream_of[i] = best;
        load[best] += work_of(probs[i]);
    }
    for (int i = 0; i < count; ++i) {
        size_t need = solve_ws_bytes_ext(probs[i].m, probs[i].n, &probs[i].opts, hpne);
        size_t c = condest_ws_bytes(probs[i].m, probs[i].n, device_sm_count());
        if (probs[i].opts.sketch_prec == LSQ_AUTO_SKETCH)
            c = std::max(c, lsq_workspace_size(LSQ_OP_CONDEST_SKETCH, probs[i].m, probs[i].n, nullptr));
        P.slot_bytes = std::max(P.slot_bytes, std::max(need, c));
    }
    P.slot_bytes = align_up(P.slot_bytes, 256);
    P.head_bytes = align_up((size_t)count * (sizeof(double) + sizeof(int32_t)) + 512, 256);
    return P;
}

lsq_status check_problem(const lsq_batch_problem& p) {
    if (!p.A || !p.b || !p.x || !p.info || p.m <= 0 || p.n <= 0 || p.lda < p.m) return LSQ_ERR_ARG;
    const lsq_opts* o = &p.opts;
    if (o->kind != LSQ_GAUSSIAN && o->kind != LSQ_SPARSE_SIGN && o->kind != LSQ_SRFT) return LSQ_ERR_ARG;
    if (o->s < p.n || o->s > p.m) return LSQ_ERR_ARG;
    if (o->kind == LSQ_SPARSE_SIGN && (o->zeta < 1 || o->zeta > 32 || o->zeta > o->s)) return LSQ_ERR_ARG;
    if (o->sketch_prec < LSQ_FP8_E4M3 || o->sketch_prec > LSQ_AUTO_SKETCH) return LSQ_ERR_ARG;
    return LSQ_OK;
}

bool is_auto(int p) { return p == LSQ_AUTO || p == LSQ_AUTO_SKETCH; }

// Capture a fan-out of per-problem work over the internal streams into one
// graph (cached in `cache` under `key`) and launch it on st.  run(i, stream,
// slot) enqueues problem i.  Every pass over the internal streams is such a
// graph: while a stream is captured, no step of a problem forks onto the
// library's shared look-ahead streams, so concurrent problems never share a
// stream.  Caller holds g_batch.mu.
template <typename F>
lsq_status capture_fanout(GraphCache& cache, const std::vector<int>& order, const std::vector<int>& stream_of,
                          char* slots, size_t slot_bytes, std::vector<unsigned char>& key, cudaStream_t st, F run) {
    if (cache.exec && key == cache.key) {
        LSQ_CUDA_TRY(cudaGraphLaunch(cache.exec, st));
        return LSQ_OK;
    }
    cache.drop();
    cudaGraph_t graph = nullptr;
    // Capture on an internal stream (the caller may use the legacy default
    // stream, which cannot be captured); the graph is then launched on st.
    cudaStream_t cs = g_batch.cap;
    LSQ_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    lsq_status cap = LSQ_OK;
    if (cudaEventRecord(g_batch.fork, cs) != cudaSuccess) cap = LSQ_ERR_CUDA;
    for (int k = 0; k < n_streams() && cap == LSQ_OK; ++k)
        if (cudaStreamWaitEvent(g_batch.sub[k], g_batch.fork, 0) != cudaSuccess) cap = LSQ_ERR_CUDA;
    for (int i : order) {
        if (cap != LSQ_OK) break;
        int k = stream_of[i];
        cap = run(i, g_batch.sub[k], slots + (size_t)k * slot_bytes);
    }
    for (int k = 0; k < n_streams() && cap == LSQ_OK; ++k) {
        if (cudaEventRecord(g_batch.join[k], g_batch.sub[k]) != cudaSuccess) cap = LSQ_ERR_CUDA;
        else if (cudaStreamWaitEvent(cs, g_batch.join[k], 0) != cudaSuccess) cap = LSQ_ERR_CUDA;
    }
    cudaError_t ec = cudaStreamEndCapture(cs, &graph);
    if (cap != LSQ_OK || ec != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();  // do not leave a capture error behind for the caller
        return cap != LSQ_OK ? cap : LSQ_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return LSQ_ERR_CUDA;
    cache.exec = exec;
    cache.key.swap(key);
    LSQ_CUDA_TRY(cudaGraphLaunch(cache.exec, st));
    return LSQ_OK;
}

// Heaviest first, each to the least-loaded internal stream.
void assign_streams(const std::vector<double>& work, std::vector<int>& order, std::vector<int>& stream_of) {
    const int count = (int)work.size();
    order.resize(count);
    stream_of.assign(count, 0);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
    double load[kMaxStreams] = {};
    for (int i : order) {
        int best = 0;
        for (int k = 1; k < n_streams(); ++k)
            if (load[k] < load[best]) best = k;
        stream_of[i] = best;
        load[best] += work[i];
    }
}

lsq_status batched(bool hpne, int32_t count, const lsq_batch_problem* probs, void* ws, size_t ws_bytes,
                   cudaStream_t st) {
    if (count <= 0 || !probs) return LSQ_ERR_ARG;
    for (int i = 0; i < count; ++i) {
        lsq_status r = check_problem(probs[i]);
        if (r != LSQ_OK) return r;
    }
    std::lock_guard<std::mutex> lk(g_batch.mu);
    lsq_status r = ensure_streams();
    if (r != LSQ_OK) return r;
    Plan P = make_plan(hpne, count, probs);
    char* base = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    size_t need = P.head_bytes + P.slot_bytes * n_streams() + 256;
    if (!ws || need > ws_bytes) return LSQ_ERR_NOMEM;
    char* slots = base + P.head_bytes;
    int sms = device_sm_count();

    // resolve AUTO precisions: one batched estimate pass (a cached graph of
    // its own), one readback
    std::vector<lsq_batch_problem> q(probs, probs + count);
    bool any_auto = false;
    for (int i = 0; i < count; ++i) any_auto |= is_auto(q[i].opts.sketch_prec);
    if (any_auto) {
        double* k0 = (double*)base;
        int32_t* ch = (int32_t*)(base + align_up(sizeof(double) * count, 256));
        std::vector<int> est_order;
        for (int i : P.order)
            if (is_auto(q[i].opts.sketch_prec)) est_order.push_back(i);
        std::vector<unsigned char> ekey(sizeof(lsq_batch_problem) * count + 64, 0);
        std::memcpy(ekey.data(), probs, sizeof(lsq_batch_problem) * count);
        unsigned char* et = ekey.data() + sizeof(lsq_batch_problem) * count;
        std::memcpy(et, &ws, sizeof(ws));
        std::memcpy(et + 8, &ws_bytes, sizeof(ws_bytes));
        r = capture_fanout(g_est, est_order, P.stream_of, slots, P.slot_bytes, ekey, st,
                           [&](int i, cudaStream_t sk, char* slot) {
                               if (q[i].opts.sketch_prec == LSQ_AUTO)
                                   return launch_condest(q[i].A, q[i].m, q[i].n, q[i].lda, k0 + i, ch + i, slot,
                                                         P.slot_bytes, sms, sk);
                               return lsq_condest_sketch(q[i].A, q[i].m, q[i].n, q[i].lda, q[i].opts.seed, k0 + i,
                                                         ch + i, slot, P.slot_bytes, sk);
                           });
        if (r != LSQ_OK) return r;
        std::vector<int32_t> host_ch(count, LSQ_FP64);
        LSQ_CUDA_TRY(cudaMemcpyAsync(host_ch.data(), ch, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, st));
        LSQ_CUDA_TRY(cudaStreamSynchronize(st));
        for (int i = 0; i < count; ++i)
            if (is_auto(q[i].opts.sketch_prec)) {
                int p = host_ch[i];
                q[i].opts.sketch_prec = (p >= LSQ_FP8_E4M3 && p <= LSQ_FP64) ? p : LSQ_FP64;
                if (q[i].opts.sketch_prec == LSQ_FP64) q[i].opts.qr_prec = LSQ_FP64;
            }
    }

    // key of the captured graph: the resolved descriptors and the buffers
    std::vector<unsigned char> key(sizeof(lsq_batch_problem) * count + 64);
    std::memcpy(key.data(), q.data(), sizeof(lsq_batch_problem) * count);
    unsigned char* tail = key.data() + sizeof(lsq_batch_problem) * count;
    std::memset(tail, 0, 64);
    std::memcpy(tail, &ws, sizeof(ws));
    std::memcpy(tail + 8, &ws_bytes, sizeof(ws_bytes));
    int32_t hp = hpne ? 1 : 0;
    std::memcpy(tail + 16, &hp, sizeof(hp));
    return capture_fanout(g_main, P.order, P.stream_of, slots, P.slot_bytes, key, st,
                          [&](int i, cudaStream_t sk, char* slot) {
                              return solve_impl_ext(hpne, q[i].A, q[i].m, q[i].n, q[i].lda, q[i].b, &q[i].opts,
                                                    q[i].x, nullptr, q[i].info, slot, P.slot_bytes, sk, nullptr);
                          });
}

// ---- batched sketch and preconditioner QR --------------------------------
size_t sketch_slot_bytes(const lsq_sketch_problem& p) { return lsq_workspace_size(LSQ_OP_SKETCH, p.m, p.n, &p.opts); }
size_t qr_slot_bytes(const lsq_qr_problem& p) { return lsq_workspace_size(LSQ_OP_PRECOND_QR, p.s, p.n, nullptr); }

lsq_status check_sketch_problem(const lsq_sketch_problem& p) {
    if (!p.A || !p.As || !p.colexp || p.m <= 0 || p.n <= 0 || p.lda < p.m || p.ldas < p.opts.s) return LSQ_ERR_ARG;
    if (p.opts.sketch_prec < LSQ_FP8_E4M3 || p.opts.sketch_prec > LSQ_FP64) return LSQ_ERR_ARG;
    return sketch_slot_bytes(p) ? LSQ_OK : LSQ_ERR_ARG;
}

lsq_status check_qr_problem(const lsq_qr_problem& p) {
    if (!p.As || !p.Rs || !p.info || p.n <= 0 || p.s < p.n || p.ldas < p.s || p.ldr < p.n) return LSQ_ERR_ARG;
    if ((p.as_prec != LSQ_FP32 && p.as_prec != LSQ_FP64) || (p.qr_prec != LSQ_FP32 && p.qr_prec != LSQ_FP64))
        return LSQ_ERR_ARG;
    return LSQ_OK;
}

template <typename Prob, typename Check, typename Slot, typename Work, typename Run>
lsq_status batched_steps(int tag, int32_t count, const Prob* probs, void* ws, size_t ws_bytes, cudaStream_t st,
                         Check check, Slot slot_of, Work work_of_p, Run run) {
    if (count <= 0 || !probs) return LSQ_ERR_ARG;
    size_t slot = 0;
    std::vector<double> work(count);
    for (int i = 0; i < count; ++i) {
        lsq_status r = check(probs[i]);
        if (r != LSQ_OK) return r;
        slot = std::max(slot, slot_of(probs[i]));
        work[i] = work_of_p(probs[i]);
    }
    slot = align_up(slot, 256);
    char* base = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    if (!ws || slot * n_streams() + 512 > ws_bytes) return LSQ_ERR_NOMEM;
    std::lock_guard<std::mutex> lk(g_batch.mu);
    lsq_status r = ensure_streams();
    if (r != LSQ_OK) return r;
    std::vector<int> order, stream_of;
    assign_streams(work, order, stream_of);
    std::vector<unsigned char> key(sizeof(Prob) * count + 64, 0);
    std::memcpy(key.data(), probs, sizeof(Prob) * count);
    unsigned char* tail = key.data() + sizeof(Prob) * count;
    std::memcpy(tail, &ws, sizeof(ws));
    std::memcpy(tail + 8, &ws_bytes, sizeof(ws_bytes));
    std::memcpy(tail + 16, &tag, sizeof(tag));
    return capture_fanout(g_main, order, stream_of, base, slot, key, st,
                          [&](int i, cudaStream_t sk, char* sl) { return run(probs[i], sl, slot, sk); });
}

size_t batched_steps_ws(size_t slot) { return align_up(slot, 256) * n_streams() + 512; }

}  // namespace

extern "C" {

size_t lsq_batched_workspace_size(int32_t hpne, int32_t count, const lsq_batch_problem* probs) {
    if (count <= 0 || !probs) return 0;
    for (int i = 0; i < count; ++i)
        if (check_problem(probs[i]) != LSQ_OK) return 0;
    Plan P = make_plan(hpne != 0, count, probs);
    return P.head_bytes + P.slot_bytes * n_streams() + 512;
}

lsq_status lsq_pne_solve_batched(int32_t count, const lsq_batch_problem* probs, void* ws, size_t ws_bytes,
                                 void* stream) {
    return batched(false, count, probs, ws, ws_bytes, (cudaStream_t)stream);
}

lsq_status lsq_hpne_solve_batched(int32_t count, const lsq_batch_problem* probs, void* ws, size_t ws_bytes,
                                  void* stream) {
    return batched(true, count, probs, ws, ws_bytes, (cudaStream_t)stream);
}

size_t lsq_sketch_batched_workspace_size(int32_t count, const lsq_sketch_problem* probs) {
    if (count <= 0 || !probs) return 0;
    size_t slot = 0;
    for (int i = 0; i < count; ++i) {
        if (check_sketch_problem(probs[i]) != LSQ_OK) return 0;
        slot = std::max(slot, sketch_slot_bytes(probs[i]));
    }
    return batched_steps_ws(slot);
}

lsq_status lsq_sketch_batched(int32_t count, const lsq_sketch_problem* probs, void* ws, size_t ws_bytes,
                              void* stream) {
    return batched_steps(
        2, count, probs, ws, ws_bytes, (cudaStream_t)stream, check_sketch_problem, sketch_slot_bytes,
        [](const lsq_sketch_problem& p) { return 2.0 * (double)p.m * (double)p.n * (double)p.opts.s; },
        [](const lsq_sketch_problem& p, char* slot, size_t bytes, cudaStream_t sk) {
            return lsq_sketch(p.A, p.m, p.n, p.lda, &p.opts, p.As, p.ldas, p.colexp, p.info, slot, bytes, sk);
        });
}

size_t lsq_precond_qr_batched_workspace_size(int32_t count, const lsq_qr_problem* probs) {
    if (count <= 0 || !probs) return 0;
    size_t slot = 0;
    for (int i = 0; i < count; ++i) {
        if (check_qr_problem(probs[i]) != LSQ_OK) return 0;
        slot = std::max(slot, qr_slot_bytes(probs[i]));
    }
    return batched_steps_ws(slot);
}

lsq_status lsq_precond_qr_batched(int32_t count, const lsq_qr_problem* probs, void* ws, size_t ws_bytes,
                                  void* stream) {
    return batched_steps(
        3, count, probs, ws, ws_bytes, (cudaStream_t)stream, check_qr_problem, qr_slot_bytes,
        [](const lsq_qr_problem& p) { return 2.0 * (double)p.n * (double)p.n * (double)p.s; },
        [](const lsq_qr_problem& p, char* slot, size_t bytes, cudaStream_t sk) {
            return lsq_precond_qr(p.As, p.s, p.n, p.ldas, p.as_prec, p.qr_prec, p.colexp, p.Rs, p.ldr, p.info, slot,
                                  bytes, sk);
        });
}

}  // extern "C"
