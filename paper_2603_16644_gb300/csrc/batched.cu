// Batched PNE / HPNE (Alg. 1 on many independent problems of uneven shape).
//
// The problems are spread over a fixed set of internal streams (heaviest
// first, each to the least-loaded stream), and the whole fan-out -- every
// kernel of every problem plus the fork/join events -- is captured into one
// CUDA graph that is launched on the caller's stream.  The executable graph
// is cached and replayed while the batch description is unchanged, so a
// repeated batched call is one graph launch.  Problems asking for the AUTO
// precision first get one batched condition-estimate pass (Sec. 6.1) and a
// single readback of the chosen precisions, because kernel selection in the
// captured graph needs them on the host.
#include "common.cuh"
#include "kernels.cuh"

#include <algorithm>
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

constexpr int kStreams = 16;

struct BatchState {
    std::mutex mu;
    int dev = -1;
    cudaStream_t sub[kStreams] = {};
    cudaStream_t cap = nullptr;  // the graph is captured here, never on the caller stream
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kStreams] = {};
    // cached executable graph and the description it was built from
    cudaGraphExec_t exec = nullptr;
    std::vector<unsigned char> key;
};
BatchState g_batch;

lsq_status ensure_streams() {
    int dev = 0;
    LSQ_CUDA_TRY(cudaGetDevice(&dev));
    if (g_batch.dev == dev && g_batch.fork) return LSQ_OK;
    for (int k = 0; k < kStreams; ++k) {
        LSQ_CUDA_TRY(cudaStreamCreateWithFlags(&g_batch.sub[k], cudaStreamNonBlocking));
        LSQ_CUDA_TRY(cudaEventCreateWithFlags(&g_batch.join[k], cudaEventDisableTiming));
    }
    LSQ_CUDA_TRY(cudaEventCreateWithFlags(&g_batch.fork, cudaEventDisableTiming));
    LSQ_CUDA_TRY(cudaStreamCreateWithFlags(&g_batch.cap, cudaStreamNonBlocking));
    g_batch.dev = dev;
    if (g_batch.exec) {
        cudaGraphExecDestroy(g_batch.exec);
        g_batch.exec = nullptr;
    }
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
    double load[kStreams] = {};
    for (int i : P.order) {
        int best = 0;
        for (int k = 1; k < kStreams; ++k)
            if (load[k] < load[best]) best = k;
        P.stream_of[i] = best;
        load[best] += work_of(probs[i]);
    }
    for (int i = 0; i < count; ++i) {
        size_t need = solve_ws_bytes_ext(probs[i].m, probs[i].n, &probs[i].opts, hpne);
        size_t c = condest_ws_bytes(probs[i].m, probs[i].n, device_sm_count());
        P.slot_bytes = std::max(P.slot_bytes, std::max(need, c));
    }
    P.slot_bytes = align_up(P.slot_bytes, 256);
    P.head_bytes = align_up((size_t)count * (sizeof(double) + sizeof(int32_t)) + 512, 256);
    return P;
}

lsq_status check_problem(const lsq_batch_problem& p) {
    if (!p.A || !p.b || !p.x || !p.info || p.m <= 0 || p.n <= 0 || p.lda < p.m) return LSQ_ERR_ARG;
    const lsq_opts* o = &p.opts;
    if (o->kind != LSQ_GAUSSIAN && o->kind != LSQ_SPARSE_SIGN) return LSQ_ERR_ARG;
    if (o->s < p.n || o->s > p.m) return LSQ_ERR_ARG;
    if (o->kind == LSQ_SPARSE_SIGN && (o->zeta < 1 || o->zeta > 32 || o->zeta > o->s)) return LSQ_ERR_ARG;
    if (o->sketch_prec < LSQ_FP8_E4M3 || o->sketch_prec > LSQ_AUTO) return LSQ_ERR_ARG;
    return LSQ_OK;
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
    size_t need = P.head_bytes + P.slot_bytes * kStreams + 256;
    if (!ws || need > ws_bytes) return LSQ_ERR_NOMEM;
    char* slots = base + P.head_bytes;
    int sms = device_sm_count();

    // resolve AUTO precisions: one batched estimate pass, one readback
    std::vector<lsq_batch_problem> q(probs, probs + count);
    bool any_auto = false;
    for (int i = 0; i < count; ++i) any_auto |= (q[i].opts.sketch_prec == LSQ_AUTO);
    if (any_auto) {
        double* k0 = (double*)base;
        int32_t* ch = (int32_t*)(base + align_up(sizeof(double) * count, 256));
        LSQ_CUDA_TRY(cudaEventRecord(g_batch.fork, st));
        for (int k = 0; k < kStreams; ++k) LSQ_CUDA_TRY(cudaStreamWaitEvent(g_batch.sub[k], g_batch.fork, 0));
        for (int i : P.order) {
            if (q[i].opts.sketch_prec != LSQ_AUTO) continue;
            int k = P.stream_of[i];
            r = launch_condest(q[i].A, q[i].m, q[i].n, q[i].lda, k0 + i, ch + i, slots + (size_t)k * P.slot_bytes,
                               P.slot_bytes, sms, g_batch.sub[k]);
            if (r != LSQ_OK) return r;
        }
        for (int k = 0; k < kStreams; ++k) {
            LSQ_CUDA_TRY(cudaEventRecord(g_batch.join[k], g_batch.sub[k]));
            LSQ_CUDA_TRY(cudaStreamWaitEvent(st, g_batch.join[k], 0));
        }
        std::vector<int32_t> host_ch(count, LSQ_FP64);
        LSQ_CUDA_TRY(cudaMemcpyAsync(host_ch.data(), ch, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, st));
        LSQ_CUDA_TRY(cudaStreamSynchronize(st));
        for (int i = 0; i < count; ++i)
            if (q[i].opts.sketch_prec == LSQ_AUTO) {
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
    if (g_batch.exec && key == g_batch.key) {
        LSQ_CUDA_TRY(cudaGraphLaunch(g_batch.exec, st));
        return LSQ_OK;
    }
    if (g_batch.exec) {
        cudaGraphExecDestroy(g_batch.exec);
        g_batch.exec = nullptr;
        g_batch.key.clear();
    }
    cudaGraph_t graph = nullptr;
    // Capture on an internal stream (the caller may use the legacy default
    // stream, which cannot be captured); the graph is then launched on st.
    cudaStream_t cs = g_batch.cap;
    LSQ_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    lsq_status cap = LSQ_OK;
    if (cudaEventRecord(g_batch.fork, cs) != cudaSuccess) cap = LSQ_ERR_CUDA;
    for (int k = 0; k < kStreams && cap == LSQ_OK; ++k)
        if (cudaStreamWaitEvent(g_batch.sub[k], g_batch.fork, 0) != cudaSuccess) cap = LSQ_ERR_CUDA;
    for (int i : P.order) {
        if (cap != LSQ_OK) break;
        int k = P.stream_of[i];
        cap = solve_impl_ext(hpne, q[i].A, q[i].m, q[i].n, q[i].lda, q[i].b, &q[i].opts, q[i].x, nullptr, q[i].info,
                             slots + (size_t)k * P.slot_bytes, P.slot_bytes, g_batch.sub[k], nullptr);
    }
    for (int k = 0; k < kStreams && cap == LSQ_OK; ++k) {
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
    g_batch.exec = exec;
    g_batch.key.swap(key);
    LSQ_CUDA_TRY(cudaGraphLaunch(g_batch.exec, st));
    return LSQ_OK;
}

}  // namespace

extern "C" {

size_t lsq_batched_workspace_size(int32_t hpne, int32_t count, const lsq_batch_problem* probs) {
    if (count <= 0 || !probs) return 0;
    for (int i = 0; i < count; ++i)
        if (check_problem(probs[i]) != LSQ_OK) return 0;
    Plan P = make_plan(hpne != 0, count, probs);
    return P.head_bytes + P.slot_bytes * kStreams + 512;
}

lsq_status lsq_pne_solve_batched(int32_t count, const lsq_batch_problem* probs, void* ws, size_t ws_bytes,
                                 void* stream) {
    return batched(false, count, probs, ws, ws_bytes, (cudaStream_t)stream);
}

lsq_status lsq_hpne_solve_batched(int32_t count, const lsq_batch_problem* probs, void* ws, size_t ws_bytes,
                                  void* stream) {
    return batched(true, count, probs, ws, ws_bytes, (cudaStream_t)stream);
}

}  // extern "C"
