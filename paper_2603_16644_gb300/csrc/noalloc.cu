// lsq_trsm_gram_noalloc: the FP64 preconditioning + Gram step without any
// caller workspace and without allocating.
//
// Who needs it: callers that cannot allocate device memory at the point of
// the call -- code running inside a memory pool or allocator callback,
// inside a framework that owns all device allocations and forbids others,
// or a real-time loop where cudaMalloc's implicit device synchronisation is
// not allowed.  They still own and pass every input and output buffer; the
// only scratch (split-K partial Gram matrices and GEMV partial sums) lives in
// the fixed array below, which each GPU that loads the library holds until
// the process exits.
#include "common.cuh"
#include "kernels.cuh"

#include <algorithm>
#include <mutex>

namespace {

// Fixed scratch: 16 MiB per device.
constexpr size_t kNoallocScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
// Per device: the context the address was looked up in, and the address.
// A device reset (cudaDeviceReset) or a new primary context invalidates the
// address, so it is looked up again whenever the current context changes.
void* g_noalloc_ctx[kMaxDevices] = {};
void* g_noalloc_ptr[kMaxDevices] = {};

// The driver's cuCtxGetCurrent, reached through the runtime (no link to the
// driver library); nullptr if unavailable.
typedef int (*CtxGetCurrentFn)(void**);
CtxGetCurrentFn ctx_get_current() {
    static CtxGetCurrentFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return (CtxGetCurrentFn)p;
        return (CtxGetCurrentFn) nullptr;
    }();
    return fn;
}

// Device address of the scratch array for the current device.  Host code may
// not use the symbol itself (it is a host-side stand-in); the address comes
// from cudaGetSymbolAddress, with that device current, once per device and
// context.
lsq_status noalloc_scratch(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LSQ_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return LSQ_ERR_ARG;
    // (before the first runtime call that creates the primary context, ctx is
    // null; the lookup then runs again on the next call, harmlessly)
    void* ctx = nullptr;
    CtxGetCurrentFn get = ctx_get_current();
    if (get && get(&ctx) != 0) ctx = nullptr;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev] || g_noalloc_ctx[dev] != ctx) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return LSQ_ERR_CUDA;
        g_noalloc_ptr[dev] = p;
        g_noalloc_ctx[dev] = ctx;
    }
    *out = g_noalloc_ptr[dev];
    return LSQ_OK;
}

}  // namespace

extern "C" lsq_status lsq_trsm_gram_noalloc(const double* A, int64_t m, int64_t n, int64_t lda, const double* Rs,
                                            int64_t ldr, const double* b, int32_t hpne, double* Ap, int64_t ldap,
                                            double* G, int64_t ldg, double* c, void* stream) {
    using namespace lsq;
    if (!A || !Rs || !b || !Ap || !G || !c || m <= 0 || n <= 0 || lda < m || ldr < n || ldap < m || ldg < n)
        return LSQ_ERR_ARG;
    // The GEMV partials must fit; the split-K partials are then capped to the rest.
    size_t gemv_bytes = align_up(gemv_t_ws_bytes(m, n), 256);
    if (gemv_bytes > kNoallocScratchBytes) return LSQ_ERR_ARG;
    void* scratch = nullptr;
    lsq_status r = noalloc_scratch(&scratch);
    if (r != LSQ_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    int sms = device_sm_count();
    r = launch_trsm_right_upper(A, m, n, lda, Rs, ldr, Ap, ldap, st);
    if (r != LSQ_OK) return r;
    GemmPlan gp = plan_gemm_kmajor(n, n, m, hpne == 0, LSQ_FP64, sms);
    size_t per_split = (size_t)n * (size_t)n * sizeof(double);
    size_t room = kNoallocScratchBytes - gemv_bytes;
    int fit = (int)std::min<size_t>(64, room / per_split);
    if (gp.splits > 1 && gp.splits > fit) {
        int sp = std::max(1, fit);
        gp.kchunk = ceil_div(ceil_div(m, sp), 32) * 32;
        gp.splits = (int)ceil_div(m, gp.kchunk);
    }
    // Every partial the reduction reads is written first: nothing needs zeroing.
    char* base = (char*)scratch;
    void* gemm_ws = gp.splits > 1 ? (void*)(base + gemv_bytes) : nullptr;
    if (hpne)
        r = launch_gemm_kmajor(gp, Ap, LSQ_FP64, ldap, A, LSQ_FP64, lda, G, ldg, gemm_ws, st);
    else
        r = launch_gemm_kmajor(gp, Ap, LSQ_FP64, ldap, Ap, LSQ_FP64, ldap, G, ldg, gemm_ws, st);
    if (r != LSQ_OK) return r;
    return launch_gemv_t(Ap, m, n, ldap, b, c, (double*)base, (int64_t)(gemv_bytes / sizeof(double)), st);
}
