// FP64 FMA throughput probe: every thread runs 8 independent DFMA chains for
// `iters` iterations.  Used to check the FP64 roofline denominator of the
// FP64 kernels on the device at hand (instrumentation, not part of Alg. 1).
#include "common.cuh"
#include "kernels.cuh"

namespace lsq {

__global__ void __launch_bounds__(256) k_probe_dfma(int64_t iters, double seed, double* __restrict__ out) {
    double a0 = seed + threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
    double a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
    const double mlt = 0.9999999, add = 1e-7;
    for (int64_t i = 0; i < iters; ++i) {
        a0 = fma(a0, mlt, add); a1 = fma(a1, mlt, add); a2 = fma(a2, mlt, add); a3 = fma(a3, mlt, add);
        a4 = fma(a4, mlt, add); a5 = fma(a5, mlt, add); a6 = fma(a6, mlt, add); a7 = fma(a7, mlt, add);
    }
    double s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
    if (s == 12345.678) out[blockIdx.x] = s;  // keeps the chains live
}

}  // namespace lsq

extern "C" int32_t lsq_probe_fp64_fma(int64_t iters, int32_t blocks, double* scratch, void* stream) {
    if (iters <= 0 || blocks <= 0 || !scratch) return LSQ_ERR_ARG;
    lsq::k_probe_dfma<<<blocks, 256, 0, (cudaStream_t)stream>>>(iters, 1.0, scratch);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}
