// Shared device helpers for liblsq: error handling, Philox4x32-10, exact
// FP64 -> low-precision rounding, workspace carving.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/lsq.h"

namespace lsq {

// Remembers the CUDA error behind the last LSQ_ERR_CUDA (lsq_last_cuda_error).
void note_cuda_error(cudaError_t e);
#define LSQ_CUDA_TRY(expr)                                  \
    do {                                                    \
        cudaError_t e__ = (expr);                           \
        if (e__ != cudaSuccess) {                           \
            ::lsq::note_cuda_error(e__);                    \
            return LSQ_ERR_CUDA;                            \
        }                                                   \
    } while (0)

// Every kernel launch goes through this check; it also counts launches
// (lsq_launch_count) so callers can verify what ran.
void note_launch();
#define LSQ_LAUNCH_CHECK()                 \
    do {                                   \
        ::lsq::note_launch();              \
        LSQ_CUDA_TRY(cudaGetLastError());  \
    } while (0)

// Stage timing (lsq_profile): events recorded around the steps of Alg. 1,
// and around single launches of the two heaviest kernels (the tensor-core
// FP64 update and the QR panel) with their algorithmic work (flops).
enum Stage {
    ST_CONDEST = 0, ST_SKETCH, ST_QR, ST_TRSM, ST_GRAM, ST_FACTOR, ST_SOLVE, ST_REFINE,
    ST_K_UPDATE, ST_K_QRPANEL, ST_K_SKETCHTC, ST_K_UPDATE3, ST_COUNT
};
void stage_mark(int stage, bool begin, cudaStream_t st, double work = 0.0);

static inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }
static inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Bump allocator over the caller's workspace (256-byte aligned pieces).
struct Carver {
    char* base;
    size_t cap;
    size_t off;
    bool ok;
    Carver(void* p, size_t c) : base((char*)p), cap(c), off(0), ok(true) {}
    template <class T>
    T* take(size_t count) {
        size_t o = align_up(off, 256);
        size_t bytes = align_up(count * sizeof(T), 256);
        off = o + bytes;
        if (off > cap || base == nullptr) { ok = false; return nullptr; }
        return (T*)(base + o);
    }
};

// ---------------------------------------------------------------------------
// Philox4x32-10, Salmon et al. SC'11 (multipliers 0xD2511F53, 0xCD9E8D57;
// key increments 0x9E3779B9, 0xBB67AE85).
// ---------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        U4 n;
        n.x = hi1 ^ c.y ^ k0;
        n.y = lo1;
        n.z = hi0 ^ c.w ^ k1;
        n.w = lo0;
        c = n;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint32_t word_of(const U4& v, int t) {
    return t == 0 ? v.x : (t == 1 ? v.y : (t == 2 ? v.z : v.w));
}

// ---------------------------------------------------------------------------
// Exact round-to-nearest-even of an FP64 value to a format with p significand
// bits and minimum normal exponent emin (subnormals kept), done on the integer
// significand so there is exactly one rounding.  Returns the rounded value as
// a double (exactly representable in the target format).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double rne_sig(double x, int p, int emin, double maxfin, bool sat) {
    if (x == 0.0 || isnan(x)) return x;
    if (isinf(x)) return sat ? copysign(maxfin, x) : x;
    unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    unsigned long long sign = bits & 0x8000000000000000ull;
    int bexp = (int)((bits >> 52) & 0x7ff);
    if (bexp == 0) return __longlong_as_double((long long)sign);  // FP64 subnormal: far below every target
    int E = bexp - 1023;
    unsigned long long mant = (bits & 0x000fffffffffffffull) | 0x0010000000000000ull;  // 53 bits
    int e = E < emin ? emin : E;
    int drop = (53 - p) + (e - E);  // low significand bits that do not fit
    unsigned long long keep;
    if (drop >= 64) {
        keep = 0;
    } else if (drop > 54) {
        keep = 0;  // below half of the smallest step
    } else {
        keep = mant >> drop;
        unsigned long long rem = mant & ((1ull << drop) - 1ull);
        unsigned long long half = 1ull << (drop - 1);
        if (rem > half || (rem == half && (keep & 1ull))) keep += 1ull;
    }
    // value = keep * 2^(e - p + 1), exact
    double y = ldexp((double)keep, e - p + 1);
    if (y > maxfin) y = sat ? maxfin : __longlong_as_double(0x7ff0000000000000ll);
    return sign ? -y : y;
}

__device__ __forceinline__ double round_to_prec(double x, int prec) {
    switch (prec) {
    case LSQ_FP8_E4M3: return rne_sig(x, 4, -6, 448.0, true);
    case LSQ_BF16: return rne_sig(x, 8, -126, 3.3895313892515355e38, false);
    case LSQ_FP16: return rne_sig(x, 11, -14, 65504.0, false);
    case LSQ_FP32: return (double)__double2float_rn(x);
    default: return x;
    }
}

// Integer-only form of the same rounding, fused with the power-of-two
// scaling 2^escale: returns the bit pattern of RNE(x * 2^escale) in the
// target format (FP8-e4m3 saturating, BF16, FP16, FP32).  No FP64
// instruction is issued (GB300 runs FP64 at 1/64 of the FP32 rate).
__device__ __forceinline__ uint32_t quant_bits(double x, int escale, int prec) {
    int p, emin, emax, bias;
    switch (prec) {
    case LSQ_FP8_E4M3: p = 4; emin = -6; emax = 8; bias = 7; break;
    case LSQ_BF16: p = 8; emin = -126; emax = 127; bias = 127; break;
    case LSQ_FP16: p = 11; emin = -14; emax = 15; bias = 15; break;
    default: p = 24; emin = -126; emax = 127; bias = 127; break;
    }
    const int mb = p - 1;                       // stored mantissa bits
    const int ebits = prec == LSQ_FP8_E4M3 ? 4 : prec == LSQ_FP16 ? 5 : 8;
    const int tot = 1 + ebits + mb;
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    uint32_t sign = (uint32_t)(b >> 63) << (tot - 1);
    int E = (int)((b >> 52) & 0x7ff);
    unsigned long long mant = b & 0x000fffffffffffffull;
    const uint32_t inf_bits = ((1u << ebits) - 1u) << mb;
    const uint32_t sat_bits = prec == LSQ_FP8_E4M3 ? 0x7Eu : inf_bits;  // 448 for e4m3fn
    if (E == 0x7ff) {
        if (mant) return sign | inf_bits | (prec == LSQ_FP8_E4M3 ? 7u : (1u << (mb - 1)));  // NaN
        return sign | sat_bits;
    }
    int ex;  // unbiased exponent of the leading significand bit
    unsigned long long sig;
    if (E == 0) {
        if (mant == 0) return sign;
        int lz = __clzll(mant) - 11;  // normalise an FP64 subnormal
        sig = mant << lz;
        ex = -1022 - lz;
    } else {
        sig = mant | 0x0010000000000000ull;
        ex = E - 1023;
    }
    ex += escale;
    int er = ex < emin ? emin : ex;
    int drop = (52 - mb) + (er - ex);
    unsigned long long keep;
    if (drop > 54) {
        keep = 0;
    } else {
        keep = sig >> drop;
        unsigned long long rem = sig & ((1ull << drop) - 1ull), half = 1ull << (drop - 1);
        if (rem > half || (rem == half && (keep & 1ull))) keep += 1ull;
    }
    if (keep == 0) return sign;
    if (keep >> p) {  // carry into a new binade
        keep >>= 1;
        er += 1;
    }
    if (keep < (1ull << mb)) return sign | (uint32_t)keep;  // subnormal (er == emin)
    uint32_t m = (uint32_t)(keep - (1ull << mb));
    if (er > emax || (prec == LSQ_FP8_E4M3 && er == emax && m == 7u)) return sign | sat_bits;
    return sign | ((uint32_t)(er + bias) << mb) | m;
}

// Store bits produced by quant_bits.
__device__ __forceinline__ void store_bits(void* base, size_t i, uint32_t bits, int prec) {
    switch (prec) {
    case LSQ_FP8_E4M3: ((uint8_t*)base)[i] = (uint8_t)bits; break;
    case LSQ_BF16: case LSQ_FP16: ((uint16_t*)base)[i] = (uint16_t)bits; break;
    default: ((uint32_t*)base)[i] = bits; break;
    }
}

// Storage size in bytes of one element of a sketch precision.
static inline int prec_bytes(int prec) {
    switch (prec) {
    case LSQ_FP8_E4M3: return 1;
    case LSQ_BF16: case LSQ_FP16: return 2;
    case LSQ_FP32: return 4;
    default: return 8;
    }
}

// Store an exactly-representable value in the packed format.
__device__ __forceinline__ void store_prec(void* base, size_t i, double v, int prec) {
    switch (prec) {
    case LSQ_FP8_E4M3: {
        __nv_fp8_storage_t s = __nv_cvt_double_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
        ((__nv_fp8_storage_t*)base)[i] = s;
        break;
    }
    case LSQ_BF16: ((__nv_bfloat16*)base)[i] = __double2bfloat16(v); break;
    case LSQ_FP16: ((__half*)base)[i] = __double2half(v); break;
    case LSQ_FP32: ((float*)base)[i] = (float)v; break;
    default: ((double*)base)[i] = v; break;
    }
}

__device__ __forceinline__ float load_prec_f(const void* base, size_t i, int prec) {
    switch (prec) {
    case LSQ_FP8_E4M3: {
        __half_raw h = __nv_cvt_fp8_to_halfraw(((const __nv_fp8_storage_t*)base)[i], __NV_E4M3);
        return __half2float(__half(h));
    }
    case LSQ_BF16: return __bfloat162float(((const __nv_bfloat16*)base)[i]);
    case LSQ_FP16: return __half2float(((const __half*)base)[i]);
    case LSQ_FP32: return ((const float*)base)[i];
    default: return (float)((const double*)base)[i];
    }
}

// Device-side status word written by kernels that detect a failure.
// info > 0: breakdown at that (1-based) pivot; -1 non-finite; -2 timeout.
__device__ __forceinline__ void set_info_once(int32_t* info, int32_t v) {
    if (info) atomicCAS(info, 0, v);
}

// 2^s (H 2^64 + L), a two's-complement 128-bit integer, rounded once to the
// nearest double (ties to even): the integer is normalised with integer
// operations and the scale goes into the exponent field (no FP64
// instruction).  Straight-line code (selects), so that the compiler
// interleaves independent conversions; results outside the normal range
// scale the rounded 53-bit significand with ldexp (rare).
__device__ __forceinline__ double fixed128_to_double(long long H, unsigned long long L, int s) {
    // magnitude: two's-complement negation of (H:L) when negative
    const unsigned long long sgn = (unsigned long long)(H >> 63);
    const unsigned long long neg = sgn & 1ull;
    const unsigned long long uL = (L ^ sgn) + neg;
    const unsigned long long uH = ((unsigned long long)H ^ sgn) + (neg & (uL == 0 ? 1ull : 0ull));
    const bool zero = (uH | uL) == 0;
    int p = uH ? 127 - __clzll((long long)uH) : 63 - __clzll((long long)uL);
    const int shl = p <= 52 ? 52 - p : 0;  // 0 .. 52
    const int shr = p > 52 ? p - 52 : 0;   // 0 .. 75
    const unsigned long long small = uL << shl;
    // bits p-52 .. p of the magnitude, the round bit below them and the sticky rest
    const unsigned long long big = shr < 64 ? ((uL >> shr) | (shr ? (uH << ((64 - shr) & 63)) : 0ull)) : (uH >> (shr - 64));
    unsigned long long mant = p > 52 ? big : small;
    const int rp = shr - 1;  // position of the round bit (when shr > 0)
    const unsigned long long rb =
        shr == 0 ? 0ull : (rp < 64 ? (uL >> (rp & 63)) & 1ull : (uH >> ((rp - 64) & 63)) & 1ull);
    const bool sticky = shr <= 1 ? false
                        : rp <= 64 ? (uL & ((rp == 64) ? ~0ull : ((1ull << (rp & 63)) - 1ull))) != 0
                                   : (uL != 0 || (uH & ((1ull << ((rp - 64) & 63)) - 1ull)) != 0);
    mant += (rb && (sticky || (mant & 1ull))) ? 1ull : 0ull;
    const bool carry = mant == (1ull << 53);
    mant = carry ? mant >> 1 : mant;
    p += carry ? 1 : 0;
    const int E = p + s + 1023;
    double r = __longlong_as_double((long long)((sgn & 0x8000000000000000ull) | ((unsigned long long)(E & 2047) << 52) |
                                                (mant & 0x000fffffffffffffull)));
    if (zero) r = 0.0;
    if (!zero && (E <= 0 || E >= 2047)) r = ldexp(neg ? -(double)mant : (double)mant, p - 52 + s);
    return r;
}

}  // namespace lsq
