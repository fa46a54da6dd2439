// Gaussian sketch entries: the ziggurat of Marsaglia & Tsang (J. Stat. Softw.
// 5(8), 2000) with 256 layers of equal area v under f(x) = exp(-x^2 / 2),
// x >= 0:
//   layer 0     the rectangle [0, r] x [0, f(r)] plus the tail x > r, drawn
//               as a rectangle of width x_0 = v / f(r);
//   layer i>=1  [0, x_i] x [f(x_i), f(x_{i+1})]: f(x_{i+1}) = f(x_i) + v / x_i,
//               x_1 = r, x_256 = 0;
// v = r f(r) + sqrt(pi/2) erfc(r / sqrt 2), r = 3.6541528853610088 (the root
// of the closure f(x_255) + v / x_255 = 1).  The tables are built once on
// the host in FP64 (no fused multiply-adds: the library's host code is built
// with -ffp-contract=off) and passed to the kernels by value.
//
// Entry (i, j): round k takes the Philox block of counter (i, j_lo, j_hi,
// 2 + 256 k).  A first-kind round: layer L = w0 & 255, sign = bit 8 of w0,
// U = (2^30 (w0 >> 9) + (w1 >> 2)) 2^-53, V = (2^26 (w2 >> 5) + (w3 >> 6))
// 2^-53; z = U x_L is kept if z < x_{L+1}, or (L >= 1) if
// f(x_L) + V (f(x_{L+1}) - f(x_L)) < exp(-z^2 / 2); in layer 0 past r the
// following rounds sample the tail (Marsaglia 1964): U1, U2 = V + 2^-53 from
// (w0, w1) and (w2, w3), e1 = -ln(U1) / r, e2 = -ln(U2), kept when
// 2 e2 > e1^2, giving r + e1.  At most 64 rounds (then 0; the chance of
// getting there is below 1e-100).  Products and sums are explicitly rounded,
// so the draw equals a plain sequential FP64 evaluation up to the accuracy
// of exp and log, which only the rare slow rounds call.
//
// The entry is the draw rounded to the nearest multiple of 2^-17 (ties to
// even), clamped to |Omega| <= 8 - 2^-17: an integer q with |q| < 2^20 times
// 2^-17.  Every entry is an FP32 value, and with the fixed exponent 2^3 it
// has only three nonzero balanced base-128 digits -- the FP64 sketch's
// digit-sliced product then needs 21 digit pairs instead of 36.
//
// The first round, which settles 98.5 % of the entries, runs on the integer
// units only: z = fl(u x_L 2^-53) < x_{L+1} is the integer test u < K_L
// (K_L, the least u for which the rounded product reaches x_{L+1}, is found
// on the host by bisection with the same FP64 product; the product is
// monotone in u), and q = rint(fl(u x_L 2^-53) 2^17) is formed from the
// 106-bit product u M_L (M_L the 53-bit significand of x_L): one rounding to
// 53 significant bits, then one to the integer, both to nearest even --
// the same two roundings as the FP64 evaluation.
#pragma once
#include "common.cuh"

namespace lsq {

constexpr int kZigN = 256;
constexpr double kZigR = 3.6541528853610088;
constexpr uint32_t kZigRounds = 64;
constexpr int32_t kZigQMax = (1 << 20) - 1;  // 8 - 2^-17 on the 2^-17 grid

struct ZigTable {
    double x[kZigN + 1];
    double f[kZigN + 1];
    unsigned long long kfast[kZigN];  // first-round acceptance: u < kfast[L]
};

// Built once per process (thread-safe), in csrc/sketch.cu.
const ZigTable& zig_table();

// The tables in shared memory (with FP32 copies of x and f for the wedge
// test's first try).
struct ZigShared {
    double x[kZigN + 1], f[kZigN + 1];
    unsigned long long kfast[kZigN];
    float x32[kZigN + 1], f32[kZigN + 1];
};

__device__ __forceinline__ void zig_stage(const ZigTable& t, ZigShared& z) {
    for (int q = threadIdx.x; q <= kZigN; q += blockDim.x) {
        z.x[q] = t.x[q];
        z.f[q] = t.f[q];
        z.x32[q] = __double2float_rn(t.x[q]);
        z.f32[q] = __double2float_rn(t.f[q]);
        if (q < kZigN) z.kfast[q] = t.kfast[q];
    }
    __syncthreads();
}

__device__ __forceinline__ double zig_uniform53(uint32_t a, uint32_t b) {
    return (double)(((uint64_t)(a >> 5) << 26) | (b >> 6)) * 0x1p-53;
}

__device__ __forceinline__ unsigned long long zig_u53(uint32_t w0, uint32_t w1) {
    return ((unsigned long long)(w0 >> 9) << 30) | (w1 >> 2);
}

// A draw z (FP64, any sign) on the grid: the signed integer rint(z 2^17),
// clamped to |q| <= 2^20 - 1.  (z 2^17 is exact; rint rounds to nearest even.)
__device__ __forceinline__ int32_t zig_grid_q(double z) {
    const double t = rint(__dmul_rn(z, 131072.0));
    return t > (double)kZigQMax ? kZigQMax : (t < -(double)kZigQMax ? -kZigQMax : (int32_t)t);
}

// rint(fl(u x 2^-53) 2^17) for 0 <= u < 2^53 and a positive normal x, on
// the integer units (see the file comment).
__device__ __forceinline__ int32_t zig_fast_q(unsigned long long u, double x) {
    const unsigned long long xb = (unsigned long long)__double_as_longlong(x);
    const unsigned long long M = (xb & 0x000fffffffffffffull) | 0x0010000000000000ull;
    const int ex = (int)(xb >> 52) - 1023;  // x = M 2^(ex - 52)
    const unsigned long long lo = u * M, hi = __umul64hi(u, M);  // P = u M < 2^106
    if ((lo | hi) == 0) return 0;
    const int nb = hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo);  // bits of P
    // R = P rounded to 53 significant bits (nearest even), P ~ R 2^s1
    unsigned long long R;
    int s1 = 0;
    if (nb <= 53) {
        R = lo;
    } else {
        s1 = nb - 53;  // 1 .. 53
        // top 53 bits, and the dropped bits' relation to one half
        const unsigned long long top = s1 >= 64 ? (hi >> (s1 - 64)) : ((lo >> s1) | (hi << (64 - s1)));
        // remainder below bit s1 against 2^(s1 - 1)
        bool above, exact_half;
        if (s1 <= 64) {
            const unsigned long long rmask = s1 == 64 ? ~0ull : ((1ull << s1) - 1);
            const unsigned long long rem = lo & rmask, half = 1ull << (s1 - 1);
            above = rem > half;
            exact_half = rem == half;
        } else {
            const unsigned long long rhi = hi & ((1ull << (s1 - 64)) - 1), half_hi = 1ull << (s1 - 65);
            above = rhi > half_hi || (rhi == half_hi && lo != 0);
            exact_half = rhi == half_hi && lo == 0;
        }
        R = top;
        if (above || (exact_half && (R & 1ull))) ++R;
        if (R == (1ull << 53)) {
            R >>= 1;
            ++s1;
        }
    }
    // fl(u x 2^-53) 2^17 = R 2^(s1 + ex - 88): round to an integer
    const int sh = 88 - ex - s1;
    unsigned long long q;
    if (sh <= 0) {
        q = (unsigned long long)kZigQMax;  // far above the clamp (not reached: z < r)
    } else if (sh >= 64) {
        q = 0;  // R < 2^54 <= 2^(sh - 1): below one half
    } else {
        q = R >> sh;
        const unsigned long long rem = R & ((1ull << sh) - 1), half = 1ull << (sh - 1);
        if (rem > half || (rem == half && (q & 1ull))) ++q;
    }
    return q > (unsigned long long)kZigQMax ? kZigQMax : (int32_t)q;
}

// The wedge test f(x_L) + V (f(x_{L+1}) - f(x_L)) < exp(-z^2 / 2), z =
// fl(u x_L 2^-53), decided in FP32 where the two sides differ by more than
// 2^-16 relative: the FP32 evaluation (z from the top 32 bits of u, the
// tables and V rounded to FP32, expf within 2 ulp) is within 5e-6 relative
// of the FP64 one, so the decision is the FP64 decision.  1 keep, 0 reject,
// -1 undecided (the FP64 test decides; 0.25 % of the wedge tests).
__device__ __forceinline__ int zig_wedge32(unsigned long long u, uint32_t w2, int L, const ZigShared& Z) {
    const float z = __fmul_rn(__uint2float_rn((uint32_t)(u >> 21)), __fmul_rn(Z.x32[L], 0x1p-32f));
    const float V = __fmul_rn(__uint2float_rn(w2 >> 8), 0x1p-24f);  // V truncated to 24 bits
    const float y = __fadd_rn(Z.f32[L], __fmul_rn(V, __fsub_rn(Z.f32[L + 1], Z.f32[L])));
    const float e = expf(__fmul_rn(__fmul_rn(-0.5f, z), z));
    const float tol = __fmul_rn(e, 0x1p-16f);
    if (y < __fsub_rn(e, tol)) return 1;
    if (y > __fadd_rn(e, tol)) return 0;
    return -1;
}

// Rounds after a first round that did not settle the entry (rare).
// w, L, neg: the first round's words, layer and sign.  Returns q.
static __device__ __noinline__ int32_t gauss_slow_q(uint64_t seed, int64_t i, int64_t j, const ZigShared& Z, U4 w, int L,
                                             bool neg) {
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    unsigned long long u = zig_u53(w.x, w.y);
    bool tail = L == 0;
    for (uint32_t k = 0; k < kZigRounds; ++k) {
        if (k > 0) {
            w = philox(U4{(uint32_t)i, (uint32_t)j, (uint32_t)((uint64_t)j >> 32), 2u + 256u * k}, k0, k1);
            if (!tail) {
                L = (int)(w.x & 255u);
                neg = (w.x >> 8) & 1u;
                u = zig_u53(w.x, w.y);
                if (u < Z.kfast[L]) {
                    const int32_t q = zig_fast_q(u, Z.x[L]);
                    return neg ? -q : q;
                }
                if (L == 0) {
                    tail = true;
                    continue;
                }
            } else {
                const double u1 = __dadd_rn(zig_uniform53(w.x, w.y), 0x1p-53);
                const double u2 = __dadd_rn(zig_uniform53(w.z, w.w), 0x1p-53);
                const double e1 = __ddiv_rn(-log(u1), kZigR);
                const double e2 = -log(u2);
                if (__dadd_rn(e2, e2) > __dmul_rn(e1, e1)) {
                    const double t = __dadd_rn(kZigR, e1);
                    return zig_grid_q(neg ? -t : t);
                }
                continue;
            }
        } else if (tail) {
            continue;  // the first round only sent the draw to the tail
        }
        // the wedge of layer L >= 1 (the kept value is z's grid integer,
        // formed on the integer units as in the first round)
        const int wd = zig_wedge32(u, w.z, L, Z);
        if (wd == 0) continue;
        if (wd < 0) {
            const double z = __dmul_rn((double)u, __dmul_rn(Z.x[L], 0x1p-53));
            const double V = zig_uniform53(w.z, w.w);
            const double y = __dadd_rn(Z.f[L], __dmul_rn(V, __dsub_rn(Z.f[L + 1], Z.f[L])));
            if (!(y < exp(__dmul_rn(__dmul_rn(-0.5, z), z)))) continue;
        }
        const int32_t q = zig_fast_q(u, Z.x[L]);
        return neg ? -q : q;
    }
    return 0;
}

// Omega(i, j) as the signed grid integer q (the entry is q 2^-17).
__device__ __forceinline__ int32_t gauss_q(uint64_t seed, int64_t i, int64_t j, const ZigShared& Z) {
    const U4 w = philox(U4{(uint32_t)i, (uint32_t)j, (uint32_t)((uint64_t)j >> 32), 2u}, (uint32_t)seed,
                        (uint32_t)(seed >> 32));
    const int L = (int)(w.x & 255u);
    const bool neg = (w.x >> 8) & 1u;
    const unsigned long long u = zig_u53(w.x, w.y);
    if (u < Z.kfast[L]) {
        const int32_t q = zig_fast_q(u, Z.x[L]);
        return neg ? -q : q;
    }
    return gauss_slow_q(seed, i, j, Z, w, L, neg);
}

// The entry as FP32 and FP64 values (both exact).
__device__ __forceinline__ float gauss_f32(uint64_t seed, int64_t i, int64_t j, const ZigShared& Z) {
    return __fmul_rn(__int2float_rn(gauss_q(seed, i, j, Z)), 0x1p-17f);
}
__device__ __forceinline__ double gauss_entry(uint64_t seed, int64_t i, int64_t j, const ZigShared& Z) {
    return (double)gauss_f32(seed, i, j, Z);
}

}  // namespace lsq
