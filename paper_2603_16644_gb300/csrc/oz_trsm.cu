// FP64 right triangular solve A_p = A R^{-1} (Alg. 1, "A_p = A R_s^{-1}" by
// substitution) with the off-diagonal work on the 5th-generation tensor cores.
//
// The columns are split recursively, [c0, c1) -> [c0, mid) + [mid, c1):
//   A_p[:, c0:mid]  = solve of the left part,
//   A_p[:, mid:c1]  = A[:, mid:c1] - A_p[:, c0:mid] R[c0:mid, mid:c1],
//   then the right part is solved in place.
// Diagonal blocks of at most OT_NB columns are solved by FP64 substitution
// (one thread per row).  The updates are FP64-accurate products built from
// BF16 digit slices:
//
//   x = 2^(E - 55) sum_{t=0}^{7} d_t 128^(7 - t) + r,  d_t in [-64, 64],
//   0 <= |r| < 2^(E - 55),
//
// with 2^E bounding the row of X (resp. the column of Y) that x belongs to.
// Every digit-pair product d_t d_u is an integer of magnitude <= 2^12, so the
// (d + 1) <= 8 pairs with t + u = d summed over K <= 512 stay <= 2^24 and are
// exact in the FP32 accumulators of tcgen05.mma (kind::f16, BF16 operands).
// Pairs with t + u <= 7 are kept (36 of 64); each group d has its own TMEM
// accumulator.  The epilogue turns the 8 group sums into two exact 64-bit
// fixed-point integers and rounds once to FP64:
//
//   sum_k X[i,k] Y[k,j] ~= 2^(Ex_i + Ey_j - 61) (hi 2^28 + lo),
//   hi = sum_{d<4} S_d 128^(3-d),  lo = sum_{d>=4} S_d 128^(7-d).
//
// Per product the dropped pairs and the truncations r contribute below
// 2^-52.6 * 2^(Ex_i + Ey_j), the order of FP64 rounding.
#include "common.cuh"
#include "gauss.cuh"
#include "kernels.cuh"
#include "tcgen05.cuh"

#include <algorithm>
#include <type_traits>

namespace lsq {

constexpr int OT_DIG = 8;                   // digits per value
constexpr int OT_BM = 128, OT_BN = 64;      // output tile (rows x columns)
constexpr int OT_BK = 64;                   // K per stage: 64 BF16 = 128 bytes
constexpr int OT_XST = 6;                   // stages of X digit tiles
constexpr int OT_KMAX = 512;                // exact FP32 group sums up to this K
constexpr int OT_KMAX3 = 1024;              // the same with three X digits (at most 3 pairs per group)
constexpr int OT_NB = 32;                   // diagonal block solved by substitution
constexpr int OT_THREADS = 608;             // warp 0 TMA, warps 1-2 MMA, warps 3-18 epilogue
constexpr int OT_XTILE = OT_BM * 128;       // bytes of one X digit tile
constexpr int OT_YTILE = OT_BN * 128;       // bytes of one Y digit tile
constexpr int32_t OT_NONFINITE = 0x7fffffff;

// ---------------------------------------------------------------------------
// Digit slicing (integer operations on the FP64 bit pattern)
// ---------------------------------------------------------------------------
// mx: the largest |x| bit pattern of a row or column.  The exponent field is
// masked: a NaN produced by arithmetic may keep its sign bit even after the
// magnitude mask (the compiler may fold the mask into an FP absolute value).
__device__ __forceinline__ int32_t ot_exp_of_max(unsigned long long mx) {
    int Eb = (int)((mx >> 52) & 0x7ff);
    if (Eb == 0x7ff) return OT_NONFINITE;
    if (mx == 0) return 0;
    return (Eb > 1 ? Eb : 1) - 1022;  // every |x| < 2^E
}

constexpr unsigned long long OT_BIAS =
    64ull * ((1ull << 42) + (1ull << 35) + (1ull << 28) + (1ull << 21) + (1ull << 14) + (1ull << 7) + 1ull);

// Balanced base-128 digits of x with |x| < 2^E (see the file comment), as
// the fields of W = V + BIAS, V = trunc(x 2^(55 - E)) in two's complement:
// adding 64 to every lower 7-bit field makes each field t >= 1 equal to
// d_t + 64 (d_t in [-64, 63]), and the arithmetic top W >> 49 is d_0 in
// [-64, 64].  A non-finite x or row exponent gives V = 0.
__device__ __forceinline__ unsigned long long ot_fields(double x, int32_t E) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const bool neg = (b >> 63) != 0;
    const int Eb = (int)((b >> 52) & 0x7ff);
    unsigned long long sig = b & 0x000fffffffffffffull;
    if (Eb != 0) sig |= 0x0010000000000000ull;
    unsigned long long V = 0;
    if (E != OT_NONFINITE && Eb != 0x7ff) {
        // only for a finite row exponent: E + 1022 must not be formed from the
        // non-finite marker (signed overflow would let the compiler assume
        // that E is never the marker)
        const int sh = (Eb != 0 ? Eb : 1) - (E + 1022) + 2;  // <= 2, so V < 2^55
        V = sh >= 0 ? (sig << sh) : (sh > -64 ? (sig >> (-sh)) : 0ull);
    }
    return (neg ? 0ull - V : V) + OT_BIAS;
}

// Digit t of W as an FP32 value: 2^23 1.5 + field, minus the same plus 64
// (exact integer arithmetic in FP32, no conversion instruction).  Its upper
// half is the BF16 encoding (the digit has at most 7 significant bits).
__device__ __forceinline__ uint32_t ot_digit_f32(unsigned long long W, int t) {
    const uint32_t f = t == 0 ? (uint32_t)((int)((long long)W >> 49) + 64)
                              : (uint32_t)((W >> (7 * (OT_DIG - 1 - t))) & 127ull);
    return __float_as_uint(__uint_as_float(0x4B400000u | f) - 12582976.0f);
}

// BF16 digits t of two values, packed (first value in the low half).
__device__ __forceinline__ uint32_t ot_digit_pair(unsigned long long W0, unsigned long long W1, int t) {
    return __byte_perm(ot_digit_f32(W0, t), ot_digit_f32(W1, t), 0x7632);
}

// Rows of X (m x K, column-major): Ex[i] and digit planes Z[(t mp + i) Kp + k]
// (K-contiguous; zero for rows m <= i < mp and for K <= k < Kp, so that every
// TMA box lies inside the planes), with the row exponents from per-block
// exponents (Eblk[b m + i] for blocks b0 .. b0+nbk-1, INT32_MIN for an
// all-zero block): a 2-D grid, one thread per row and 64-wide range of K
// (blockIdx.y), so that many loads are in flight.
__global__ void __launch_bounds__(128) k_ot_rowslice_e(const double* __restrict__ X, int64_t m, int64_t mp,
                                                       int64_t K, int64_t ld, int64_t Kp, int32_t* __restrict__ Ex,
                                                       uint16_t* __restrict__ Z, const int32_t* __restrict__ Eblk,
                                                       int64_t b0, int nbk) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= mp) return;
    int32_t eb = INT32_MIN;
    if (i < m)
        for (int b = 0; b < nbk; ++b) eb = max(eb, Eblk[(b0 + b) * m + i]);
    const int32_t E = eb == INT32_MIN ? 0 : eb;
    const int64_t kb = (int64_t)blockIdx.y * 64;
    if (blockIdx.y == 0) Ex[i] = E;
    const double* row = X + i;
    const int64_t Kr = i < m ? K : 0;
#pragma unroll 1
    for (int64_t k0 = kb; k0 < kb + 64; k0 += 16) {
        double xv[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) xv[q] = k0 + q < Kr ? row[(k0 + q) * ld] : 0.0;
        uint32_t pk[OT_DIG][8];
#pragma unroll
        for (int q2 = 0; q2 < 8; ++q2) {
            const unsigned long long W0 = ot_fields(xv[2 * q2], E), W1 = ot_fields(xv[2 * q2 + 1], E);
#pragma unroll
            for (int t = 0; t < OT_DIG; ++t) pk[t][q2] = ot_digit_pair(W0, W1, t);
        }
        // 32 bytes (one sector) per digit plane
#pragma unroll
        for (int t = 0; t < OT_DIG; ++t) {
            uint4* dst = (uint4*)(Z + ((int64_t)t * mp + i) * Kp + k0);
            dst[0] = make_uint4(pk[t][0], pk[t][1], pk[t][2], pk[t][3]);
            dst[1] = make_uint4(pk[t][4], pk[t][5], pk[t][6], pk[t][7]);
        }
    }
}

// Row maxima of |X| (bit patterns, the sign cleared; atomicMax orders them
// like the values) over 64-wide K ranges, one thread per row; Mx zeroed.
__global__ void __launch_bounds__(128) k_ot_rowmax2d(const double* __restrict__ X, int64_t m, int64_t K, int64_t ld,
                                                     unsigned long long* __restrict__ Mx) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int64_t k0 = (int64_t)blockIdx.y * 64, k1 = min64(K, k0 + 64);
    unsigned long long mx = 0;
    for (int64_t k = k0; k < k1; ++k) {
        const unsigned long long a = (unsigned long long)__double_as_longlong(X[i + k * ld]) & 0x7fffffffffffffffull;
        mx = a > mx ? a : mx;
    }
    if (mx) atomicMax(&Mx[i], mx);
}

// The rows' exponents in the per-block convention (INT32_MIN for a zero row).
__global__ void k_ot_rowexp(const unsigned long long* __restrict__ Mx, int64_t m, int32_t* __restrict__ Eb) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) Eb[i] = Mx[i] == 0 ? INT32_MIN : ot_exp_of_max(Mx[i]);
}

// The same, with the digit planes written as whole 128-byte lines: a CTA
// converts a 64-row x 64-column block of X (two threads per row, 32 columns
// each, reading X a column at a time, coalesced over rows), stages the 8 BF16
// digit tiles in shared memory in the 128-byte-swizzled layout of the TMA
// (16-byte chunk j of row r at chunk j ^ (r mod 8): conflict-free for one
// thread per row), and stores each plane's tile with one TMA store.  (Stores
// of 16 bytes to 32 different rows per warp instruction reach ~1 TB/s; whole
// lines reach ~6 TB/s.)  tmZ: the X digit planes, boxes of 64 columns x 64
// rows x 1 plane.
constexpr int OT_RS_ROWS = 64;
// tma_x: X's block comes in by one TMA load (tmX: FP64, boxes of 64 rows x 64
// columns, zero outside) into shared memory [64 columns][64 rows]; otherwise
// every thread loads its values (coalesced over rows, a column at a time).
// own_exp (with tma_x, K <= 64): the row exponents are those of the rows'
// largest values, formed here (the two threads of a row combine their maxima)
// instead of from the diagonal kernel's per-block exponents.
template <bool tma_x, bool own_exp>
__global__ void __launch_bounds__(128) k_ot_rowslice_s(const __grid_constant__ CUtensorMap tmZ,
                                                       const __grid_constant__ CUtensorMap tmX,
                                                       const double* __restrict__ X, int64_t m, int64_t mp, int64_t K,
                                                       int64_t ld, int32_t* __restrict__ Ex,
                                                       const int32_t* __restrict__ Eblk, int64_t b0, int nbk,
                                                       int32_t* __restrict__ err) {
    extern __shared__ unsigned char rs_raw[];
    uint8_t* stage = (uint8_t*)(((uintptr_t)rs_raw + 1023) & ~(uintptr_t)1023);  // [8][64 rows][128 B]
    const double* xt = (const double*)(stage + OT_DIG * OT_RS_ROWS * 128);      // [64 columns][64 rows]
    __shared__ uint64_t xfull;
    __shared__ unsigned long long rmax[2][OT_RS_ROWS];
    __shared__ int rs_bad;
    const int r = threadIdx.x & (OT_RS_ROWS - 1), h = threadIdx.x >> 6;
    const int64_t i0 = (int64_t)blockIdx.x * OT_RS_ROWS, kb = (int64_t)blockIdx.y * 64;
    const int64_t i = i0 + r;
    static_assert(tma_x || !own_exp, "own exponents need the staged block");
    if constexpr (tma_x) {
        if (threadIdx.x == 0) {
            rs_bad = 0;
            mbar_init(&xfull, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            mbar_expect_tx(&xfull, OT_RS_ROWS * 64 * 8);
            tma_load_2d((void*)xt, &tmX, &xfull, (int)i0, (int)kb);
        }
        __syncthreads();
    }
    int32_t E = 0;
    if constexpr (!own_exp) {
        int32_t eb = INT32_MIN;
        if (i < m)
            for (int b = 0; b < nbk; ++b) eb = max(eb, Eblk[(b0 + b) * m + i]);
        E = eb == INT32_MIN ? 0 : eb;
    }
    const double* row = X + i;
    const int64_t Kr = i < m ? K : 0;
    if constexpr (tma_x) {
        if (!mbar_wait(&xfull, 0)) rs_bad = 1;
        __syncthreads();
        if (rs_bad) {  // every thread leaves here together
            if (threadIdx.x == 0) {
                set_info_once(err, -2);
                mbar_wait(&xfull, 0);  // bounded: the copy in flight, before the CTA ends
            }
            return;
        }
    }
    if constexpr (own_exp) {
        unsigned long long mx = 0;
        for (int q = 0; q < 32; ++q) {
            const unsigned long long v =
                (unsigned long long)__double_as_longlong(xt[(32 * h + q) * OT_RS_ROWS + r]) & 0x7fffffffffffffffull;
            mx = v > mx ? v : mx;
        }
        rmax[h][r] = mx;
        __syncthreads();
        mx = rmax[0][r] > rmax[1][r] ? rmax[0][r] : rmax[1][r];
        E = ot_exp_of_max(mx);
    }
    if (blockIdx.y == 0 && h == 0) Ex[i] = E;
#pragma unroll 1
    for (int bb = 0; bb < 2; ++bb) {
        const int kl = 32 * h + 16 * bb;  // first of 16 columns within the block
        const int64_t k0 = kb + kl;
        double xv[16];
        if constexpr (tma_x) {
#pragma unroll
            for (int q = 0; q < 16; ++q) xv[q] = xt[(kl + q) * OT_RS_ROWS + r];  // zero outside X (TMA fill)
        } else {
#pragma unroll
            for (int q = 0; q < 16; ++q) xv[q] = k0 + q < Kr ? row[(k0 + q) * ld] : 0.0;
        }
        uint32_t pk[OT_DIG][8];
#pragma unroll
        for (int q2 = 0; q2 < 8; ++q2) {
            const unsigned long long W0 = ot_fields(xv[2 * q2], E), W1 = ot_fields(xv[2 * q2 + 1], E);
#pragma unroll
            for (int t = 0; t < OT_DIG; ++t) pk[t][q2] = ot_digit_pair(W0, W1, t);
        }
        const int j = kl / 8;  // first 16-byte chunk of the 32 bytes of these columns
#pragma unroll
        for (int t = 0; t < OT_DIG; ++t) {
            uint8_t* rowp = stage + ((size_t)t * OT_RS_ROWS + r) * 128;
            *(uint4*)(rowp + ((j ^ (r & 7)) << 4)) = make_uint4(pk[t][0], pk[t][1], pk[t][2], pk[t][3]);
            *(uint4*)(rowp + (((j + 1) ^ (r & 7)) << 4)) = make_uint4(pk[t][4], pk[t][5], pk[t][6], pk[t][7]);
        }
    }
    // the tiles are written through the generic proxy and read by the TMA
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int t = 0; t < OT_DIG; ++t)
            tma_store_3d(&tmZ, stage + (size_t)t * OT_RS_ROWS * 128, (int)kb, (int)i0, t);
        tma_store_wait_read();
    }
    __syncthreads();
}

// Columns of Y (K x N, entry (k, j) at Y[k sk + j sj]): Ey[j] and digit
// planes Z[(u Np + j) Kp + k] (zero for columns N <= j < Np and for
// K <= k < Kp).  One CTA per column.
__global__ void __launch_bounds__(128) k_ot_colslice(const double* __restrict__ Y, int64_t K, int64_t N, int64_t Np,
                                                     int64_t sk, int64_t sj, int64_t Kp, int32_t* __restrict__ Ey,
                                                     uint16_t* __restrict__ Z) {
    const int64_t j = blockIdx.x;
    const double* col = Y + j * sj;
    const int64_t Kr = j < N ? K : 0;
    unsigned long long mx = 0;
    for (int64_t k = threadIdx.x; k < Kr; k += blockDim.x) {
        unsigned long long v = (unsigned long long)__double_as_longlong(col[k * sk]) & 0x7fffffffffffffffull;
        mx = v > mx ? v : mx;
    }
    for (int off = 16; off > 0; off >>= 1) {
        unsigned long long o = __shfl_xor_sync(0xffffffffu, mx, off);
        mx = o > mx ? o : mx;
    }
    __shared__ unsigned long long w[4];
    __shared__ int32_t Es;
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int q = 0; q < 4; ++q) t = w[q] > t ? w[q] : t;
        Es = ot_exp_of_max(t);
        Ey[j] = Es;
    }
    __syncthreads();
    const int32_t E = Es;
    for (int64_t k = threadIdx.x; k < Kp; k += blockDim.x) {
        const unsigned long long W = ot_fields(k < Kr ? col[k * sk] : 0.0, E);
#pragma unroll
        for (int u = 0; u < OT_DIG; ++u) Z[((int64_t)u * Np + j) * Kp + k] = (uint16_t)(ot_digit_f32(W, u) >> 16);
    }
}

// ---------------------------------------------------------------------------
// Update C_out = C_in - X Y over 128 x 64 tiles (C_in may equal C_out).
// ---------------------------------------------------------------------------
// Results outside the normal range (rare): scaled in FP64.  Not inlined, so
// that the FP64 instructions of this path are never executed speculatively.
__device__ __noinline__ double ot_fixed_to_double_slow(long long hi, long long lo, int s) {
    return ldexp(fma((double)hi, 268435456.0, (double)lo), s);
}

// 2^s (hi 2^28 + lo) for |hi|, |lo| < 2^47, rounded once to nearest-even:
// the exact integer (below 2^76) is normalised with integer operations and
// the scale goes into the exponent field (no FP64 instruction on the common
// path).  Straight-line code (selects), so that the compiler interleaves
// independent conversions; the epilogue's throughput is bound by these
// integer operations when K is small.
__device__ __forceinline__ double ot_fixed_to_double(long long hi, long long lo, int s) {
    unsigned long long L = (unsigned long long)hi << 28;
    long long H = hi >> 36;
    const unsigned long long L2 = L + (unsigned long long)lo;
    H += (lo >> 63) + (L2 < L ? 1 : 0);
    L = L2;
    // magnitude: two's-complement negation of (H:L) when negative (H < 2^11)
    const unsigned long long sgn = (unsigned long long)(H >> 63);
    const unsigned long long neg = sgn & 1ull;
    const unsigned long long uL = (L ^ sgn) + neg;
    const unsigned long long uH = ((unsigned long long)H ^ sgn) + (neg & (uL == 0 ? 1ull : 0ull));
    const bool zero = (uH | uL) == 0;
    int p = uH ? 127 - __clzll((long long)uH) : 63 - __clzll((long long)uL);
    const int shl = p <= 52 ? 52 - p : 0;  // 0 .. 52
    const int shr = p > 52 ? p - 52 : 0;   // 0 .. 22
    const unsigned long long small = uL << shl;
    const unsigned long long big = (uL >> shr) | (shr ? (uH << ((64 - shr) & 63)) : 0ull);
    unsigned long long mant = p > 52 ? big : small;
    const unsigned long long rb = shr ? (uL >> ((shr - 1) & 63)) & 1ull : 0ull;
    const bool sticky = shr > 1 ? (uL & ((1ull << ((shr - 1) & 63)) - 1ull)) != 0 : false;
    mant += (rb && (sticky || (mant & 1ull))) ? 1ull : 0ull;
    const bool carry = mant == (1ull << 53);
    mant = carry ? mant >> 1 : mant;
    p += carry ? 1 : 0;
    const int E = p + s + 1023;
    double r = __longlong_as_double((long long)((sgn & 0x8000000000000000ull) | ((unsigned long long)(E & 2047) << 52) |
                                                (mant & 0x000fffffffffffffull)));
    if (zero) r = 0.0;
    if (!zero && (E <= 0 || E >= 2047)) r = ot_fixed_to_double_slow(hi, lo, s);
    return r;
}

// Persistent: one CTA per SM walks the tiles (column tiles fastest, so that
// CTAs sharing a row block of X digits run together).  Warp 0 streams the
// digit tiles of consecutive tiles through the rings; warps 1 and 2 issue the
// MMAs of a tile as soon as the epilogue has taken the previous tile's group
// sums out of TMEM (tfree); warps 3-18 drain TMEM into registers, release it,
// and convert and store while the next tile's MMAs run.
// 19 warps: three of the four schedulers hold 5 warps, and a scheduler's
// register file (16 K registers) then allows 96 registers per thread.
constexpr int OT_EPI_WARPS = 16;

// Tile t -> (first row, first column).  GROUPED: bands of OT_GM row tiles
// with the row tiles fastest inside a band, so that a wave of CTAs spans about
// OT_GM row tiles and gridDim / OT_GM column tiles and shares the digit tiles
// of both operands through L2.  The FP64 sketch's 64 x 64 tiles use it: with
// the column tiles fastest over all rows a wave spanned 2.4 row tiles and read
// the Y digit planes once per wave (2.3 -> 1.1 GB of DRAM traffic per launch,
// 1.7 % less time).  The TRSM updates (many row tiles, few column tiles) keep
// the column tiles fastest: a CTA then stays on one column tile, and the
// banded order raised their traffic by 30 % at the same time.
constexpr int OT_GM = 8;
template <bool GROUPED>
__device__ __forceinline__ void ot_tile_coords(int t, int ntj, int nti, int64_t& i0, int64_t& j0) {
    if (!GROUPED) {
        i0 = (int64_t)(t / ntj) * OT_BM;
        j0 = (int64_t)(t % ntj) * OT_BN;
        return;
    }
    const int per = OT_GM * ntj;
    const int first = (t / per) * OT_GM;
    const int gs = min(nti - first, OT_GM);
    const int w = t % per;
    i0 = (int64_t)(first + w % gs) * OT_BM;
    j0 = (int64_t)(w / gs) * OT_BN;
}

// XD: digits of X taken (8, or 3 when X's lower digits are known to vanish);
// pairs (t, u) with t < XD and t + u <= 7.
template <int XD>
__global__ void __launch_bounds__(OT_THREADS, 1)
    k_ot_update(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY, int64_t m,
                int64_t N, int64_t K, const int32_t* __restrict__ Ex, const int32_t* __restrict__ Ey,
                const double* Cin, int64_t ldi, double* Cout, int64_t ldo, int32_t* __restrict__ err, int ntj,
                int ntiles) {
    extern __shared__ unsigned char ot_raw[];
    uint8_t* base = (uint8_t*)(((uintptr_t)ot_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sY = base;                                // 2 stages x 8 digit tiles
    uint8_t* sX = sY + 2 * OT_DIG * OT_YTILE;          // OT_XST stages x 1 tile
    uint64_t* yfull = (uint64_t*)(sX + OT_XST * OT_XTILE);
    uint64_t* yempty = yfull + 2;
    uint64_t* xfull = yempty + 2;
    uint64_t* xempty = xfull + OT_XST;
    uint64_t* accf = xempty + OT_XST;  // MMA -> epilogue: a tile's group sums are complete
    uint64_t* tfree = accf + 1;        // epilogue -> MMA: TMEM has been read
    uint64_t* mdone = tfree + 1;       // every MMA of the CTA has completed
    uint32_t* tslot = (uint32_t*)(mdone + 1);
    volatile int* bad = (volatile int*)(tslot + 1);
    int* cnt = (int*)(tslot + 2);  // x issued, x consumed (issuer 0), y issued, y consumed (0), x / y consumed (1)

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nslab = (int)((K + OT_BK - 1) / OT_BK);
    const int ntl = ntiles > (int)blockIdx.x ? (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&yfull[s], 1);
            mbar_init(&yempty[s], 2);
        }
        for (int s = 0; s < OT_XST; ++s) {
            mbar_init(&xfull[s], 1);
            mbar_init(&xempty[s], 2);
        }
        mbar_init(accf, 2);
        mbar_init(tfree, OT_EPI_WARPS);
        mbar_init(mdone, 2);
        *bad = 0;
        cnt[0] = cnt[1] = cnt[2] = cnt[3] = cnt[4] = cnt[5] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(tslot, 512);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    if (warp == 0 && lane == 0) {
        // producer: per slab the 8 Y digit tiles (the next slab's go out after
        // X tile 3 of the current one, or after its last), then the XD X digit
        // tiles
        const int total = ntl * nslab;  // slabs over all tiles of this CTA
        auto slab_tile = [&](int g, int64_t& i0, int64_t& j0, int& s) {
            const int tl = (int)blockIdx.x + (g / nslab) * (int)gridDim.x;
            s = g % nslab;
            ot_tile_coords<XD == 3>(tl, ntj, ntiles / ntj, i0, j0);
        };
        auto load_y = [&](int g) -> bool {
            int64_t i0, j0;
            int s;
            slab_tile(g, i0, j0, s);
            const int ys = g & 1;
            if (g >= 2 && !mbar_wait(&yempty[ys], (uint32_t)(((g >> 1) - 1) & 1))) return false;
            mbar_expect_tx(&yfull[ys], OT_DIG * OT_YTILE);
            for (int u = 0; u < OT_DIG; ++u)
                tma_load_3d(sY + (ys * OT_DIG + u) * OT_YTILE, &tmY, &yfull[ys], s * OT_BK, (int)j0, u);
            cnt[2] = g + 1;
            return true;
        };
        int xq = 0;
        if (total > 0 && !load_y(0)) *bad = 1;
        for (int g = 0; g < total && !*bad; ++g) {
            int64_t i0, j0;
            int s;
            slab_tile(g, i0, j0, s);
            constexpr int YT = XD > 4 ? 4 : XD - 1;
            for (int t = 0; t < XD; ++t, ++xq) {
                if (t == YT && g + 1 < total && !load_y(g + 1)) {
                    *bad = 1;
                    break;
                }
                const int xs = xq % OT_XST;
                if (xq >= OT_XST && !mbar_wait(&xempty[xs], (uint32_t)(((xq / OT_XST) - 1) & 1))) {
                    *bad = 1;
                    break;
                }
                mbar_expect_tx(&xfull[xs], OT_XTILE);
                tma_load_3d(sX + xs * OT_XTILE, &tmX, &xfull[xs], s * OT_BK, (int)i0, t);
                cnt[0] = xq + 1;
            }
        }
    } else if (warp == 1 || warp == 2) {
        // MMA issuers: pair (t, u) with t + u <= 7 into accumulator t + u.
        // Two warps issue, each owning the accumulators of its groups (18
        // pairs each): no two threads accumulate into the same TMEM columns.
        // The 4 K steps of one pair go back to back into the same accumulator
        // (measured: interleaving accumulators, even with operand A kept in
        // the collector buffer, is 40 % - 3x slower).  Each warp runs its loop
        // in convergence, fully unrolled over the digits with the ownership
        // fixed at compile time, so that the descriptors are warp-uniform
        // values; lane 0 issues (measured: descriptors formed per MMA by a
        // single divergent thread cost ~160 cycles per MMA and issuer, against
        // ~48 cycles per MMA for the pair when they are uniform).  Both
        // commit every stage and tile.
        const uint32_t lead = lane == 0 ? 1u : 0u;
        auto issue = [&](auto issc) {
            constexpr int ISS = decltype(issc)::value;
            constexpr unsigned OWN1 = (1u << 1) | (1u << 2) | (1u << 5) | (1u << 6);  // groups of issuer 1
            constexpr uint32_t idesc = umma_idesc(1u, OT_BM, OT_BN);
            const uint64_t dx0 = umma_desc(smem_u32(sX)), dy0 = umma_desc(smem_u32(sY));
            int xq = 0, g = 0;
            for (int i = 0; i < ntl; ++i) {
                if (__shfl_sync(0xffffffffu, *bad, 0)) return;
                if (i > 0 && !__all_sync(0xffffffffu, mbar_wait(tfree, (uint32_t)((i - 1) & 1)))) {
                    *bad = 1;
                    return;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                for (int s = 0; s < nslab; ++s, ++g, xq += XD) {
                    const int ys = g & 1;
                    if (!__all_sync(0xffffffffu, mbar_wait(&yfull[ys], (uint32_t)((g >> 1) & 1)))) {
                        *bad = 1;
                        return;
                    }
                    if (lead) cnt[ISS ? 5 : 3] = g + 1;
                    const uint64_t dy = dy0 + (uint64_t)(ys * (OT_DIG * OT_YTILE >> 4));
                    // 16-wide K steps past K (zero digits) are not issued: lane
                    // 0's issue predicate per step, set once per slab
                    const int64_t krem = K - (int64_t)s * OT_BK;
                    const uint32_t lk[4] = {lead, krem > 16 ? lead : 0u, krem > 32 ? lead : 0u, krem > 48 ? lead : 0u};
#pragma unroll
                    for (int t = 0; t < XD; ++t) {
                        const int xs = (xq + t) % OT_XST;
                        if (!__all_sync(0xffffffffu, mbar_wait(&xfull[xs], (uint32_t)(((xq + t) / OT_XST) & 1)))) {
                            *bad = 1;
                            return;
                        }
                        if (lead) cnt[ISS ? 4 : 1] = xq + t + 1;
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint64_t ad = dx0 + (uint64_t)(xs * (OT_XTILE >> 4));
#pragma unroll
                        for (int u = 0; u + t < OT_DIG; ++u) {
                            if ((int)((OWN1 >> (t + u)) & 1u) != ISS) continue;
                            const uint64_t bd = dy + (uint64_t)(u * (OT_YTILE >> 4));
                            const uint32_t acc = tmem + (uint32_t)((t + u) * OT_BN);
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk)  // 4 x 16 BF16 of K per stage
                                umma_f16_w(acc, ad + 2 * kk, bd + 2 * kk, idesc, (s | t | kk) != 0 ? 1u : 0u, lk[kk]);
                        }
                        umma_commit_w(&xempty[xs], lead);
                    }
                    umma_commit_w(&yempty[ys], lead);
                }
                umma_commit_w(accf, lead);  // fires when this issuer's MMAs of the tile have completed
            }
        };
        if (warp == 1) issue(std::integral_constant<int, 0>());
        else issue(std::integral_constant<int, 1>());
    } else if (warp >= 3) {
        // epilogue warp e = warp - 3: TMEM lane quadrant warp % 4 (its rows)
        // and a quarter of the tile's columns: [16 (e / 4), +16), or
        // [8 (e / 4), +8) when the tile has at most 32 valid columns (so that
        // every epilogue warp has work in the narrow updates)
        const int quad = warp & 3, cq = (warp - 3) >> 2;
        const uint32_t tq = tmem + ((uint32_t)(quad * 32) << 16);
        // drain W columns of the 8 group sums, release the TMEM, convert and store
        auto epi = [&](auto Wc, int64_t row, int64_t c0) {
            constexpr int W = decltype(Wc)::value;
            const uint32_t tl = tq + (uint32_t)(cq * W);
            long long hi[W], lo[W];
#pragma unroll
            for (int d = 0; d < OT_DIG; d += 2) {
                uint32_t va[W], vb[W];
                if constexpr (W == 16) {
                    tmem_ld16_nowait(tl + (uint32_t)(d * OT_BN), va);
                    tmem_ld16_nowait(tl + (uint32_t)((d + 1) * OT_BN), vb);
                } else {
                    tmem_ld8_nowait(tl + (uint32_t)(d * OT_BN), va);
                    tmem_ld8_nowait(tl + (uint32_t)((d + 1) * OT_BN), vb);
                }
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < W; ++j) {
                    const long long a = (long long)__float2int_rn(__uint_as_float(va[j]));
                    const long long b = (long long)__float2int_rn(__uint_as_float(vb[j]));
                    if (d == 0) hi[j] = a * 128 + b;
                    else if (d == 2) hi[j] = (hi[j] * 128 + a) * 128 + b;
                    else if (d == 4) lo[j] = a * 128 + b;
                    else lo[j] = (lo[j] * 128 + a) * 128 + b;
                }
            }
            // this tile's TMEM is read: the next tile's MMAs may start
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(tfree);
            if (row < m) {
                const int32_t ex = Ex[row];
#pragma unroll
                for (int h = 0; h < W / 8; ++h) {
                    double cin[8];
                    int32_t ey[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int64_t col = c0 + 8 * h + j;
                        cin[j] = col < N ? Cin[row + col * ldi] : 0.0;
                        ey[j] = col < N ? Ey[col] : 0;
                    }
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int64_t col = c0 + 8 * h + j;
                        if (col < N) {
                            double val;
                            if (ex == OT_NONFINITE || ey[j] == OT_NONFINITE)
                                val = __longlong_as_double(0x7ff8000000000000ll);
                            else
                                val = ot_fixed_to_double(hi[8 * h + j], lo[8 * h + j], ex + ey[j] - 61);
                            Cout[row + col * ldo] = cin[j] - val;
                        }
                    }
                }
            }
        };
        for (int i = 0; i < ntl; ++i) {
            const int tile = (int)blockIdx.x + i * (int)gridDim.x;
            int64_t i0, j0;
            ot_tile_coords<XD == 3>(tile, ntj, ntiles / ntj, i0, j0);
            const int64_t row = i0 + quad * 32 + lane;
            const bool narrow = N - j0 <= 32;
            const int64_t c0 = j0 + cq * (narrow ? 8 : 16);
            if (row < m) {  // this tile's C_in entries into L2 while its MMAs run
                for (int j = 0; j < (narrow ? 8 : 16); ++j)
                    if (c0 + j < N) asm volatile("prefetch.global.L2 [%0];" ::"l"(Cin + row + (c0 + j) * ldi));
            }
            const bool ok = mbar_wait(accf, (uint32_t)(i & 1));
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (!ok) *bad = 1;
            if (!__all_sync(0xffffffffu, ok && !*bad)) break;
            if (narrow) epi(std::integral_constant<int, 8>(), row, c0);
            else epi(std::integral_constant<int, 16>(), row, c0);
        }
    }
    if ((warp == 1 || warp == 2) && lane == 0) umma_commit(mdone);  // fires when every MMA issued has completed
    __syncthreads();
    if (*bad) {
        if (threadIdx.x == 0) {
            set_info_once(err, -2);
            // wait (bounded) for copies issued but never consumed, then the MMAs
            for (int q = min(cnt[1], cnt[4]); q < cnt[0]; ++q)
                mbar_wait(&xfull[q % OT_XST], (uint32_t)((q / OT_XST) & 1));
            for (int g = min(cnt[3], cnt[5]); g < cnt[2]; ++g) mbar_wait(&yfull[g & 1], (uint32_t)((g >> 1) & 1));
            mbar_wait(mdone, 0);
        }
        __syncthreads();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        tmem_dealloc(tmem, 512);
    }
}

// ---------------------------------------------------------------------------
// Diagonal block: Ap[i, 0:nc] = src[i, 0:nc] R_jj^{-1} (R_jj upper, nc <= NB)
// by substitution, one thread per row.  Each x_j is scaled by the reciprocal
// of R[j, j] (one rounding more than a division).
// ---------------------------------------------------------------------------
// Also records, per row, the exponent of the largest |x| of the block
// (Eblk[blk m + i], INT32_MIN if the block row is zero), from which the
// updates take the row exponents of their X operand without a pass over it.
template <int NB>
__global__ void __launch_bounds__(64) k_ot_diag(const double* src, int64_t lds, const double* __restrict__ R,
                                                 int64_t ldr, int nc, int64_t m, double* Ap, int64_t ldap,
                                                 int32_t* __restrict__ Eblk, int64_t blk) {
    __shared__ double Rb[NB][NB];
    __shared__ double rinv[NB];
    for (int q = threadIdx.x; q < NB * NB; q += blockDim.x) {
        int k = q % NB, j = q / NB;
        Rb[k][j] = (k < nc && j < nc) ? R[k + (int64_t)j * ldr] : (k == j ? 1.0 : 0.0);
    }
    __syncthreads();
    if (threadIdx.x < NB) rinv[threadIdx.x] = 1.0 / Rb[threadIdx.x][threadIdx.x];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double x[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) x[j] = j < nc ? src[i + (int64_t)j * lds] : 0.0;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        double v = x[j];
#pragma unroll
        for (int k = 0; k < j; ++k) v = fma(-x[k], Rb[k][j], v);
        x[j] = v * rinv[j];
    }
#pragma unroll
    for (int j = 0; j < NB; ++j)
        if (j < nc) Ap[i + (int64_t)j * ldap] = x[j];
    // the row maximum from the values just stored (this thread's own writes),
    // so that the substitution keeps its register footprint
    unsigned long long mx = 0;
    for (int j = 0; j < nc; ++j) {
        const unsigned long long a =
            (unsigned long long)__double_as_longlong(*(volatile const double*)(Ap + i + (int64_t)j * ldap)) &
            0x7fffffffffffffffull;
        mx = a > mx ? a : mx;
    }
    Eblk[blk * m + i] = mx == 0 ? INT32_MIN : ot_exp_of_max(mx);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static int64_t ot_kp(int64_t K) { return ceil_div(K, OT_BK) * OT_BK; }
static int64_t ot_pad(int64_t v, int64_t b) { return ceil_div(v, b) * b; }

// Split point of [c0, c1): the left part is a multiple of OT_NB columns and
// at most OT_KMAX (the K of the update that follows).
static int64_t ot_mid(int64_t c0, int64_t c1) {
    int64_t w = c1 - c0;
    int64_t left = ceil_div(ceil_div(w, 2), OT_NB) * OT_NB;
    return c0 + std::min<int64_t>(left, OT_KMAX);
}

static bool ot_map(CUtensorMap* map, const void* base, int64_t Kp, int64_t rows, int box_rows);
static bool ot_map_f64(CUtensorMap* map, const double* base, int64_t rows, int64_t cols, int64_t ld);
static size_t ot_update_smem() { return 1024 + 2 * OT_DIG * OT_YTILE + OT_XST * OT_XTILE + 512; }

// Scratch of one update with M rows, N columns and inner dimension K.
size_t ot_update_ws_bytes(int64_t M, int64_t N, int64_t K) {
    const int64_t mp = ot_pad(M, OT_BM), Np = ot_pad(N, OT_BN), Kp = ot_kp(K);
    return align_up(sizeof(uint16_t) * OT_DIG * (size_t)mp * Kp, 256) + align_up(sizeof(int32_t) * mp, 256) +
           align_up(sizeof(uint16_t) * OT_DIG * (size_t)Np * Kp, 256) + align_up(sizeof(int32_t) * Np, 256) +
           align_up(sizeof(unsigned long long) * mp, 256) + align_up(sizeof(int32_t) * mp, 256) + 256;
}

// The negated Gaussian sketch operator's K chunk as the update's X digit
// planes: rows i < s of -Omega, columns j0 .. j0 + kc - 1 (global indices of
// Omega's columns), entries -q 2^-17 (csrc/gauss.cuh) sliced with the fixed
// row exponent E = 3 (|Omega| < 8): V = -q 2^35, so only digits 0..2 can be
// nonzero and only those planes are written.  Rows s <= i < mp and columns
// kc <= k < Kp are zero.  One warp per row and 64 columns (two per lane):
// each plane's row segment is one 128-byte store.
__global__ void __launch_bounds__(256) k_ot_gauss_digits(const ZigTable tab, uint64_t seed, int64_t s, int64_t j0,
                                                         int64_t kc, int64_t mp, int64_t Kp,
                                                         uint16_t* __restrict__ Z, int32_t* __restrict__ Ex) {
    __shared__ ZigShared Zs;
    zig_stage(tab, Zs);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t k = (int64_t)blockIdx.x * 64 + 2 * lane;
    for (int64_t i = (int64_t)blockIdx.y * 8 + warp; i < mp; i += (int64_t)gridDim.y * 8) {
        unsigned long long W[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int32_t q = (i < s && k + h < kc) ? gauss_q(seed, i, j0 + k + h, Zs) : 0;
            W[h] = (unsigned long long)(-(long long)q * (1ll << 35)) + OT_BIAS;
        }
#pragma unroll
        for (int t = 0; t < 3; ++t)
            *(uint32_t*)(Z + ((int64_t)t * mp + i) * Kp + k) = ot_digit_pair(W[0], W[1], t);
        if (blockIdx.x == 0 && lane == 0) Ex[i] = 3;
    }
}

// Pieces of an update's scratch: X digit planes and row exponents, then the Y
// digit planes and column exponents.
struct OtUpd {
    uint16_t* Zx;
    int32_t* Ex;
    uint16_t* Zy;
    int32_t* Ey;
    unsigned long long* Mx;  // row maxima of X (bit patterns), for the 2-D slicing
    int32_t* Eb;             // their exponents
    int64_t mp, Np, Kp;
};

static OtUpd ot_upd_ptrs(void* ws, int64_t M, int64_t N, int64_t K) {
    OtUpd U;
    U.mp = ot_pad(M, OT_BM);
    U.Np = ot_pad(N, OT_BN);
    U.Kp = ot_kp(K);
    char* base = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    U.Zx = (uint16_t*)base;
    base += align_up(sizeof(uint16_t) * OT_DIG * (size_t)U.mp * U.Kp, 256);
    U.Ex = (int32_t*)base;
    base += align_up(sizeof(int32_t) * U.mp, 256);
    U.Zy = (uint16_t*)base;
    base += align_up(sizeof(uint16_t) * OT_DIG * (size_t)U.Np * U.Kp, 256);
    U.Ey = (int32_t*)base;
    base += align_up(sizeof(int32_t) * U.Np, 256);
    U.Mx = (unsigned long long*)base;
    base += align_up(sizeof(unsigned long long) * U.mp, 256);
    U.Eb = (int32_t*)base;
    return U;
}

lsq_status ot_gauss_digits(uint64_t seed, int64_t s, int64_t j0, int64_t kc, int64_t N, void* ws, size_t ws_bytes,
                           cudaStream_t st) {
    if (s <= 0 || kc <= 0 || kc > OT_KMAX3 || !ws || ws_bytes < ot_update_ws_bytes(s, N, kc)) return LSQ_ERR_ARG;
    const OtUpd U = ot_upd_ptrs(ws, s, N, kc);
    const dim3 grid((unsigned)(U.Kp / 64), (unsigned)std::min<int64_t>(ceil_div(U.mp, 8), 256));
    k_ot_gauss_digits<<<grid, 256, 0, st>>>(zig_table(), seed, s, j0, kc, U.mp, U.Kp, U.Zx, U.Ex);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

// C_out = C_in - X Y (M x N; X: M x K column-major, ld ldx; Y: entry (k, j)
// at Y[k sk + j sj]) with FP64 accuracy on the tensor cores; K <= 512.
// C_in may equal C_out (same ld).  xmode: 0 slice X here; 1 slice X with the
// row exponents from the per-block exponents Eblk (blocks b0 .. b0+nbk-1).
lsq_status ot_gemm_update(const double* X, int64_t ldx, const double* Y, int64_t sk, int64_t sj, const double* Cin,
                          int64_t ldi, double* Cout, int64_t ldo, int64_t M, int64_t N, int64_t K, void* ws,
                          size_t ws_bytes, int32_t* err, cudaStream_t st, int xmode, const int32_t* Eblk, int64_t b0,
                          int nbk, int x_digits) {
    if (M <= 0 || N <= 0 || K <= 0) return LSQ_OK;
    // exact group sums: at most 8 pairs of digits (|d_t d_u| <= 2^12) per
    // group over K <= 512, or 3 pairs over K <= 1024 with three X digits
    if (K > (x_digits == 3 ? OT_KMAX3 : OT_KMAX) || !ws || ws_bytes < ot_update_ws_bytes(M, N, K) ||
        (x_digits != 3 && x_digits != OT_DIG))
        return LSQ_ERR_ARG;
    const OtUpd U = ot_upd_ptrs(ws, M, N, K);
    CUtensorMap tzs, txs;
    if (xmode == 2) {
        // X's digit planes and row exponents are already in the scratch
        // (ot_gauss_digits), three digits per value
        if (x_digits != 3) return LSQ_ERR_ARG;
    } else if (xmode == 1 && ot_map(&tzs, U.Zx, U.Kp, U.mp, OT_RS_ROWS)) {
        const dim3 rg((unsigned)(U.mp / OT_RS_ROWS), (unsigned)(U.Kp / 64));
        if (ldx % 2 == 0 && ((uintptr_t)X % 16) == 0 && ot_map_f64(&txs, X, M, K, ldx)) {
            const size_t rsm = 1024 + (size_t)OT_DIG * OT_RS_ROWS * 128 + (size_t)OT_RS_ROWS * 64 * 8;
            LSQ_CUDA_TRY(
                cudaFuncSetAttribute(k_ot_rowslice_s<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
            k_ot_rowslice_s<true, false><<<rg, 128, rsm, st>>>(tzs, txs, X, M, U.mp, K, ldx, U.Ex, Eblk, b0, nbk, err);
        } else {
            const size_t rsm = 1024 + (size_t)OT_DIG * OT_RS_ROWS * 128;
            LSQ_CUDA_TRY(
                cudaFuncSetAttribute(k_ot_rowslice_s<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
            k_ot_rowslice_s<false, false><<<rg, 128, rsm, st>>>(tzs, tzs, X, M, U.mp, K, ldx, U.Ex, Eblk, b0, nbk, err);
        }
    } else if (xmode == 0 && K <= 64 && ldx % 2 == 0 && ((uintptr_t)X % 16) == 0 &&
               ot_map(&tzs, U.Zx, U.Kp, U.mp, OT_RS_ROWS) && ot_map_f64(&txs, X, M, K, ldx)) {
        const size_t rsm = 1024 + (size_t)OT_DIG * OT_RS_ROWS * 128 + (size_t)OT_RS_ROWS * 64 * 8;
        LSQ_CUDA_TRY(cudaFuncSetAttribute(k_ot_rowslice_s<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)rsm));
        k_ot_rowslice_s<true, true><<<dim3((unsigned)(U.mp / OT_RS_ROWS), 1u), 128, rsm, st>>>(
            tzs, txs, X, M, U.mp, K, ldx, U.Ex, nullptr, 0, 0, err);
    } else if (xmode == 1) {
        k_ot_rowslice_e<<<dim3((unsigned)(U.mp / 128), (unsigned)(U.Kp / 64)), 128, 0, st>>>(
            X, M, U.mp, K, ldx, U.Kp, U.Ex, U.Zx, Eblk, b0, nbk);
    } else {
        // row maxima over a 2-D grid (rows x 64-wide K ranges), then the
        // slicing on the same grid: every SM has work even when M is small
        LSQ_CUDA_TRY(cudaMemsetAsync(U.Mx, 0, sizeof(unsigned long long) * (size_t)U.mp, st));
        const dim3 g2((unsigned)(U.mp / 128), (unsigned)(U.Kp / 64));
        k_ot_rowmax2d<<<g2, 128, 0, st>>>(X, M, K, ldx, U.Mx);
        LSQ_LAUNCH_CHECK();
        k_ot_rowexp<<<(unsigned)ceil_div(M, 256), 256, 0, st>>>(U.Mx, M, U.Eb);
        LSQ_LAUNCH_CHECK();
        k_ot_rowslice_e<<<g2, 128, 0, st>>>(X, M, U.mp, K, ldx, U.Kp, U.Ex, U.Zx, U.Eb, 0, 1);
    }
    LSQ_LAUNCH_CHECK();
    k_ot_colslice<<<(unsigned)U.Np, 128, 0, st>>>(Y, K, N, U.Np, sk, sj, U.Kp, U.Ey, U.Zy);
    LSQ_LAUNCH_CHECK();
    CUtensorMap tx, ty;
    if (!ot_map(&tx, U.Zx, U.Kp, U.mp, OT_BM) || !ot_map(&ty, U.Zy, U.Kp, U.Np, OT_BN)) return LSQ_ERR_CUDA;
    const size_t smem = ot_update_smem();
    auto kern = x_digits == 3 ? k_ot_update<3> : k_ot_update<OT_DIG>;
    LSQ_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int ntj = (int)(U.Np / OT_BN), ntiles = (int)(ntj * (U.mp / OT_BM));
    const int grid = std::min(ntiles, device_sm_count());
    const int stage = x_digits == 3 ? ST_K_UPDATE3 : ST_K_UPDATE;
    stage_mark(stage, true, st);
    kern<<<grid, OT_THREADS, smem, st>>>(tx, ty, M, N, K, U.Ex, U.Ey, Cin, ldi, Cout, ldo, err, ntj, ntiles);
    LSQ_LAUNCH_CHECK();
    // tensor-core work: the digit pairs actually issued
    const double pairs = x_digits == 3 ? 21.0 : 36.0;
    stage_mark(stage, false, st, pairs * 2.0 * (double)M * (double)N * (double)K);
    return LSQ_OK;
}

static void ot_max_update(int64_t m, int64_t c0, int64_t c1, size_t& need) {
    if (c1 - c0 <= OT_NB) return;
    int64_t mid = ot_mid(c0, c1);
    need = std::max(need, ot_update_ws_bytes(m, c1 - mid, mid - c0));
    ot_max_update(m, c0, mid, need);
    ot_max_update(m, mid, c1, need);
}

// Update scratch, then the per-block row exponents (m x ceil(n / OT_NB) int32).
static size_t ot_eblk_offset(int64_t m, int64_t n) {
    size_t need = 256;
    ot_max_update(m, 0, n, need);
    return align_up(need, 256);
}

size_t ot_trsm_ws_bytes(int64_t m, int64_t n) {
    return ot_eblk_offset(m, n) + align_up(sizeof(int32_t) * (size_t)m * ceil_div(n, OT_NB), 256) + 512;
}

// Digit planes as a 3-D tensor (k, row, digit); Kp and rows are multiples of
// the box, so no box reaches outside.
static bool ot_map(CUtensorMap* map, const void* base, int64_t Kp, int64_t rows, int box_rows) {
    EncodeTiledFn enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)OT_DIG};
    cuuint64_t strides[2] = {(cuuint64_t)(Kp * 2), (cuuint64_t)(rows * Kp * 2)};
    cuuint32_t box[3] = {(cuuint32_t)OT_BK, (cuuint32_t)box_rows, 1u};
    cuuint32_t estr[3] = {1u, 1u, 1u};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// FP64 column-major rows x cols (leading dimension ld, even; base 16-byte
// aligned): boxes of 64 rows x 64 columns, no swizzle, zero fill outside.
static bool ot_map_f64(CUtensorMap* map, const double* base, int64_t rows, int64_t cols, int64_t ld) {
    EncodeTiledFn enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 8)};
    cuuint32_t box[2] = {(cuuint32_t)OT_RS_ROWS, 64u};
    cuuint32_t estr[2] = {1u, 1u};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct OtCtx {
    int64_t m;
    const double* R;
    int64_t ldr;
    double* Ap;
    int64_t ldap;
    void* ws;
    size_t ws_bytes;
    int32_t* Eblk;
    int32_t* err;
    cudaStream_t st;
};

// Columns [c0, c1) of the right-hand side are in src (ld lds); results in Ap.
static lsq_status ot_solve(const OtCtx& C, int64_t c0, int64_t c1, const double* src, int64_t lds) {
    if (c1 - c0 <= OT_NB) {
        // 64-thread CTAs: 1024 of them over 152 SMs puts at most 7 on an SM
        // against an average of 6.7 (128-thread CTAs: 4 against 3.4)
        k_ot_diag<OT_NB><<<(unsigned)ceil_div(C.m, 64), 64, 0, C.st>>>(src + c0 * lds, lds, C.R + c0 + c0 * C.ldr,
                                                                       C.ldr, (int)(c1 - c0), C.m,
                                                                       C.Ap + c0 * C.ldap, C.ldap, C.Eblk,
                                                                       c0 / OT_NB);
        LSQ_LAUNCH_CHECK();
        return LSQ_OK;
    }
    const int64_t mid = ot_mid(c0, c1);
    lsq_status r = ot_solve(C, c0, mid, src, lds);
    if (r != LSQ_OK) return r;
    r = ot_gemm_update(C.Ap + c0 * C.ldap, C.ldap, C.R + c0 + mid * C.ldr, 1, C.ldr, src + mid * lds, lds,
                       C.Ap + mid * C.ldap, C.ldap, C.m, c1 - mid, mid - c0, C.ws, C.ws_bytes, C.err, C.st, 1,
                       C.Eblk, c0 / OT_NB, (int)((mid - c0) / OT_NB));
    if (r != LSQ_OK) return r;
    return ot_solve(C, mid, c1, C.Ap, C.ldap);
}

bool ot_trsm_supported() { return tensor_map_encoder() != nullptr; }

lsq_status ot_trsm(const double* A, int64_t m, int64_t n, int64_t lda, const double* R, int64_t ldr, double* Ap,
                   int64_t ldap, void* ws, size_t ws_bytes, int32_t* err, cudaStream_t st) {
    if (!A || !R || !Ap || m <= 0 || n <= 0 || lda < m || ldap < m || ldr < n) return LSQ_ERR_ARG;
    if (!ot_trsm_supported()) return LSQ_ERR_ARG;
    if (!ws || ws_bytes < ot_trsm_ws_bytes(m, n)) return LSQ_ERR_NOMEM;
    char* base = (char*)ws;
    OtCtx C{m, R, ldr, Ap, ldap, ws, ws_bytes, (int32_t*)(base + ot_eblk_offset(m, n) + 256), err, st};
    return ot_solve(C, 0, n, A, lda);
}

}  // namespace lsq
