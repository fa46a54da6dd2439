// FP64 Gram matrix G = X^T X (and the product X^T Y of two m x n matrices)
// on the FP8 tensor cores, exact to a 56-bit
// fixed-point representation of every column (digit slicing in the manner
// of Ozaki, Ogita & Oishi's error-free matrix multiplication):
//
//   x_ip = 2^(e_p) * sum_{t=0}^{S-1} d_t(i,p) 16^-(t+1) + r_ip,
//          d_t in [-15, 15], |r_ip| < 2^(e_p - 56)   (S = 14 digits),
//
// where 2^(e_p) bounds column p.  Digit products are integers below 2^8, so
// a K-chunk of up to 65536 rows sums exactly in the FP32 accumulators of
// tcgen05.mma (kind::f8f6f4, E4M3 operands).  Every digit-pair block (t, u)
// with t + u <= S - 1 is one tensor-core contraction over the rows; the
// blocks are combined in FP64 in a fixed order (smallest weight first) and
// scaled by 2^(e_p + e_q).  Dropped pairs and the residuals r contribute
// below 2^-55 of |x_p| |x_q| per row, the same order as FP64 rounding.
//
// Digits are extracted with integer operations on the FP64 bit pattern (no
// FP64 instruction in the slicing pass).
#include "common.cuh"
#include "kernels.cuh"

#include <algorithm>

namespace lsq {

constexpr int OZ_S = 14;        // digits per value (4 bits each: 56 bits)
constexpr int64_t OZ_KCHUNK = 65536;  // rows summed exactly per FP32 accumulator

lsq_status launch_tc_tiles_fp8(const void* X, int64_t ldx, int64_t rowsX, const void* Y, int64_t ldy, int64_t rowsY,
                               int64_t K, int64_t kchunk, const int2* tiles, int64_t ntiles, float* out, int32_t* err,
                               cudaStream_t st);

// e_p: exponent with max_i |x_ip| < 2^(e_p) (frexp exponent of the column max),
// from the bit patterns (integer max, no FP64 instruction).
__global__ void k_oz_colexp(const double* __restrict__ X, int64_t m, int64_t ld, int32_t* __restrict__ e) {
    int64_t p = blockIdx.x;
    const unsigned long long* col = (const unsigned long long*)(X + p * ld);
    unsigned long long mx = 0;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
        unsigned long long v = col[i] & 0x7fffffffffffffffull;
        mx = v > mx ? v : mx;
    }
    for (int off = 16; off > 0; off >>= 1) {
        unsigned long long o = __shfl_xor_sync(0xffffffffu, mx, off);
        mx = o > mx ? o : mx;
    }
    __shared__ unsigned long long w[32];
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t = w[q] > t ? w[q] : t;
        int Eb = (int)((t >> 52) & 0x7ff);
        e[p] = (t == 0 || Eb == 0) ? 0 : Eb - 1022;
    }
}

__device__ __forceinline__ uint8_t e4m3_of_digit(int d) {
    // exact E4M3 encoding of an integer in [-15, 15]
    uint32_t a = (uint32_t)(d < 0 ? -d : d);
    if (a == 0) return 0;
    int E = 31 - __clz(a);                       // 0..3
    uint32_t mant = (a - (1u << E)) << (3 - E);  // 3 bits
    return (uint8_t)(((d < 0) ? 0x80u : 0u) | ((uint32_t)(E + 7) << 3) | mant);
}

// Z row (t * np + p), column i  <-  digit t of x_ip.  Rows p >= n and
// columns i >= m (padding) are zero.
__global__ void k_oz_slice(const double* __restrict__ X, int64_t m, int64_t n, int64_t ld,
                           const int32_t* __restrict__ e, int64_t np, int64_t ldz, uint8_t* __restrict__ Z) {
    int64_t p = blockIdx.y;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ldz; i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long V = 0;
        bool neg = false;
        if (p < n && i < m) {
            unsigned long long b = (unsigned long long)__double_as_longlong(X[i + p * ld]);
            neg = (b >> 63) != 0;
            int Eb = (int)((b >> 52) & 0x7ff);
            if (Eb != 0 && Eb != 0x7ff) {
                unsigned long long sig = (b & 0x000fffffffffffffull) | 0x0010000000000000ull;
                int sh = (Eb - 1023) - e[p] + 4;  // x 2^(56 - e_p) = sig 2^(E_a - 52 + 56 - e_p)
                if (sh >= 0) V = sig << sh;       // sh <= 3: V < 2^56
                else if (sh > -64) V = sig >> (-sh);
            }
        }
#pragma unroll
        for (int t = 0; t < OZ_S; ++t) {
            int d = (int)((V >> (4 * (OZ_S - 1 - t))) & 15ull);
            Z[((int64_t)t * np + p) * ldz + i] = e4m3_of_digit(neg ? -d : d);
        }
    }
}

// G[p, q] from the digit-pair tiles.  pair_tile[(t * S + u) * nb * nb + P * nb
// + Q] = index of the tile holding C_tu[P block, Q block], or -1 (symmetric
// case: then C_tu = C_ut^T is read from the (u, t) tile at (Q, P)).  sym:
// only p >= q is formed and mirrored; ex / ey: column exponents of X / Y.
__global__ void k_oz_combine(const float* __restrict__ T, const int32_t* __restrict__ pair_tile, int64_t ntiles,
                             int chunks, int64_t n, int64_t nb, const int32_t* __restrict__ ex,
                             const int32_t* __restrict__ ey, int sym, double* __restrict__ G, int64_t ldg) {
    int64_t total = n * n;
    for (int64_t q2 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q2 < total; q2 += (int64_t)gridDim.x * blockDim.x) {
        int64_t p = q2 % n, q = q2 / n;
        if (sym && p < q) continue;
        int64_t P = p >> 7, Q = q >> 7, r = p & 127, c = q & 127;
        double acc = 0.0;
        for (int d = 2 * OZ_S - 2; d >= 0; --d) {  // weight 16^-(d+2), smallest first
            if (d > OZ_S - 1) continue;               // dropped: t + u > S - 1
            double w = ldexp(1.0, -4 * (d + 2));
            for (int t = 0; t <= d; ++t) {
                int u = d - t;
                int32_t id = pair_tile[((int64_t)(t * OZ_S + u) * nb + P) * nb + Q];
                int64_t off;
                if (id >= 0) {
                    off = (int64_t)id * 16384 + r + c * 128;
                } else {
                    id = pair_tile[((int64_t)(u * OZ_S + t) * nb + Q) * nb + P];
                    off = (int64_t)id * 16384 + c + r * 128;
                }
                for (int z = 0; z < chunks; ++z) acc = fma(w, (double)T[(int64_t)z * ntiles * 16384 + off], acc);
            }
        }
        double g = ldexp(acc, ex[p] + ey[q]);
        G[p + q * ldg] = g;
        if (sym) G[q + p * ldg] = g;
    }
}

struct OzPlan {
    int64_t np, nb, ldz, ntiles, kchunk;
    int chunks;
    size_t z_bytes, t_bytes, tiles_bytes, map_bytes, e_bytes, total;
};

static OzPlan oz_plan(int64_t m, int64_t n, bool sym) {
    OzPlan P;
    P.np = ceil_div(n, 128) * 128;
    P.nb = P.np / 128;
    P.ldz = ceil_div(m, 128) * 128;
    P.kchunk = std::min<int64_t>(OZ_KCHUNK, P.ldz);
    P.chunks = (int)ceil_div(P.ldz, P.kchunk);
    // symmetric: pairs t <= u with t + u <= S-1, blocks P >= Q for t == u, all
    // (P, Q) for t < u; otherwise every pair with t + u <= S-1 and every block
    int64_t nt = 0;
    for (int t = 0; t < OZ_S; ++t)
        for (int u = sym ? t : 0; u < OZ_S; ++u)
            if (t + u <= OZ_S - 1) nt += (sym && t == u) ? P.nb * (P.nb + 1) / 2 : P.nb * P.nb;
    P.ntiles = nt;
    P.z_bytes = align_up((size_t)OZ_S * P.np * P.ldz, 256) * (sym ? 1 : 2);
    P.t_bytes = align_up(sizeof(float) * 16384 * (size_t)nt * P.chunks, 256);
    P.tiles_bytes = align_up(sizeof(int2) * (size_t)nt, 256);
    P.map_bytes = align_up(sizeof(int32_t) * (size_t)OZ_S * OZ_S * P.nb * P.nb, 256);
    P.e_bytes = align_up(sizeof(int32_t) * (size_t)n, 256) * (sym ? 1 : 2);
    P.total = P.z_bytes + P.t_bytes + P.tiles_bytes + P.map_bytes + P.e_bytes + 1024;
    return P;
}

size_t oz_gram_ws_bytes(int64_t m, int64_t n) { return oz_plan(m, n, true).total; }
size_t oz_gemm_tn_ws_bytes(int64_t m, int64_t n) { return oz_plan(m, n, false).total; }

// Tile list (grouped so that neighbouring CTAs share the Y-row block of a
// pair) and the (t, u, P, Q) -> tile map, built on the device by one thread in
// a fixed order (no host copies: the call stays capturable in a CUDA graph).
__global__ void k_oz_tiles(int64_t nb, int64_t np, int sym, int2* __restrict__ tiles, int32_t* __restrict__ map) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (int64_t q = 0; q < (int64_t)OZ_S * OZ_S * nb * nb; ++q) map[q] = -1;
    int32_t k = 0;
    for (int u = 0; u < OZ_S; ++u)
        for (int64_t Q = 0; Q < nb; ++Q)
            for (int t = 0; t < OZ_S; ++t) {
                if (t + u > OZ_S - 1 || (sym && t > u)) continue;
                for (int64_t Pb = 0; Pb < nb; ++Pb) {
                    if (sym && t == u && Pb < Q) continue;
                    map[((int64_t)(t * OZ_S + u) * nb + Pb) * nb + Q] = k;
                    tiles[k] = make_int2((int)(t * np + Pb * 128), (int)(u * np + Q * 128));
                    ++k;
                }
            }
}

// G = X^T Y (n x n) from the digit planes of X and Y (the same planes when
// Y is X, which is the symmetric case).
static lsq_status oz_run(const double* X, int64_t ldx, const double* Y, int64_t ldy, bool sym, int64_t m, int64_t n,
                         double* G, int64_t ldg, void* ws, size_t ws_bytes, int32_t* err, cudaStream_t st) {
    OzPlan P = oz_plan(m, n, sym);
    if (!ws || ws_bytes < P.total) return LSQ_ERR_NOMEM;
    if (OZ_S * P.np > 0x7fffffff || P.ldz > 0x7fffffff) return LSQ_ERR_ARG;
    char* base = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    const size_t zb = P.z_bytes / (sym ? 1 : 2), eb = P.e_bytes / (sym ? 1 : 2);
    uint8_t* Zx = (uint8_t*)base;
    uint8_t* Zy = sym ? Zx : Zx + zb;
    float* T = (float*)(base + P.z_bytes);
    int2* tiles = (int2*)(base + P.z_bytes + P.t_bytes);
    int32_t* map = (int32_t*)(base + P.z_bytes + P.t_bytes + P.tiles_bytes);
    int32_t* ex = (int32_t*)(base + P.z_bytes + P.t_bytes + P.tiles_bytes + P.map_bytes);
    int32_t* ey = sym ? ex : (int32_t*)((char*)ex + eb);
    k_oz_tiles<<<1, 1, 0, st>>>(P.nb, P.np, sym ? 1 : 0, tiles, map);
    LSQ_LAUNCH_CHECK();
    dim3 gs((unsigned)std::min<int64_t>(ceil_div(P.ldz, 256), 64), (unsigned)P.np);
    k_oz_colexp<<<(unsigned)n, 256, 0, st>>>(X, m, ldx, ex);
    LSQ_LAUNCH_CHECK();
    k_oz_slice<<<gs, 256, 0, st>>>(X, m, n, ldx, ex, P.np, P.ldz, Zx);
    LSQ_LAUNCH_CHECK();
    if (!sym) {
        k_oz_colexp<<<(unsigned)n, 256, 0, st>>>(Y, m, ldy, ey);
        LSQ_LAUNCH_CHECK();
        k_oz_slice<<<gs, 256, 0, st>>>(Y, m, n, ldy, ey, P.np, P.ldz, Zy);
        LSQ_LAUNCH_CHECK();
    }
    lsq_status r = launch_tc_tiles_fp8(Zx, P.ldz, OZ_S * P.np, Zy, P.ldz, OZ_S * P.np, P.ldz, P.kchunk, tiles,
                                       P.ntiles, T, err, st);
    if (r != LSQ_OK) return r;
    k_oz_combine<<<(unsigned)std::min<int64_t>(ceil_div(n * n, 256), 16384), 256, 0, st>>>(
        T, map, P.ntiles, P.chunks, n, P.nb, ex, ey, sym ? 1 : 0, G, ldg);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

lsq_status oz_gram(const double* X, int64_t m, int64_t n, int64_t ld, double* G, int64_t ldg, void* ws,
                   size_t ws_bytes, int32_t* err, cudaStream_t st) {
    return oz_run(X, ld, X, ld, true, m, n, G, ldg, ws, ws_bytes, err, st);
}

lsq_status oz_gemm_tn(const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t m, int64_t n, double* G,
                      int64_t ldg, void* ws, size_t ws_bytes, int32_t* err, cudaStream_t st) {
    return oz_run(X, ldx, Y, ldy, false, m, n, G, ldg, ws, ws_bytes, err, st);
}

}  // namespace lsq
