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
// blocks are combined exactly in integers, scaled by 2^(e_p + e_q) and
// rounded once.  Dropped pairs and the residuals r contribute below 2^-55 of
// |x_p| |x_q| per row, the same order as FP64 rounding.
//
// Digits are extracted with integer operations on the FP64 bit pattern (no
// FP64 instruction in the slicing pass).
#include "common.cuh"
#include "kernels.cuh"

#include <algorithm>

namespace lsq {

constexpr int OZ_S = 14;        // digits per value (4 bits each: 56 bits)
constexpr int64_t OZ_KCHUNK = 65536;  // rows summed exactly per FP32 accumulator
constexpr int32_t OZ_NONFINITE = INT32_MAX;  // column exponent of a column holding an Inf or NaN

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
        e[p] = Eb == 0x7ff ? OZ_NONFINITE : (t == 0 || Eb == 0) ? 0 : Eb - 1022;
    }
}

// Two FP32 values to E4M3 (the first in the upper byte); exact for the
// integer digits in [-15, 15].
__device__ __forceinline__ uint32_t e4m3x2(float hi, float lo) {
    unsigned short r;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(hi), "f"(lo));
    return r;
}

// Z row (t * np + p), column i  <-  digit t of x_ip.  Rows p >= n and
// columns i >= m (padding) are zero.  4 consecutive rows per thread: a warp
// reads 1 KB of a column and writes 128 contiguous bytes of every digit
// plane.  Digit t of |x| is a nibble of V = |x| 2^(56 - e_p); its signed FP32
// value is s (2^23 1.5 + nibble) - s 2^23 1.5 (s = +-1; exact, and +0 for a
// zero nibble), converted in pairs by the hardware.
__global__ void __launch_bounds__(256) k_oz_slice(const double* __restrict__ X, int64_t m, int64_t n, int64_t ld,
                                                  const int32_t* __restrict__ e, int64_t np, int64_t ldz,
                                                  uint8_t* __restrict__ Z) {
    const int64_t p = blockIdx.y;
    const int32_t ep = p < n ? e[p] : 0;
    const double* col = X + p * ld;
    for (int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4; i0 < ldz;
         i0 += (int64_t)gridDim.x * blockDim.x * 4) {
        unsigned long long V[4];
        float sg[4], off[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const unsigned long long b =
                (p < n && i0 + q < m) ? (unsigned long long)__double_as_longlong(col[i0 + q]) : 0ull;
            const int Eb = (int)((b >> 52) & 0x7ff);
            V[q] = 0;
            if (Eb != 0 && Eb != 0x7ff && ep != OZ_NONFINITE) {
                const unsigned long long sig = (b & 0x000fffffffffffffull) | 0x0010000000000000ull;
                const int sh = (Eb - 1023) - ep + 4;  // x 2^(56 - e_p) = sig 2^(E_a - 52 + 56 - e_p)
                if (sh >= 0) V[q] = sig << sh;        // sh <= 3: V < 2^56
                else if (sh > -64) V[q] = sig >> (-sh);
            }
            sg[q] = (b >> 63) ? -1.0f : 1.0f;
            off[q] = -sg[q] * 12582912.0f;
        }
#pragma unroll
        for (int t = 0; t < OZ_S; ++t) {
            float d[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t nib = (uint32_t)(V[q] >> (4 * (OZ_S - 1 - t))) & 15u;
                d[q] = fmaf(sg[q], __uint_as_float(0x4B400000u | nib), off[q]);
            }
            *(uint32_t*)(Z + ((int64_t)t * np + p) * ldz + i0) = e4m3x2(d[1], d[0]) | (e4m3x2(d[3], d[2]) << 16);
        }
    }
}

// G[p, q] from the digit-pair tiles.  pair_tile[(t * S + u) * nb * nb + P * nb
// + Q] = index of the tile holding C_tu[P block, Q block], or -1 (symmetric
// case: then C_tu = C_ut^T is read from the (u, t) tile at (Q, P)).  Tiles are
// 128 x 128 FP32, column-major; chunk z of tile id starts at (z ntiles + id)
// 16384.  Every tile value is an integer below 2^24 in magnitude, so each
// weight class d = t + u sums exactly in 64-bit integers,
//   S_d = sum_{t + u = d} sum_z C_tu,z[p, q],
// and I = sum_{d=0}^{S-1} S_d 16^(S-1-d) (Horner, 128-bit) is the exact
// digit-sliced sum: G[p, q] = I 2^(e_p + e_q - 4 (S + 1)), rounded once.
// One CTA per (P, Q) block (P >= Q when sym) and 32-column quarter; thread
// (r = tid mod 128, c = c0 + tid / 128 + 2k, k < 16) owns 16 entries.  Tiles
// read transposed are staged through shared memory; the loads of the next
// tile are issued before the current one is summed.  sym: only p >= q is
// formed and mirrored; ex / ey: column exponents of X / Y (OZ_NONFINITE
// marks a column holding an Inf or NaN: its entries are NaN).
constexpr int OZ_CB_THREADS = 256;

__device__ __forceinline__ int64_t oz_item_base(const int32_t* __restrict__ pair_tile, int64_t ntiles, int64_t nb,
                                                int64_t P, int64_t Q, int d, int t, int z, bool& tr) {
    const int u = d - t;
    int32_t id = pair_tile[((int64_t)(t * OZ_S + u) * nb + P) * nb + Q];
    tr = false;
    if (id < 0) {
        id = pair_tile[((int64_t)(u * OZ_S + t) * nb + Q) * nb + P];
        tr = true;
    }
    return id < 0 ? -1 : ((int64_t)z * ntiles + id) * 16384;
}

__device__ __forceinline__ void oz_item_load(const float* __restrict__ T, int64_t base, bool tr, int r, int cb,
                                             int c0, float (&v)[16]) {
    if (base < 0) {
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = 0.f;
    } else if (!tr) {
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = T[base + r + (int64_t)(cb + 2 * k) * 128];
    } else {
        // rows r' of the stored (u, t) tile hold our columns c0 .. c0 + 31 at r' 128 + c
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int f = threadIdx.x + OZ_CB_THREADS * j;
            const float4 w = *(const float4*)(T + base + (int64_t)(f >> 3) * 128 + c0 + (f & 7) * 4);
            v[4 * j] = w.x;
            v[4 * j + 1] = w.y;
            v[4 * j + 2] = w.z;
            v[4 * j + 3] = w.w;
        }
    }
}

__global__ void __launch_bounds__(OZ_CB_THREADS) k_oz_combine(const float* __restrict__ T,
                                                              const int32_t* __restrict__ pair_tile, int64_t ntiles,
                                                              int chunks, int64_t n, int64_t nb,
                                                              const int32_t* __restrict__ ex,
                                                              const int32_t* __restrict__ ey, int sym,
                                                              double* __restrict__ G, int64_t ldg) {
    __shared__ float tr_s[128][33];
    const int c0 = (int)(blockIdx.x & 3) * 32;
    const int64_t blk = blockIdx.x >> 2;
    int64_t P, Q;
    if (sym) {
        P = 0;
        while ((P + 1) * (P + 2) / 2 <= blk) ++P;
        Q = blk - P * (P + 1) / 2;
    } else {
        P = blk % nb;
        Q = blk / nb;
    }
    const int r = threadIdx.x & 127;
    const int cb = c0 + (threadIdx.x >> 7);
    long long H[16], S[16];
    unsigned long long L[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) H[k] = 0, L[k] = 0, S[k] = 0;
    int d = 0, t = 0, z = 0;
    bool tr;
    int64_t base = oz_item_base(pair_tile, ntiles, nb, P, Q, d, t, z, tr);
    float cur[16];
    oz_item_load(T, base, tr, r, cb, c0, cur);
    for (;;) {
        // next item in the order d, t, z
        int dn = d, tn = t, zn = z + 1;
        if (zn == chunks) zn = 0, ++tn;
        if (tn > dn) tn = 0, ++dn;
        const bool more = dn < OZ_S;
        bool trn = false;
        float nxt[16];
        if (more) {
            const int64_t bn = oz_item_base(pair_tile, ntiles, nb, P, Q, dn, tn, zn, trn);
            oz_item_load(T, bn, trn, r, cb, c0, nxt);
        }
        if (!tr) {
#pragma unroll
            for (int k = 0; k < 16; ++k) S[k] += (long long)__float2int_rz(cur[k]);
        } else {
            __syncthreads();  // the previous transposed tile has been read
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int f = threadIdx.x + OZ_CB_THREADS * j;
#pragma unroll
                for (int e = 0; e < 4; ++e) tr_s[f >> 3][(f & 7) * 4 + e] = cur[4 * j + e];
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < 16; ++k) S[k] += (long long)__float2int_rz(tr_s[r][cb - c0 + 2 * k]);
        }
        if (dn != d || !more) {
            // weight class d complete: I = 16 I + S_d
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                H[k] = (long long)(((unsigned long long)H[k] << 4) | (L[k] >> 60));
                L[k] <<= 4;
                const unsigned long long l2 = L[k] + (unsigned long long)S[k];
                H[k] += (S[k] >> 63) + (l2 < L[k] ? 1 : 0);
                L[k] = l2;
                S[k] = 0;
            }
        }
        if (!more) break;
        d = dn, t = tn, z = zn, tr = trn;
#pragma unroll
        for (int k = 0; k < 16; ++k) cur[k] = nxt[k];
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int64_t p = P * 128 + r, q = Q * 128 + cb + 2 * k;
        if (p >= n || q >= n || (sym && p < q)) continue;
        const int32_t a = ex[p], b = ey[q];
        const double g = (a == OZ_NONFINITE || b == OZ_NONFINITE) ? __longlong_as_double(0x7ff8000000000000ll)
                                                                  : fixed128_to_double(H[k], L[k], a + b - 4 * (OZ_S + 1));
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
    // tiles of 128 x 256: an X block P against the Y blocks 2 Qp and 2 Qp + 1.
    // Symmetric: pairs t <= u with t + u <= S-1, all (P, Qp) for t < u and
    // those with 2 Qp <= P for t == u; otherwise every pair with t + u <= S-1
    // and every (P, Qp).  ntiles counts 128-column halves (2 per tile).
    const int64_t nq = ceil_div(P.nb, 2);
    int64_t nt = 0;
    for (int t = 0; t < OZ_S; ++t)
        for (int u = sym ? t : 0; u < OZ_S; ++u) {
            if (t + u > OZ_S - 1) continue;
            if (sym && t == u)
                for (int64_t Pb = 0; Pb < P.nb; ++Pb) nt += Pb / 2 + 1;
            else
                nt += P.nb * nq;
        }
    P.ntiles = 2 * nt;
    P.z_bytes = align_up((size_t)OZ_S * P.np * P.ldz, 256) * (sym ? 1 : 2);
    P.t_bytes = align_up(sizeof(float) * 16384 * (size_t)P.ntiles * P.chunks, 256);
    P.tiles_bytes = align_up(sizeof(int2) * (size_t)nt, 256);
    P.map_bytes = align_up(sizeof(int32_t) * (size_t)OZ_S * OZ_S * P.nb * P.nb, 256);
    P.e_bytes = align_up(sizeof(int32_t) * (size_t)n, 256) * (sym ? 1 : 2);
    P.total = P.z_bytes + P.t_bytes + P.tiles_bytes + P.map_bytes + P.e_bytes + 1024;
    return P;
}

size_t oz_gram_ws_bytes(int64_t m, int64_t n) { return oz_plan(m, n, true).total; }
size_t oz_gemm_tn_ws_bytes(int64_t m, int64_t n) { return oz_plan(m, n, false).total; }

// Tile list and the (t, u, P, Q) -> half-tile map (2 k + (Q & 1) for tile
// k, i.e. the 128 x 128 block at (2 k + (Q & 1)) 16384 of the output), built
// on the device in a fixed order (no host copies: the call stays capturable
// in a CUDA graph).  A tile pairs X tile (t, P) (digit t, 128 rows) with Y
// tile (u, Qp) (digit u, 256 rows).  The X tiles are taken in groups of
// OZ_GX; inside a group the Y tiles run outer and the group's X tiles inner,
// so that a wave of 152 CTAs spans about OZ_GX X tiles and 152 / OZ_GX Y
// tiles and both are shared through L2 while the wave moves along K (with
// the Y tiles outer over all X tiles a wave read ~152 distinct X tiles).  One
// CTA: each group's tiles are counted by one thread, prefix summed in group
// order, and each group's range is filled by its thread.
constexpr int OZ_GX = 16;

__device__ __forceinline__ bool oz_tile_valid(int t, int64_t P, int u, int64_t Qp, int sym) {
    if (t + u > OZ_S - 1 || (sym && t > u)) return false;
    return !(sym && t == u && P < 2 * Qp);  // P >= 2 Qp when t == u
}

__global__ void k_oz_tiles(int64_t nb, int64_t np, int sym, int2* __restrict__ tiles, int32_t* __restrict__ map) {
    extern __shared__ int32_t oz_cnt[];  // groups + 1
    const int64_t nq = (nb + 1) / 2;
    const int64_t nx = (int64_t)OZ_S * nb, ny = (int64_t)OZ_S * nq;
    const int64_t groups = (nx + OZ_GX - 1) / OZ_GX;
    for (int64_t q = threadIdx.x; q < (int64_t)OZ_S * OZ_S * nb * nb; q += blockDim.x) map[q] = -1;
    for (int64_t g = threadIdx.x; g < groups; g += blockDim.x) {
        int32_t c = 0;
        const int64_t x1 = min(nx, (g + 1) * OZ_GX);
        for (int64_t yj = 0; yj < ny; ++yj)
            for (int64_t xi = g * OZ_GX; xi < x1; ++xi)
                c += oz_tile_valid((int)(xi / nb), xi % nb, (int)(yj / nq), yj % nq, sym) ? 1 : 0;
        oz_cnt[g + 1] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        oz_cnt[0] = 0;
        for (int64_t g = 0; g < groups; ++g) oz_cnt[g + 1] += oz_cnt[g];
    }
    __syncthreads();
    for (int64_t g = threadIdx.x; g < groups; g += blockDim.x) {
        int32_t k = oz_cnt[g];
        const int64_t x1 = min(nx, (g + 1) * OZ_GX);
        for (int64_t yj = 0; yj < ny; ++yj) {
            const int u = (int)(yj / nq);
            const int64_t Qp = yj % nq;
            for (int64_t xi = g * OZ_GX; xi < x1; ++xi) {
                const int t = (int)(xi / nb);
                const int64_t Pb = xi % nb;
                if (!oz_tile_valid(t, Pb, u, Qp, sym)) continue;
                for (int h = 0; h < 2; ++h) {
                    const int64_t Q = 2 * Qp + h;
                    if (Q < nb && !(sym && t == u && Q > Pb))
                        map[((int64_t)(t * OZ_S + u) * nb + Pb) * nb + Q] = 2 * k + h;
                }
                tiles[k] = make_int2((int)(t * np + Pb * 128), (int)(u * np + 2 * Qp * 128));
                ++k;
            }
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
    const size_t tsm = sizeof(int32_t) * (size_t)(ceil_div((int64_t)OZ_S * P.nb, OZ_GX) + 1);
    if (tsm > 48 * 1024) return LSQ_ERR_ARG;
    k_oz_tiles<<<1, 256, tsm, st>>>(P.nb, P.np, sym ? 1 : 0, tiles, map);
    LSQ_LAUNCH_CHECK();
    dim3 gs((unsigned)std::min<int64_t>(ceil_div(P.ldz, 256 * 4), 64), (unsigned)P.np);
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
                                       P.ntiles / 2, T, err, st);
    if (r != LSQ_OK) return r;
    const int64_t cblocks = (sym ? P.nb * (P.nb + 1) / 2 : P.nb * P.nb) * 4;
    k_oz_combine<<<(unsigned)cblocks, OZ_CB_THREADS, 0, st>>>(
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
