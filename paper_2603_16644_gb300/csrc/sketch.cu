// Sketch step of Alg. 1 ("Sketch A_s = Omega A" in precision u_p):
//   - sparse-sign operator generation (Philox4x32-10 + Lemire rejection),
//   - deterministic CSR transpose of Omega (rows of Omega in ascending j),
//   - per-column power-of-two scaling and rounding of A to u_p,
//   - sparse-sign gather A_s[i,:] = sum_j Omega_ij Ahat[j,:] (FP32 or FP64
//     accumulation in ascending j: bit-identical to a sequential sum),
//   - Gaussian operator generation (ziggurat in FP64, rounded to u_p).
// The Gaussian product itself is a dense contraction (gemm.cu / sketch_tc.cu).
#include "common.cuh"
#include "gauss.cuh"
#include "kernels.cuh"

#include <algorithm>
#include <cmath>
#include <type_traits>

namespace lsq {

// ---------------------------------------------------------------------------
// Sparse-sign operator: one thread per column j of Omega.
// ---------------------------------------------------------------------------
__global__ void k_sparse_gen(uint64_t seed, int64_t m, uint32_t s, int zeta, int32_t* __restrict__ idx,
                             int8_t* __restrict__ sgn, int32_t* __restrict__ err, int64_t j0) {
    const int64_t jl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (jl >= m) return;
    const int64_t j = j0 + jl;  // global column of Omega (row of the unsharded A)
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    uint32_t thresh = (0u - s) % s;
    int32_t got_idx[32];
    int got = 0;
    for (uint32_t blk = 0; got < zeta; ++blk) {
        if (blk > (1u << 20)) { set_info_once(err, -2); return; }
        U4 w = philox(U4{blk, (uint32_t)j, (uint32_t)((uint64_t)j >> 32), 0u}, k0, k1);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if (got >= zeta) break;
            uint64_t prod = (uint64_t)word_of(w, t) * (uint64_t)s;
            if ((uint32_t)prod < thresh) continue;
            int32_t cand = (int32_t)(prod >> 32);
            bool dup = false;
            for (int q = 0; q < got; ++q) dup |= (got_idx[q] == cand);
            if (!dup) got_idx[got++] = cand;
        }
    }
    U4 ws = philox(U4{0u, (uint32_t)j, (uint32_t)((uint64_t)j >> 32), 1u}, k0, k1);
    for (int t = 0; t < zeta; ++t) {
        idx[jl * zeta + t] = got_idx[t];
        sgn[jl * zeta + t] = ((ws.x >> t) & 1u) ? (int8_t)-1 : (int8_t)1;
    }
}

__global__ void k_count_rows(const int32_t* __restrict__ idx, int64_t nnz, int32_t* __restrict__ counts) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nnz) atomicAdd(&counts[idx[q]], 1);
}

// Exclusive scan of s counts -> rowptr[0..s]; one block of 1024 threads.
__global__ void k_scan_rows(const int32_t* __restrict__ counts, int64_t s, int32_t* __restrict__ rowptr,
                            int32_t* __restrict__ cursor, int32_t* __restrict__ maxcount) {
    __shared__ int32_t part[1024];
    __shared__ int32_t pmax[1024];
    int tid = threadIdx.x;
    int64_t per = ceil_div_dev(s, 1024);
    int64_t lo = tid * per, hi = min(s, lo + per);
    int32_t sum = 0, mx = 0;
    for (int64_t i = lo; i < hi; ++i) { sum += counts[i]; mx = max(mx, counts[i]); }
    part[tid] = sum;
    pmax[tid] = mx;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        int32_t v = tid >= off ? part[tid - off] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    for (int off = 512; off > 0; off >>= 1) {
        if (tid < off) pmax[tid] = max(pmax[tid], pmax[tid + off]);
        __syncthreads();
    }
    int32_t run = part[tid] - sum;
    for (int64_t i = lo; i < hi; ++i) { rowptr[i] = run; cursor[i] = run; run += counts[i]; }
    if (tid == 1023) rowptr[s] = part[1023];
    if (tid == 0) *maxcount = pmax[0];
}

// Scatter (j | sign bit) into row segments; order inside a segment is fixed
// afterwards by k_sort_rows.
__global__ void k_fill_rows(const int32_t* __restrict__ idx, const int8_t* __restrict__ sgn, int64_t m, int zeta,
                            int32_t* __restrict__ cursor, uint32_t* __restrict__ col) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= m * zeta) return;
    int64_t j = q / zeta;
    int32_t r = idx[q];
    int32_t pos = atomicAdd(&cursor[r], 1);
    col[pos] = (uint32_t)j | (sgn[q] < 0 ? 0x80000000u : 0u);
}

// Sort each row segment by column index j (bitonic sort in shared memory).
// Dynamic shared memory holds `cap` uint32 entries (cap a power of two).
__global__ void k_sort_rows(const int32_t* __restrict__ rowptr, uint32_t* __restrict__ col, int cap,
                            int32_t* __restrict__ err) {
    extern __shared__ uint32_t seg[];
    int64_t r = blockIdx.x;
    int32_t lo = rowptr[r], hi = rowptr[r + 1];
    int len = hi - lo;
    if (len > cap) {
        if (threadIdx.x == 0) set_info_once(err, -3);
        return;
    }
    int pw = 1;
    while (pw < len) pw <<= 1;
    for (int i = threadIdx.x; i < pw; i += blockDim.x) seg[i] = i < len ? col[lo + i] : 0xffffffffu;
    __syncthreads();
    for (int k = 2; k <= pw; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int i = threadIdx.x; i < pw; i += blockDim.x) {
                int p = i ^ jj;
                if (p > i) {
                    uint32_t a = seg[i], b = seg[p];
                    uint32_t ka = a == 0xffffffffu ? a : (a & 0x7fffffffu);
                    uint32_t kb = b == 0xffffffffu ? b : (b & 0x7fffffffu);
                    bool up = (i & k) == 0;
                    if ((ka > kb) == up) { seg[i] = b; seg[p] = a; }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < len; i += blockDim.x) col[lo + i] = seg[i];
}

// ---------------------------------------------------------------------------
// Column scaling: colmax over rows (atomicMax on the bit pattern of a
// non-negative double, which orders like the value), then the exponent.
// ---------------------------------------------------------------------------
__global__ void k_colmax(const double* __restrict__ A, int64_t m, int64_t n, int64_t lda, int64_t rows_per_block,
                         unsigned long long* __restrict__ colmax) {
    int64_t c = blockIdx.y;
    int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    int64_t r1 = min(m, r0 + rows_per_block);
    // |a| as the bit pattern with the sign cleared: for non-NaN doubles the
    // integer order is the value order, so no FP64 instruction is needed
    unsigned long long mx = 0;
    const unsigned long long* col = (const unsigned long long*)(A + c * lda);
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        unsigned long long v = col[i] & 0x7fffffffffffffffull;
        mx = v > mx ? v : mx;
    }
    for (int off = 16; off > 0; off >>= 1) {
        unsigned long long o = __shfl_xor_sync(0xffffffffu, mx, off);
        mx = o > mx ? o : mx;
    }
    __shared__ unsigned long long wmax[32];
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        unsigned long long v = threadIdx.x < (blockDim.x >> 5) ? wmax[threadIdx.x] : 0ull;
        for (int off = 16; off > 0; off >>= 1) {
            unsigned long long o = __shfl_xor_sync(0xffffffffu, v, off);
            v = o > v ? o : v;
        }
        if (threadIdx.x == 0) atomicMax(&colmax[c], v);
    }
}

__global__ void k_colexp(const unsigned long long* __restrict__ colmax, int64_t n, int prec, int32_t* __restrict__ e) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    double mx = __longlong_as_double((long long)colmax[c]);
    int t = prec == LSQ_FP8_E4M3 ? 8 : (prec == LSQ_FP16 ? 15 : 0);
    if (prec == LSQ_FP64 || mx == 0.0 || !isfinite(mx)) { e[c] = 0; return; }
    int E;
    frexp(mx, &E);
    e[c] = t - E;
}

// Ahat in ROW-major order (n contiguous per row j), for the sparse gather.
// 32x32 tiles through shared memory so both the read of column-major A and
// the write are coalesced.
__global__ void k_quantize_rm(const double* __restrict__ A, int64_t m, int64_t n, int64_t lda,
                              const int32_t* __restrict__ colexp, int prec, void* __restrict__ out) {
    __shared__ unsigned long long tile[32][33];
    int64_t j0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
    int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    const bool f64 = prec == LSQ_FP64;
    for (int k = ty; k < 32; k += 8) {
        int64_t j = j0 + tx, c = c0 + k;
        unsigned long long v = 0;
        if (j < m && c < n) {
            double a = A[j + c * lda];
            v = f64 ? (unsigned long long)__double_as_longlong(a) : (unsigned long long)quant_bits(a, colexp[c], prec);
        }
        tile[k][tx] = v;
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        int64_t j = j0 + k, c = c0 + tx;
        if (j < m && c < n) {
            if (f64) ((unsigned long long*)out)[(size_t)j * n + c] = tile[tx][k];
            else store_bits(out, (size_t)j * n + c, (uint32_t)tile[tx][k], prec);
        }
    }
}

// The same with 64 x 64 tiles and 16-byte row-major stores (ES bytes per
// element; n * ES a multiple of 16).
template <int ES>
__global__ void __launch_bounds__(256) k_quantize_rm_v(const double* __restrict__ A, int64_t m, int64_t n,
                                                       int64_t lda, const int32_t* __restrict__ colexp, int prec,
                                                       void* __restrict__ out) {
    using W = typename std::conditional<ES == 8, unsigned long long, uint32_t>::type;
    __shared__ W tile[64][65];  // [column][row]
    const int64_t j0 = (int64_t)blockIdx.x * 64, c0 = (int64_t)blockIdx.y * 64;
    const int t = threadIdx.x, tx = t & 63, ty = t >> 6;
    for (int c = ty; c < 64; c += 4) {
        const int64_t j = j0 + tx, cc = c0 + c;
        W v = 0;
        if (j < m && cc < n) {
            const double a = A[j + cc * lda];
            if constexpr (ES == 8) v = (W)__double_as_longlong(a);
            else v = (W)quant_bits(a, colexp[cc], prec);
        }
        tile[c][tx] = v;
    }
    __syncthreads();
    constexpr int PER = 16 / ES;  // elements per 16-byte store
    constexpr int GRP = 64 / PER;  // stores per row of the tile
    for (int q = t; q < 64 * GRP; q += 256) {
        const int r = q / GRP, g = q % GRP;
        const int64_t j = j0 + r, cc = c0 + (int64_t)g * PER;
        if (j >= m || cc >= n) continue;
        uint32_t w[4] = {0, 0, 0, 0};
        if constexpr (ES == 8) {
            const unsigned long long a = tile[g * 2][r], b = tile[g * 2 + 1][r];
            w[0] = (uint32_t)a; w[1] = (uint32_t)(a >> 32); w[2] = (uint32_t)b; w[3] = (uint32_t)(b >> 32);
        } else {
#pragma unroll
            for (int e = 0; e < PER; ++e) {
                const uint32_t bits = tile[g * PER + e][r];
                const int word = (e * ES) / 4, sh = ((e * ES) % 4) * 8;
                w[word] |= (ES == 4 ? bits : (bits & ((1u << (8 * ES)) - 1u))) << sh;
            }
        }
        *(uint4*)((char*)out + ((size_t)j * n + cc) * ES) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Ahat in COLUMN-major order with leading dimension ldq (K-major operand of
// the Gaussian sketch GEMM).
__global__ void k_quantize_cm(const double* __restrict__ A, int64_t m, int64_t n, int64_t lda,
                              const int32_t* __restrict__ colexp, int prec, void* __restrict__ out, int64_t ldq) {
    int64_t c = blockIdx.y;
    int e = colexp[c];
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < ldq; j += (int64_t)gridDim.x * blockDim.x) {
        if (prec == LSQ_FP64) {
            ((double*)out)[(size_t)c * ldq + j] = j < m ? A[j + c * lda] : 0.0;
        } else {
            store_bits(out, (size_t)c * ldq + j, j < m ? quant_bits(A[j + c * lda], e, prec) : 0u, prec);
        }
    }
}

// Sparse-sign gather, one block per sketch row i: acc[c] = sum over the row's
// nonzeros (ascending j) of +-Ahat[j, c]; FP32 accumulation for low
// precisions, FP64 for FP64.  As column-major (ld ldas), float or double.
template <typename TS, typename TACC>
__global__ void k_sparse_gather(const int32_t* __restrict__ rowptr, const uint32_t* __restrict__ col,
                                const TS* __restrict__ Ahat, int64_t n, TACC* __restrict__ As, int64_t ldas) {
    __shared__ uint32_t ent[256];
    int64_t i = blockIdx.x;
    int32_t lo = rowptr[i], hi = rowptr[i + 1];
    for (int64_t c0 = 0; c0 < n; c0 += (int64_t)blockDim.x * 4) {
        TACC acc[4] = {0, 0, 0, 0};
        for (int32_t k0 = lo; k0 < hi; k0 += 256) {
            int cnt = min(256, hi - k0);
            __syncthreads();
            if (threadIdx.x < cnt) ent[threadIdx.x] = col[k0 + threadIdx.x];
            __syncthreads();
            for (int q = 0; q < cnt; ++q) {
                uint32_t e = ent[q];
                const TS* row = Ahat + (size_t)(e & 0x7fffffffu) * n;
                bool neg = (e >> 31) != 0;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    int64_t c = c0 + (int64_t)u * blockDim.x + threadIdx.x;
                    if (c < n) {
                        TACC v = (TACC)to_acc<TS, TACC>(row[c]);
                        acc[u] = neg ? acc[u] - v : acc[u] + v;
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int64_t c = c0 + (int64_t)u * blockDim.x + threadIdx.x;
            if (c < n) As[i + c * ldas] = acc[u];
        }
    }
}

// The same gather with 16-byte loads: 8 sketch rows per block (one warp each),
// lane l owning VW = 16 / sizeof(TS) consecutive columns of a 32 VW chunk; 8
// entries' rows are loaded before they are added in the row's order (so the
// sums are the same, bit for bit); the 8 rows of a chunk go out through
// shared memory so that each column's 8 consecutive rows form one store.
// Needs n * sizeof(TS) to be a multiple of 16.
template <typename TS, typename TACC>
__global__ void __launch_bounds__(256) k_sparse_gather_v(const int32_t* __restrict__ rowptr,
                                                         const uint32_t* __restrict__ col,
                                                         const TS* __restrict__ Ahat, int64_t s, int64_t n,
                                                         TACC* __restrict__ As, int64_t ldas) {
    constexpr int VW = 16 / (int)sizeof(TS);
    constexpr int CH = 32 * VW;  // columns per chunk
    __shared__ TACC tile[8][CH + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 8 + warp;
    const bool live = i < s;
    const int32_t lo = live ? rowptr[i] : 0, hi = live ? rowptr[i + 1] : 0;
    for (int64_t c0 = 0; c0 < n; c0 += CH) {
        const int64_t cl = c0 + (int64_t)lane * VW;  // first column of this lane
        const bool cin = cl < n;
        TACC acc[VW];
#pragma unroll
        for (int v = 0; v < VW; ++v) acc[v] = (TACC)0;
        for (int32_t k0 = lo; k0 < hi; k0 += 32) {
            const int cnt = min(32, hi - k0);
            const uint32_t my = lane < cnt ? col[k0 + lane] : 0u;
            for (int q0 = 0; q0 < cnt; q0 += 8) {
                uint4 raw[8];
                uint32_t e[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    e[u] = __shfl_sync(0xffffffffu, my, (q0 + u) & 31);
                    const TS* row = Ahat + (size_t)(e[u] & 0x7fffffffu) * n;
                    raw[u] = (q0 + u < cnt && cin) ? *(const uint4*)(row + cl) : make_uint4(0, 0, 0, 0);
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (q0 + u < cnt) {
                        const bool neg = (e[u] >> 31) != 0;
                        const TS* vals = reinterpret_cast<const TS*>(&raw[u]);
#pragma unroll
                        for (int v = 0; v < VW; ++v) {
                            const TACC x = (TACC)to_acc<TS, TACC>(vals[v]);
                            acc[v] = neg ? acc[v] - x : acc[v] + x;
                        }
                    }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int v = 0; v < VW; ++v) tile[warp][lane * VW + v] = acc[v];
        __syncthreads();
        for (int q = threadIdx.x; q < 8 * CH; q += 256) {
            const int r = q & 7, c = q >> 3;
            const int64_t gi = (int64_t)blockIdx.x * 8 + r, gc = c0 + c;
            if (gi < s && gc < n) As[gi + gc * ldas] = tile[r][c];
        }
    }
}

// ---------------------------------------------------------------------------
// Gaussian operator (the ziggurat and its grid: csrc/gauss.cuh).  The tables:
// x_L and f(x_L) by the equal-area recurrence in FP64, and the first round's
// integer acceptance bounds K_L = min{u : fl(u (x_L 2^-53)) >= x_{L+1}} by
// bisection with the same FP64 product.
// ---------------------------------------------------------------------------
const ZigTable& zig_table() {
    static const ZigTable t = [] {
        ZigTable z{};
        const double fr = std::exp(-0.5 * kZigR * kZigR);
        const double tail = std::sqrt(0.5 * 3.14159265358979323846) * std::erfc(kZigR / std::sqrt(2.0));
        const double v = kZigR * fr + tail;
        z.x[0] = v / fr;
        z.x[1] = kZigR;
        z.f[0] = 0.0;
        z.f[1] = fr;
        for (int i = 1; i < kZigN - 1; ++i) {
            const double fnext = z.f[i] + v / z.x[i];
            z.x[i + 1] = std::sqrt(-2.0 * std::log(fnext));
            z.f[i + 1] = std::exp(-0.5 * z.x[i + 1] * z.x[i + 1]);
        }
        z.x[kZigN] = 0.0;
        z.f[kZigN] = 1.0;
        for (int L = 0; L < kZigN; ++L) {
            const double xs = z.x[L] * 0x1p-53;
            unsigned long long lo = 0, hi = 1ull << 53;  // the answer lies in [lo, hi]
            while (lo < hi) {
                const unsigned long long mid = lo + (hi - lo) / 2;
                if ((double)mid * xs >= z.x[L + 1]) hi = mid;
                else lo = mid + 1;
            }
            z.kfast[L] = lo;
        }
        return z;
    }();
    return t;
}

__global__ void k_gauss_gen(const ZigTable tab, uint64_t seed, int64_t s, int64_t m, int prec,
                            void* __restrict__ Om, int64_t ldo, int64_t j0) {
    __shared__ ZigShared Z;
    zig_stage(tab, Z);
    for (int64_t i = blockIdx.y; i < s; i += gridDim.y) {
        for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < ldo; j += (int64_t)gridDim.x * blockDim.x) {
            if (prec == LSQ_FP64) {
                ((double*)Om)[(size_t)i * ldo + j] = j < m ? gauss_entry(seed, i, j0 + j, Z) : 0.0;
            } else {
                store_bits(Om, (size_t)i * ldo + j, j < m ? quant_bits(gauss_entry(seed, i, j0 + j, Z), 0, prec) : 0u,
                           prec);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// FP32 Gaussian sketch on the BF16 tensor cores.  An FP32 value x (24-bit
// significand) is the exact sum of three BF16 pieces:
//   h = bf16(x), r = x - h (exact), m = bf16(r), l = r - m (exact, 8 bits).
// Omega_hat Ahat = sum over the pairs (t, u) of pieces with t + u <= 2 (the
// three dropped pairs weigh below 2^-24 relative), i.e. one BF16 GEMM over a
// K six times longer whose six K segments of length L hold
//   Omega_hat rows: l m h m h h        Ahat columns: h m l h m h
// (segment q pairs piece t_q of Omega_hat with piece u_q of Ahat).  The
// smallest pairs come first, so the FP32 accumulator is still small while it
// adds them and the rounding of the running sum at full size happens over
// one segment only, as in a plain FP32 sum.  Padding beyond m is zero.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float to_f32_rn(double x) { return __double2float_rn(x); }
__device__ __forceinline__ float to_f32_rn(float x) { return x; }

__device__ __forceinline__ void split3_bf16(float x, uint16_t& h, uint16_t& m, uint16_t& l) {
    __nv_bfloat16 bh = __float2bfloat16_rn(x);
    float r = __fsub_rn(x, __bfloat162float(bh));
    __nv_bfloat16 bm = __float2bfloat16_rn(r);
    float r2 = __fsub_rn(r, __bfloat162float(bm));
    __nv_bfloat16 bl = __float2bfloat16_rn(r2);
    h = __bfloat16_as_ushort(bh);
    m = __bfloat16_as_ushort(bm);
    l = __bfloat16_as_ushort(bl);
}

// The BF16 piece operands of the FP32 sketch are stored K-blocked: element
// (row r, k) of an operand with `rows` rows at ((k / 64) rows + r) 64 + k % 64,
// so that every 64-wide K slice of 128 rows the GEMM loads is one contiguous
// 16 KB range (few DRAM pages and TLB entries per load, whatever m).
__device__ __forceinline__ size_t kblk(int64_t k, int64_t r, int64_t rows) {
    return ((size_t)(k >> 6) * (size_t)rows + (size_t)r) * 64 + (size_t)(k & 63);
}

// Omega_hat rows (FP32-rounded Gaussian entries) as BF16 pieces: K segments
// of length L (a multiple of 64) l m h m h h, K-blocked over the s rows.
__global__ void k_gauss_split3(const ZigTable tab, uint64_t seed, int64_t s, int64_t m, int64_t L,
                               uint16_t* __restrict__ X, int64_t j0) {
    __shared__ ZigShared Z;
    zig_stage(tab, Z);
    for (int64_t i = blockIdx.y; i < s; i += gridDim.y) {
        for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < L; j += (int64_t)gridDim.x * blockDim.x) {
            uint16_t h = 0, mi = 0, l = 0;
            if (j < m) split3_bf16(gauss_f32(seed, i, j0 + j, Z), h, mi, l);
            X[kblk(j, i, s)] = l;
            X[kblk(L + j, i, s)] = mi;
            X[kblk(2 * L + j, i, s)] = h;
            X[kblk(3 * L + j, i, s)] = mi;
            X[kblk(4 * L + j, i, s)] = h;
            X[kblk(5 * L + j, i, s)] = h;
        }
    }
}

// Ahat = FP32(A 2^colexp) columns as BF16 pieces: K segments h m l h m h,
// K-blocked over the n columns.
__global__ void k_quantize_split3(const double* __restrict__ A, int64_t m, int64_t n, int64_t lda,
                                  const int32_t* __restrict__ colexp, int64_t L, uint16_t* __restrict__ Y) {
    const int64_t c = blockIdx.y;
    const int e = colexp[c];
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < L; j += (int64_t)gridDim.x * blockDim.x) {
        uint16_t h = 0, mi = 0, l = 0;
        if (j < m) split3_bf16(__uint_as_float(quant_bits(A[j + c * lda], e, LSQ_FP32)), h, mi, l);
        Y[kblk(j, c, n)] = h;
        Y[kblk(L + j, c, n)] = mi;
        Y[kblk(2 * L + j, c, n)] = l;
        Y[kblk(3 * L + j, c, n)] = h;
        Y[kblk(4 * L + j, c, n)] = mi;
        Y[kblk(5 * L + j, c, n)] = h;
    }
}

// Gram X^T X of FP32-rounded columns on the BF16 tensor cores: the six
// pairs of pieces (t, u), t + u <= 2, chained through ONE array of seven K
// segments per column, h l h m m h h: the GEMM reads X at segment offset 0
// and Y at offset 1, which pairs (h,l) (l,h) (h,m) (m,m) (m,h) (h,h) -- the
// full-size pair last, as in the sketch.  Column c at Z + c * 7L.
template <typename TI>
__global__ void k_gram_split3(const TI* __restrict__ A, int64_t m, int64_t n, int64_t lda, int64_t L,
                              uint16_t* __restrict__ Z) {
    const int64_t c = blockIdx.y;
    uint16_t* col = Z + (size_t)c * 7 * L;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < L; j += (int64_t)gridDim.x * blockDim.x) {
        uint16_t h = 0, mi = 0, l = 0;
        if (j < m) split3_bf16(to_f32_rn(A[j + c * lda]), h, mi, l);
        col[j] = h;
        col[L + j] = l;
        col[2 * L + j] = h;
        col[3 * L + j] = mi;
        col[4 * L + j] = mi;
        col[5 * L + j] = h;
        col[6 * L + j] = h;
    }
}

// ---------------------------------------------------------------------------
// Subsampled randomized Walsh-Hadamard sketch Omega = S F D (Eq. e_sketch):
// rows of A signed by D, zero-padded to m' = 2^ceil(log2 m), the unscaled
// Sylvester-Hadamard transform F applied to every column by butterfly levels
// h = 1, 2, ..., m'/2 in that order ((a, b) -> (a + b, a - b) on pairs
// (i, i + h), i & h = 0), in FP32 (FP64 for an FP64 sketch), then d rows
// sampled with replacement.  Each butterfly is evaluated exactly as in a
// sequential sweep, so the result does not depend on the parallel schedule.
//   D: bit (j & 31) of word (j >> 5) & 3 of Philox counter (j >> 7, 0, 0, 3);
//   S: word (t & 3) of counter (t >> 2, 0, 0, 4), masked to [0, m').
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t u4_word(const U4& w, int k) {
    return k == 0 ? w.x : k == 1 ? w.y : k == 2 ? w.z : w.w;
}

template <typename T>
__global__ void k_srft_load(const double* __restrict__ A, int64_t m, int64_t n, int64_t lda,
                            const int32_t* __restrict__ colexp, int prec, uint64_t seed, int64_t mp, int64_t cpb,
                            T* __restrict__ W) {
    const int64_t c0 = (int64_t)blockIdx.y * cpb, c1 = min64(n, c0 + cpb);
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < mp; j += (int64_t)gridDim.x * blockDim.x) {
        bool neg = false;
        if (j < m) {
            const U4 w = philox(U4{(uint32_t)((uint64_t)j >> 7), 0u, 0u, 3u}, (uint32_t)seed, (uint32_t)(seed >> 32));
            neg = (u4_word(w, (int)((j >> 5) & 3)) >> (j & 31)) & 1u;
        }
        for (int64_t c = c0; c < c1; ++c) {
            T v = (T)0;
            if (j < m) {
                if (prec == LSQ_FP64) {
                    v = (T)A[j + c * lda];
                } else {
                    // the value rounded to u_p (with the column scaling) is exact in FP32
                    double q = round_to_prec(ldexp(A[j + c * lda], colexp[c]), prec);
                    v = (T)q;
                }
                if (neg) v = -v;
            }
            W[(size_t)c * mp + j] = v;
        }
    }
}

// levels h = 1 .. B/2 inside blocks of B consecutive entries of a column
template <typename T>
__global__ void __launch_bounds__(512) k_fwht_block(T* __restrict__ W, int64_t mp, int B) {
    extern __shared__ __align__(16) unsigned char fw_raw[];
    T* x = reinterpret_cast<T*>(fw_raw);
    T* base = W + (size_t)blockIdx.y * mp + (size_t)blockIdx.x * B;
    for (int i = threadIdx.x; i < B; i += blockDim.x) x[i] = base[i];
    __syncthreads();
    for (int h = 1; h < B; h <<= 1) {
        for (int p = threadIdx.x; p < B / 2; p += blockDim.x) {
            const int i = (p / h) * 2 * h + (p % h);
            const T a = x[i], b = x[i + h];
            x[i] = a + b;
            x[i + h] = a - b;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < B; i += blockDim.x) base[i] = x[i];
}

// levels h = B .. mp/2: for 32 consecutive offsets o of a column, the
// K = mp / B entries o + k B held in shared memory, levels k-wise
template <typename T>
__global__ void __launch_bounds__(256) k_fwht_stride(T* __restrict__ W, int64_t mp, int B) {
    extern __shared__ __align__(16) unsigned char fs_raw[];
    T* x = reinterpret_cast<T*>(fs_raw);  // [K][32]
    const int K = (int)(mp / B);
    const int o0 = blockIdx.x * 32;
    T* col = W + (size_t)blockIdx.y * mp;
    for (int q = threadIdx.x; q < K * 32; q += blockDim.x) {
        const int k = q >> 5, o = q & 31;
        x[q] = col[(size_t)k * B + o0 + o];
    }
    __syncthreads();
    for (int h = 1; h < K; h <<= 1) {
        for (int q = threadIdx.x; q < (K / 2) * 32; q += blockDim.x) {
            const int p = q >> 5, o = q & 31;
            const int i = (p / h) * 2 * h + (p % h);
            const T a = x[i * 32 + o], b = x[(i + h) * 32 + o];
            x[i * 32 + o] = a + b;
            x[(i + h) * 32 + o] = a - b;
        }
        __syncthreads();
    }
    for (int q = threadIdx.x; q < K * 32; q += blockDim.x) {
        const int k = q >> 5, o = q & 31;
        col[(size_t)k * B + o0 + o] = x[q];
    }
}

template <typename T, typename TO>
__global__ void k_srft_gather(const T* __restrict__ W, int64_t mp, int64_t n, uint64_t seed, int64_t s,
                              TO* __restrict__ As, int64_t ldas) {
    const int64_t c = blockIdx.y;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < s; t += (int64_t)gridDim.x * blockDim.x) {
        const U4 w = philox(U4{(uint32_t)((uint64_t)t >> 2), 0u, 0u, 4u}, (uint32_t)seed, (uint32_t)(seed >> 32));
        const int64_t row = (int64_t)(u4_word(w, (int)(t & 3)) & (uint32_t)(mp - 1));
        As[t + c * ldas] = (TO)W[(size_t)c * mp + row];
    }
}

int64_t srft_order(int64_t m) {
    int64_t mp = 1;
    while (mp < m) mp <<= 1;
    return mp;
}

size_t srft_ws_bytes(int64_t m, int64_t n, int prec) {
    return (prec == LSQ_FP64 ? 8 : 4) * (size_t)srft_order(m) * (size_t)n;
}

template <typename T>
static lsq_status srft_run(const double* A, int64_t m, int64_t n, int64_t lda, const int32_t* colexp, int prec,
                           uint64_t seed, int64_t s, T* W, void* As, int64_t ldas, cudaStream_t st) {
    const int64_t mp = srft_order(m);
    if (mp > ((int64_t)1 << 30)) return LSQ_ERR_ARG;
    const int64_t cpb = 8;  // columns per block of the load
    dim3 gl((unsigned)min64(ceil_div(mp, 256), 4096), (unsigned)ceil_div(n, cpb));
    k_srft_load<T><<<gl, 256, 0, st>>>(A, m, n, lda, colexp, prec, seed, mp, cpb, W);
    LSQ_LAUNCH_CHECK();
    const int B = (int)std::min<int64_t>(mp, 4096);
    k_fwht_block<T><<<dim3((unsigned)(mp / B), (unsigned)n), 512, sizeof(T) * B, st>>>(W, mp, B);
    LSQ_LAUNCH_CHECK();
    if (mp > B) {
        const int K = (int)(mp / B);
        const size_t smem = sizeof(T) * (size_t)K * 32;
        if (smem > 200 * 1024) return LSQ_ERR_ARG;
        if (smem > 48 * 1024)
            LSQ_CUDA_TRY(cudaFuncSetAttribute(k_fwht_stride<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_fwht_stride<T><<<dim3((unsigned)(B / 32), (unsigned)n), 256, smem, st>>>(W, mp, B);
        LSQ_LAUNCH_CHECK();
    }
    dim3 gg((unsigned)min64(ceil_div(s, 256), 1024), (unsigned)n);
    if (prec == LSQ_FP64)
        k_srft_gather<T, double><<<gg, 256, 0, st>>>(W, mp, n, seed, s, (double*)As, ldas);
    else
        k_srft_gather<T, float><<<gg, 256, 0, st>>>(W, mp, n, seed, s, (float*)As, ldas);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

lsq_status launch_srft(const double* A, int64_t m, int64_t n, int64_t lda, const int32_t* colexp, int prec,
                       uint64_t seed, int64_t s, void* W, void* As, int64_t ldas, cudaStream_t st) {
    if (prec == LSQ_FP64) return srft_run<double>(A, m, n, lda, colexp, prec, seed, s, (double*)W, As, ldas, st);
    return srft_run<float>(A, m, n, lda, colexp, prec, seed, s, (float*)W, As, ldas, st);
}

__global__ void k_gauss_inspect(const ZigTable tab, uint64_t seed, int64_t s, int64_t m, int prec,
                                double* __restrict__ Om) {
    __shared__ ZigShared Z;
    zig_stage(tab, Z);
    int64_t total = s * m;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = q % s, j = q / s;
        Om[q] = round_to_prec(gauss_entry(seed, i, j, Z), prec);
    }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
lsq_status launch_sparse_gen(uint64_t seed, int64_t m, int64_t s, int zeta, int32_t* idx, int8_t* sgn, int32_t* err, int64_t j0,
                             cudaStream_t st) {
    k_sparse_gen<<<(unsigned)ceil_div(m, 128), 128, 0, st>>>(seed, m, (uint32_t)s, zeta, idx, sgn, err, j0);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

int sort_cap_for(int64_t m, int64_t s, int zeta) {
    // mean + generous slack; segments above the cap are reported via err = -3
    double mean = (double)m * zeta / (double)s;
    double want = mean + 12.0 * sqrt(mean + 1.0) + 64.0;
    int cap = 256;
    while (cap < want && cap < 16384) cap <<= 1;
    return cap;
}

lsq_status launch_sparse_csr(const int32_t* idx, const int8_t* sgn, int64_t m, int64_t s, int zeta, int32_t* counts,
                             int32_t* rowptr, int32_t* cursor, uint32_t* col, int32_t* maxcount, int32_t* err,
                             cudaStream_t st) {
    LSQ_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int32_t) * (size_t)s, st));
    int64_t nnz = m * zeta;
    k_count_rows<<<(unsigned)ceil_div(nnz, 256), 256, 0, st>>>(idx, nnz, counts);
    LSQ_LAUNCH_CHECK();
    k_scan_rows<<<1, 1024, 0, st>>>(counts, s, rowptr, cursor, maxcount);
    LSQ_LAUNCH_CHECK();
    k_fill_rows<<<(unsigned)ceil_div(nnz, 256), 256, 0, st>>>(idx, sgn, m, zeta, cursor, col);
    LSQ_LAUNCH_CHECK();
    int cap = sort_cap_for(m, s, zeta);
    size_t smem = sizeof(uint32_t) * (size_t)cap;
    if (smem > 48 * 1024) LSQ_CUDA_TRY(cudaFuncSetAttribute(k_sort_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_sort_rows<<<(unsigned)s, 256, smem, st>>>(rowptr, col, cap, err);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

lsq_status launch_colexp(const double* A, int64_t m, int64_t n, int64_t lda, int prec, unsigned long long* colmax,
                         int32_t* colexp, cudaStream_t st) {
    LSQ_CUDA_TRY(cudaMemsetAsync(colmax, 0, sizeof(unsigned long long) * (size_t)n, st));
    int64_t rpb = 8192;
    dim3 grid((unsigned)ceil_div(m, rpb), (unsigned)n);
    k_colmax<<<grid, 256, 0, st>>>(A, m, n, lda, rpb, colmax);
    LSQ_LAUNCH_CHECK();
    // row-sharded A: the column maxima over every shard
    lsq_status r = reduce_partial(colmax, n, LSQ_REDUCE_MAX_U64, st);
    if (r != LSQ_OK) return r;
    k_colexp<<<(unsigned)ceil_div(n, 128), 128, 0, st>>>(colmax, n, prec, colexp);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

lsq_status launch_quantize_rm(const double* A, int64_t m, int64_t n, int64_t lda, const int32_t* colexp, int prec,
                              void* out, cudaStream_t st) {
    const int es = prec_bytes(prec);
    if ((n * es) % 16 == 0 && ((uintptr_t)out % 16) == 0) {
        dim3 g((unsigned)ceil_div(m, 64), (unsigned)ceil_div(n, 64));
        switch (es) {
        case 1: k_quantize_rm_v<1><<<g, 256, 0, st>>>(A, m, n, lda, colexp, prec, out); break;
        case 2: k_quantize_rm_v<2><<<g, 256, 0, st>>>(A, m, n, lda, colexp, prec, out); break;
        case 4: k_quantize_rm_v<4><<<g, 256, 0, st>>>(A, m, n, lda, colexp, prec, out); break;
        default: k_quantize_rm_v<8><<<g, 256, 0, st>>>(A, m, n, lda, colexp, prec, out); break;
        }
        LSQ_LAUNCH_CHECK();
        return LSQ_OK;
    }
    dim3 grid((unsigned)ceil_div(m, 32), (unsigned)ceil_div(n, 32));
    k_quantize_rm<<<grid, dim3(32, 8), 0, st>>>(A, m, n, lda, colexp, prec, out);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

lsq_status launch_quantize_cm(const double* A, int64_t m, int64_t n, int64_t lda, const int32_t* colexp, int prec,
                              void* out, int64_t ldq, cudaStream_t st) {
    dim3 grid((unsigned)min64(ceil_div(ldq, 256), 64), (unsigned)n);
    k_quantize_cm<<<grid, 256, 0, st>>>(A, m, n, lda, colexp, prec, out, ldq);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

lsq_status launch_sparse_gather(const int32_t* rowptr, const uint32_t* col, const void* Ahat, int prec, int64_t s,
                                int64_t n, void* As, int64_t ldas, cudaStream_t st) {
    int threads = 256;
    if ((n * prec_bytes(prec)) % 16 == 0 && ((uintptr_t)Ahat % 16) == 0) {
        const unsigned g = (unsigned)ceil_div(s, 8);
        switch (prec) {
        case LSQ_FP8_E4M3:
            k_sparse_gather_v<__nv_fp8_storage_t, float><<<g, 256, 0, st>>>(
                rowptr, col, (const __nv_fp8_storage_t*)Ahat, s, n, (float*)As, ldas);
            break;
        case LSQ_BF16:
            k_sparse_gather_v<__nv_bfloat16, float><<<g, 256, 0, st>>>(rowptr, col, (const __nv_bfloat16*)Ahat, s, n,
                                                                       (float*)As, ldas);
            break;
        case LSQ_FP16:
            k_sparse_gather_v<__half, float><<<g, 256, 0, st>>>(rowptr, col, (const __half*)Ahat, s, n, (float*)As,
                                                                ldas);
            break;
        case LSQ_FP32:
            k_sparse_gather_v<float, float><<<g, 256, 0, st>>>(rowptr, col, (const float*)Ahat, s, n, (float*)As,
                                                               ldas);
            break;
        default:
            k_sparse_gather_v<double, double><<<g, 256, 0, st>>>(rowptr, col, (const double*)Ahat, s, n,
                                                                 (double*)As, ldas);
            break;
        }
        LSQ_LAUNCH_CHECK();
        return LSQ_OK;
    }
    switch (prec) {
    case LSQ_FP8_E4M3:
        k_sparse_gather<__nv_fp8_storage_t, float><<<(unsigned)s, threads, 0, st>>>(
            rowptr, col, (const __nv_fp8_storage_t*)Ahat, n, (float*)As, ldas);
        break;
    case LSQ_BF16:
        k_sparse_gather<__nv_bfloat16, float><<<(unsigned)s, threads, 0, st>>>(rowptr, col, (const __nv_bfloat16*)Ahat,
                                                                              n, (float*)As, ldas);
        break;
    case LSQ_FP16:
        k_sparse_gather<__half, float><<<(unsigned)s, threads, 0, st>>>(rowptr, col, (const __half*)Ahat, n,
                                                                       (float*)As, ldas);
        break;
    case LSQ_FP32:
        k_sparse_gather<float, float><<<(unsigned)s, threads, 0, st>>>(rowptr, col, (const float*)Ahat, n, (float*)As,
                                                                      ldas);
        break;
    default:
        k_sparse_gather<double, double><<<(unsigned)s, threads, 0, st>>>(rowptr, col, (const double*)Ahat, n,
                                                                        (double*)As, ldas);
        break;
    }
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

lsq_status launch_gauss_gen(uint64_t seed, int64_t s, int64_t m, int prec, void* Om, int64_t ldo, int64_t j0,
                            cudaStream_t st) {
    // a few thousand blocks, each staging the tables once
    dim3 grid((unsigned)min64(ceil_div(ldo, 256), 64), (unsigned)min64(s, 64));
    k_gauss_gen<<<grid, 256, 0, st>>>(zig_table(), seed, s, m, prec, Om, ldo, j0);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

lsq_status launch_gauss_split3(uint64_t seed, int64_t s, int64_t m, int64_t L, uint16_t* X, int64_t j0,
                               cudaStream_t st) {
    if (L % 64) return LSQ_ERR_ARG;
    dim3 grid((unsigned)min64(ceil_div(L, 256), 64), (unsigned)min64(s, 64));
    k_gauss_split3<<<grid, 256, 0, st>>>(zig_table(), seed, s, m, L, X, j0);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

lsq_status launch_quantize_split3(const double* A, int64_t m, int64_t n, int64_t lda, const int32_t* colexp,
                                  int64_t L, uint16_t* Y, cudaStream_t st) {
    if (L % 64) return LSQ_ERR_ARG;
    dim3 grid((unsigned)min64(ceil_div(L, 256), 64), (unsigned)n);
    k_quantize_split3<<<grid, 256, 0, st>>>(A, m, n, lda, colexp, L, Y);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

template <typename TI>
lsq_status launch_gram_split3(const TI* A, int64_t m, int64_t n, int64_t lda, int64_t L, uint16_t* Z, cudaStream_t st) {
    dim3 grid((unsigned)min64(ceil_div(L, 256), 64), (unsigned)n);
    k_gram_split3<TI><<<grid, 256, 0, st>>>(A, m, n, lda, L, Z);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}
template lsq_status launch_gram_split3<double>(const double*, int64_t, int64_t, int64_t, int64_t, uint16_t*,
                                               cudaStream_t);
template lsq_status launch_gram_split3<float>(const float*, int64_t, int64_t, int64_t, int64_t, uint16_t*,
                                              cudaStream_t);

lsq_status launch_gauss_inspect(uint64_t seed, int64_t s, int64_t m, int prec, double* Om, cudaStream_t st) {
    unsigned grid = (unsigned)min64(ceil_div(s * m, 256), 4096);
    k_gauss_inspect<<<grid, 256, 0, st>>>(zig_table(), seed, s, m, prec, Om);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

}  // namespace lsq
