// Gaussian sketch A_s = Omega_hat * Ahat (Alg. 1, "Sketch A_s = Omega A" in
// u_p) for 8- and 16-bit u_p on the 5th-generation tensor cores.
//
// Both operands are K-major (K = m): Omega_hat row-major s x m, Ahat
// column-major m x n.  One CTA computes a 128 x 128 tile of A_s over a K
// range, warp-specialised:
//   warp 0     one lane issues TMA loads (128 B of K x 128 rows per operand,
//              128-byte swizzle) into a 6-stage shared-memory ring;
//   warp 1     allocates 128 TMEM columns; one lane issues tcgen05.mma
//              (kind::f16 for BF16/FP16, kind::f8f6f4 for FP8-e4m3; FP32
//              accumulators in TMEM) and commits each stage back to the
//              producer;
//   warps 2-5  read the accumulators with tcgen05.ld (each warp its 32-lane
//              quadrant) and store FP32 results.
// Every mbarrier wait is bounded (2 s of %globaltimer); on a timeout the
// kernel records an error, waits (bounded) for its own copies and MMAs, frees
// its TMEM and returns.
#include "common.cuh"
#include "kernels.cuh"
#include "tcgen05.cuh"

#include <algorithm>
#include <mutex>

namespace lsq {

constexpr int TC_BM = 128, TC_BN = 128, TC_STAGES = 6, TC_THREADS = 192;
constexpr int TC_TILE_BYTES = 128 * 128;  // 128 rows x 128 bytes of K
// stages of the A / B ring for a tile N wide (192 KB of shared memory)
__host__ __device__ constexpr int tc_stages(int BN) { return (12 * TC_TILE_BYTES) / (TC_TILE_BYTES + BN * 128); }
// Instruction descriptor: D = F32, A/B format, both K-major, M = 128, N = BN.
template <int KIND, int BN>
__device__ __forceinline__ uint32_t tc_idesc() {
    return umma_idesc(KIND == 0 ? 1u : 0u, TC_BM, BN);
}

// executed by the whole issuer warp; lane `lead` issues
template <int KIND>
__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum,
                                     uint32_t lead) {
    if (KIND == 2) umma_f8_w(tmem_d, a, b, idesc, accum, lead);
    else umma_f16_w(tmem_d, a, b, idesc, accum, lead);
}

template <int KIND, int BN>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_sketch_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int64_t M, int64_t N,
                int64_t K, int64_t kchunk, float* __restrict__ out, int64_t ldo, int64_t split_stride,
                int32_t* __restrict__ err, const int2* __restrict__ tiles, int64_t ntiles, int blocked) {
    constexpr int ES = KIND == 2 ? 1 : 2;  // element bytes
    constexpr int BKE = 128 / ES;          // K elements per stage
    constexpr int ST = tc_stages(BN);
    constexpr int BBYTES = BN * 128;       // B tile: BN rows x 128 bytes of K
    extern __shared__ unsigned char tc_raw[];
    uint8_t* base = (uint8_t*)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = base;
    uint8_t* sB = sA + ST * TC_TILE_BYTES;
    uint64_t* full = (uint64_t*)(sB + ST * BBYTES);
    uint64_t* empty = full + ST;
    uint64_t* accb = empty + ST;
    uint32_t* tslot = (uint32_t*)(accb + 1);
    volatile int* bad = (volatile int*)(tslot + 1);
    int* issued = (int*)(tslot + 2);
    int* consumed = (int*)(tslot + 3);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // tile list mode: blockIdx.x picks (m0, n0) and the tile is written to its
    // own 128 x 128 slot (column-major, ld 128) of `out`; otherwise the
    // column tiles run fastest, so that the CTAs of a wave share the row
    // tiles of A (the larger operand) and read B once per wave
    const int2 tl = tiles ? tiles[blockIdx.x] : make_int2(0, 0);
    const int64_t m0 = tiles ? (int64_t)tl.x : (int64_t)blockIdx.y * TC_BM;
    const int64_t n0 = tiles ? (int64_t)tl.y : (int64_t)blockIdx.x * BN;
    const int64_t kb0 = (int64_t)blockIdx.z * kchunk;
    const int64_t kb1 = min64(K, kb0 + kchunk);
    const int nk = (int)((kb1 - kb0 + BKE - 1) / BKE);

    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accb, 1);
        *bad = 0;
        *issued = 0;
        *consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    if (warp == 0 && lane == 0) {
        // producer
        for (int kb = 0; kb < nk; ++kb) {
            int s = kb % ST, r = kb / ST;
            if (kb >= ST && !mbar_wait(&empty[s], (uint32_t)((r - 1) & 1))) {
                *bad = 1;
                break;
            }
            if (*bad) break;
            mbar_expect_tx(&full[s], TC_TILE_BYTES + BBYTES);
            int x = (int)(kb0 + (int64_t)kb * BKE);
            if (blocked) {
                // K-blocked operands: block x / BKE holds every row's 128 bytes
                tma_load_3d(sA + s * TC_TILE_BYTES, &tmA, &full[s], 0, (int)m0, x / BKE);
                tma_load_3d(sB + s * BBYTES, &tmB, &full[s], 0, (int)n0, x / BKE);
            } else {
                tma_load_2d(sA + s * TC_TILE_BYTES, &tmA, &full[s], x, (int)m0);
                tma_load_2d(sB + s * BBYTES, &tmB, &full[s], x, (int)n0);
            }
            *issued = kb + 1;
        }
    } else if (warp == 1) {
        // MMA issuer: the whole warp runs the loop in convergence, so that the
        // stage descriptors are warp-uniform values; lane 0 issues
        const uint32_t lead = lane == 0 ? 1u : 0u;
        const uint32_t idesc = tc_idesc<KIND, BN>();
        const uint64_t da0 = umma_desc(smem_u32(sA)), db0 = umma_desc(smem_u32(sB));
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % ST, r = kb / ST;
            if (!__all_sync(0xffffffffu, mbar_wait(&full[s], (uint32_t)(r & 1)))) {
                *bad = 1;
                break;
            }
            if (lead) *consumed = kb + 1;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t ad = da0 + (uint64_t)(s * (TC_TILE_BYTES >> 4));
            const uint64_t bd = db0 + (uint64_t)(s * (BBYTES >> 4));
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)  // 4 x 32 bytes of K per stage
                umma<KIND>(tmem, ad + 2 * kk, bd + 2 * kk, idesc, (kb | kk) != 0 ? 1u : 0u, lead);
            umma_commit_w(&empty[s], lead);
        }
        umma_commit_w(accb, lead);  // fires when every MMA issued above has completed
    } else if (warp >= 2) {
        // epilogue: TMEM lanes 32*(warp % 4) .. +31 hold rows of the tile
        bool ok = mbar_wait(accb, 0);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!ok) *bad = 1;
        // tcgen05.ld is warp-collective: take the decision once per warp
        const bool go = __all_sync(0xffffffffu, ok && !*bad && nk > 0);
        if (go) {
            const int quad = warp & 3;
            const int64_t row = m0 + quad * 32 + lane;
            float* o = tiles ? out + ((int64_t)blockIdx.z * ntiles + blockIdx.x) * (TC_BM * BN) - m0 - n0 * ldo
                             : out + (int64_t)blockIdx.z * split_stride;
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 16) {
                uint32_t v[16];
                uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (row < M) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        int64_t col = n0 + c0 + j;
                        if (col < N) o[row + col * ldo] = __uint_as_float(v[j]);
                    }
                }
            }
        }
    }
    __syncthreads();
    if (*bad) {
        if (threadIdx.x == 0) {
            set_info_once(err, -2);
            // wait (bounded) for loads issued but never consumed, then for the MMAs
            for (int kb = *consumed; kb < *issued; ++kb) mbar_wait(&full[kb % ST], (uint32_t)((kb / ST) & 1));
            mbar_wait(accb, 0);
        }
        __syncthreads();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
    }
}

__global__ void k_reduce_f32(const float* __restrict__ part, int splits, int64_t M, int64_t N, float* __restrict__ C,
                             int64_t ldc) {
    int64_t total = M * N;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int z = 0; z < splits; ++z) s += part[(int64_t)z * total + q];
        C[(q % M) + (q / M) * ldc] = s;
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
EncodeTiledFn tensor_map_encoder() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        cudaGetLastError();
    });
    return fn;
}

static bool make_map(CUtensorMap* map, const void* base, int prec, int64_t K, int64_t rows, int64_t ld,
                     int box_rows = 128) {
    EncodeTiledFn enc = tensor_map_encoder();
    if (!enc) return false;
    int es = prec == LSQ_FP8_E4M3 ? 1 : 2;
    CUtensorMapDataType dt = prec == LSQ_FP8_E4M3 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                             : prec == LSQ_BF16   ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                  : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * es)};
    cuuint32_t box[2] = {(cuuint32_t)(128 / es), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1u, 1u};
    CUresult r = enc(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// A K-blocked operand: element (row r, k) at ((k / B) rows + r) B + k % B with
// B = 128 bytes of K (64 BF16/FP16 or 128 FP8 values); every box of B x
// box_rows is one contiguous range.  K a multiple of B.
static bool make_map_blocked(CUtensorMap* map, const void* base, int prec, int64_t K, int64_t rows,
                             int box_rows = 128) {
    EncodeTiledFn enc = tensor_map_encoder();
    if (!enc) return false;
    const int es = prec == LSQ_FP8_E4M3 ? 1 : 2;
    const int64_t B = 128 / es;
    if (K % B) return false;
    CUtensorMapDataType dt = prec == LSQ_FP8_E4M3 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                             : prec == LSQ_BF16   ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                  : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    cuuint64_t dims[3] = {(cuuint64_t)B, (cuuint64_t)rows, (cuuint64_t)(K / B)};
    cuuint64_t strides[2] = {(cuuint64_t)128, (cuuint64_t)(rows * 128)};
    cuuint32_t box[3] = {(cuuint32_t)B, (cuuint32_t)box_rows, 1u};
    cuuint32_t estr[3] = {1u, 1u, 1u};
    CUresult r = enc(map, dt, 3, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool sketch_tc_supported(int prec) {
    return (prec == LSQ_FP8_E4M3 || prec == LSQ_BF16 || prec == LSQ_FP16) && tensor_map_encoder() != nullptr;
}

// Tile width: 128 x 256 output tiles (two 128-row blocks of Y per MMA, 25 %
// less shared-memory and L2 traffic per flop than 128 x 128) when N fills them.
static int tc_bn(int64_t N) { return N >= 256 ? 256 : TC_BN; }

// K blocks (128 bytes of K each) per split at most.  A wave of CTAs shares
// its operand slabs through L2 only while its CTAs stay close in K; over a
// long K they drift apart.  Measured on the FP32 sketch of the 262144 x 4096
// problem (K = 1.57e6 BF16 pieces, 1024 output tiles): one split 105 ms,
// splits of 4096 / 2048 / 1024 K blocks 111-117 ms, of 512 K blocks 60 ms
// (1.8 PFLOP/s of tensor work).  Shorter accumulation chains in the FP32
// accumulators are also more accurate.
constexpr int64_t TC_KBLOCKS_MAX = 512;

// Split count: fill the SMs when the tile grid is small, and at most
// TC_KBLOCKS_MAX K blocks per split; at least 4 stages of K per split.
static int tc_splits(int64_t M, int64_t N, int64_t K, int prec, int sms) {
    int64_t tiles = ceil_div(M, TC_BM) * ceil_div(N, tc_bn(N));
    int64_t bke = prec == LSQ_FP8_E4M3 ? 128 : 64;
    int64_t kblocks = ceil_div(K, bke);
    int64_t want = std::max<int64_t>(1, sms / std::max<int64_t>(1, tiles));
    want = std::max<int64_t>(want, ceil_div(kblocks, TC_KBLOCKS_MAX));
    int64_t cap = std::max<int64_t>(1, kblocks / 4);
    return (int)std::min<int64_t>(std::min<int64_t>(want, cap), 64);
}

size_t sketch_tc_ws_bytes(int64_t s, int64_t n, int64_t m, int prec, int sms) {
    int sp = tc_splits(s, n, m, prec, sms);
    return sp > 1 ? align_up(sizeof(float) * (size_t)sp * s * n, 256) : 0;
}

lsq_status launch_sketch_tc(const void* Om, int64_t ldo, const void* Ahat, int64_t ldq, int prec, int64_t s,
                            int64_t n, int64_t m, float* As, int64_t ldas, void* ws, size_t ws_bytes, int32_t* err,
                            cudaStream_t st, bool blocked) {
    if (!sketch_tc_supported(prec)) return LSQ_ERR_ARG;
    if ((ldo % 16) || (ldq % 16) || ((uintptr_t)Om % 16) || ((uintptr_t)Ahat % 16)) return LSQ_ERR_ARG;
    const int bn = tc_bn(n);
    CUtensorMap ta, tb;
    if (blocked) {
        if (!make_map_blocked(&ta, Om, prec, m, s) || !make_map_blocked(&tb, Ahat, prec, m, n, bn)) return LSQ_ERR_ARG;
    } else if (!make_map(&ta, Om, prec, m, s, ldo) || !make_map(&tb, Ahat, prec, m, n, ldq, bn)) {
        return LSQ_ERR_CUDA;
    }
    int sms = device_sm_count();
    int splits = tc_splits(s, n, m, prec, sms);
    int64_t bke = prec == LSQ_FP8_E4M3 ? 128 : 64;
    int64_t kchunk = ceil_div(ceil_div(m, splits), bke) * bke;
    splits = (int)ceil_div(m, kchunk);
    float* out = As;
    int64_t ldout = ldas, stride = 0;
    if (splits > 1) {
        if (!ws || ws_bytes < sizeof(float) * (size_t)splits * s * n) return LSQ_ERR_NOMEM;
        out = (float*)ws;
        ldout = s;
        stride = s * n;
    }
    size_t smem = 1024 + (size_t)tc_stages(bn) * (TC_TILE_BYTES + (size_t)bn * 128) + 256;
    dim3 grid((unsigned)ceil_div(n, bn), (unsigned)ceil_div(s, TC_BM), (unsigned)splits);
    stage_mark(ST_K_SKETCHTC, true, st);
    auto go = [&](auto kern) -> lsq_status {
        LSQ_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<grid, TC_THREADS, smem, st>>>(ta, tb, s, n, m, kchunk, out, ldout, stride, err, nullptr, 0,
                                             blocked ? 1 : 0);
        return LSQ_OK;
    };
    lsq_status lr;
    if (prec == LSQ_BF16) lr = bn == 256 ? go(k_sketch_tc<0, 256>) : go(k_sketch_tc<0, TC_BN>);
    else if (prec == LSQ_FP16) lr = bn == 256 ? go(k_sketch_tc<1, 256>) : go(k_sketch_tc<1, TC_BN>);
    else lr = bn == 256 ? go(k_sketch_tc<2, 256>) : go(k_sketch_tc<2, TC_BN>);
    if (lr != LSQ_OK) return lr;
    LSQ_LAUNCH_CHECK();
    stage_mark(ST_K_SKETCHTC, false, st, 2.0 * (double)s * (double)n * (double)m);
    if (splits > 1) {
        k_reduce_f32<<<(unsigned)std::min<int64_t>(ceil_div(s * n, 256), 8192), 256, 0, st>>>(out, splits, s, n, As,
                                                                                            ldas);
        LSQ_LAUNCH_CHECK();
    }
    return LSQ_OK;
}

}  // namespace lsq

namespace lsq {

// Tile-list launch (FP8-e4m3 operands): tiles[i] = (row of X, row of Y) of a
// 128 x 256 output tile (256 consecutive rows of Y); tile i of K chunk z goes
// to out + (z ntiles + i) 32768 (column-major, ld 128).  The wide tile reads
// 12 KB of operands per 128 x 256 x 32 MMA instead of 8 KB per 128 x 128 x 32:
// 25 % less shared-memory traffic per flop (operands and TMA writes).
lsq_status launch_tc_tiles_fp8(const void* X, int64_t ldx, int64_t rowsX, const void* Y, int64_t ldy, int64_t rowsY,
                               int64_t K, int64_t kchunk, const int2* tiles, int64_t ntiles, float* out, int32_t* err,
                               cudaStream_t st) {
    constexpr int BN = 256;
    if ((ldx % 16) || (ldy % 16) || ((uintptr_t)X % 16) || ((uintptr_t)Y % 16) || kchunk % 128) return LSQ_ERR_ARG;
    CUtensorMap ta, tb;
    if (!make_map(&ta, X, LSQ_FP8_E4M3, K, rowsX, ldx) || !make_map(&tb, Y, LSQ_FP8_E4M3, K, rowsY, ldy, BN))
        return LSQ_ERR_CUDA;
    int chunks = (int)ceil_div(K, kchunk);
    size_t smem = 1024 + (size_t)tc_stages(BN) * (TC_TILE_BYTES + BN * 128) + 256;
    LSQ_CUDA_TRY(cudaFuncSetAttribute(k_sketch_tc<2, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((unsigned)ntiles, 1, (unsigned)chunks);
    k_sketch_tc<2, BN><<<grid, TC_THREADS, smem, st>>>(ta, tb, rowsX, rowsY, K, kchunk, out, TC_BM, 0, err, tiles,
                                                      ntiles, 0);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
}

}  // namespace lsq

extern "C" lsq_status lsq_tc_gemm(int32_t prec, const void* X, int64_t ldx, const void* Y, int64_t ldy, int64_t M,
                                  int64_t N, int64_t K, float* C, int64_t ldc, int32_t* info, void* ws,
                                  size_t ws_bytes, void* stream) {
    using namespace lsq;
    if (!X || !Y || !C || M <= 0 || N <= 0 || K <= 0 || ldx < K || ldy < K || ldc < M) return LSQ_ERR_ARG;
    if (!sketch_tc_supported(prec)) return LSQ_ERR_ARG;
    return launch_sketch_tc(X, ldx, Y, ldy, prec, M, N, K, C, ldc, ws, ws_bytes, info, (cudaStream_t)stream);
}

extern "C" size_t lsq_tc_gemm_workspace_size(int32_t prec, int64_t M, int64_t N, int64_t K) {
    using namespace lsq;
    return sketch_tc_ws_bytes(M, N, K, prec, device_sm_count()) + 256;
}
