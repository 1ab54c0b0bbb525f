// tc_gemm.cu -- split-TF32 ("3xTF32") dense products on the 5th-generation
// tensor cores (tcgen05) for the low-precision transforms of Algorithm 3
// (steps 8 and 10: V^T R V and V Y V^T).
//
// C (M x N) = A B with both operands given K-contiguous ("K-major"):
//   A(i, k) = a[k + i * lda]   (row i of A is contiguous),
//   B(k, j) = b[k + j * ldb]   (column j of B is contiguous),
// FP32 in global memory.  Each operand x is split on the fly into
// hi = tf32(x) (round to nearest, 10 explicit mantissa bits) and
// lo = tf32(x - hi); C = A_hi B_hi + A_hi B_lo + A_lo B_hi is accumulated in
// FP32 in tensor memory (relative error about 2^-21, close to FP32).
//
// Persistent: one CTA per SM loops over 128 x 128 tiles of C (the upper
// block triangle for the mirrored epilogue), K in steps of 32, with warp
// roles: warp 0 issues the TMA loads of the FP32 tiles (128 rows x 128
// bytes, 128-byte swizzle) into a 3-stage ring; warps 2-5 split each landed
// stage in shared memory (hi in place, lo beside it); warp 1 issues 3 x 4
// tcgen05.mma (M = 128, N = 128, K = 8) per stage into one of two
// 128-column TMEM accumulators and commits them to the stage's mbarrier;
// warps 6-9 read the other accumulator back with tcgen05.ld for the fused
// epilogue of the previous tile.  Every mbarrier wait is bounded (about 2 s
// of globaltimer) and ends early once another role has given up; then the
// kernel records status 6, drains its outstanding copies (bounded too),
// frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "internal.h"
#include "tc_common.cuh"
#include "tc_gemm.h"

namespace sqm {

static constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 32, TC_STAGES = 3;
static constexpr int TC_SPLIT_WARPS = 4;
// warp 0 TMA, warp 1 MMA, warps 2-5 split, warps 6-9 epilogue
static constexpr int TC_THREADS = 32 * (2 + TC_SPLIT_WARPS + 4);
static constexpr int TC_TILE_BYTES = TC_BM * TC_BK * 4;          // 16 KB
static constexpr int TC_STAGE_BYTES = 4 * TC_TILE_BYTES;          // A, A_lo, B, B_lo
static constexpr int TC_SMEM = TC_STAGES * TC_STAGE_BYTES + 1024 + 256;

// round an FP32 value to TF32 (nearest, ties away from zero on the bit
// pattern); the result keeps 10 explicit mantissa bits
__device__ __forceinline__ float to_tf32(float x)
{
    uint32_t b = __float_as_uint(x);
    b = (b + 0x1000u) & 0xFFFFE000u;
    return __uint_as_float(b);
}

// the fused epilogue of one row of a tile for accumulator columns
// c0 .. c0+31 (r: the row's 32 FP32 values); the FP64 epilogues go in two
// halves of 16 columns, each with all its loads first (the stores go to the
// same array, so a load after them would wait out a full round trip)
template <int EPI>
__device__ __forceinline__ void tc3_epilogue_chunk(const uint32_t (&r)[32], int row, int n0, int c0, int N,
                                                   const TcEpilogue &ep)
{
    if (EPI == TC_EPI_SYM_ADD_F64) {
#pragma unroll
        for (int h = 0; h < 32; h += 16) {
            double old[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int col = n0 + c0 + h + j;
                old[j] = (col < N && row <= col) ? ep.X[row + (int64_t)col * ep.ldx] : 0.0;
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int col = n0 + c0 + h + j;
                if (col >= N || row > col) continue;
                const double x = old[j] + (double)__uint_as_float(r[h + j]) * ep.scale;
                ep.X[row + (int64_t)col * ep.ldx] = x;
                ep.X[col + (int64_t)row * ep.ldx] = x;
            }
        }
    } else if (EPI == TC_EPI_CSTORE || EPI == TC_EPI_CSTORE_T) {
        // accumulator columns (2q, 2q+1) = (Re, Im) of complex column q
#pragma unroll
        for (int j = 0; j < 32; j += 2) {
            const int col = n0 + c0 + j;
            if (col >= N) continue;  // N even: col + 1 < N as well
            const int q = col >> 1;
            const int64_t at = EPI == TC_EPI_CSTORE ? (row + (int64_t)q * ep.ldc) : (q + (int64_t)row * ep.ldc);
            *reinterpret_cast<float2 *>(ep.C + 2 * at) = make_float2(__uint_as_float(r[j]), __uint_as_float(r[j + 1]));
        }
    } else if (EPI == TC_EPI_RE_F64_STORE || EPI == TC_EPI_RE_F64_ADD) {
#pragma unroll
        for (int h = 0; h < 32; h += 16) {
            double old[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int col = n0 + c0 + h + j;
                old[j] = (EPI == TC_EPI_RE_F64_ADD && col < N) ? ep.X[row + (int64_t)col * ep.ldx] : 0.0;
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int col = n0 + c0 + h + j;
                if (col >= N) continue;
                ep.X[row + (int64_t)col * ep.ldx] = old[j] + (double)__uint_as_float(r[h + j]) * ep.scale;
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int col = n0 + c0 + j;
            if (col >= N) continue;
            const float v = __uint_as_float(r[j]);
            if (EPI == TC_EPI_STORE) ep.C[row + (int64_t)col * ep.ldc] = v;
            else ep.C[row + (int64_t)col * ep.ldc] = v / (ep.s[row] + ep.s[col]);
        }
    }
}

// bounded mbarrier wait that also ends once another role has failed (the
// role that times out raises the flag)
__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t parity, volatile int *fail)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (*fail) return false;
        if (globaltimer_ns() - t0 > 2000000000ull) {
            *fail = 1;
            return false;
        }
    }
    return true;
}

template <int EPI>
__global__ void __launch_bounds__(TC_THREADS, 1)
tc3_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M, int N,
                int K, TcEpilogue ep, int *err)
{
    extern __shared__ unsigned char smraw[];
    __shared__ volatile int s_fail;
    __shared__ int s_issued, s_consumed, s_committed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    static_assert(TC_BN % 2 == 0, "complex column pairs stay within a tile");
    // tiles: row-major over the (M / 128) x (N / 128) grid, or its upper
    // block triangle for the mirrored epilogue
    const int TM = (M + TC_BM - 1) / TC_BM, TN = (N + TC_BN - 1) / TC_BN;
    const bool tri = EPI == TC_EPI_SYM_ADD_F64;
    const int ntiles = tri ? TN * (TN + 1) / 2 : TM * TN;  // the mirrored product is square
    auto tile_origin = [&](int q, int &m0, int &n0) {
        if (tri) {
            int I = 0;
            while (q >= TN - I) { q -= TN - I; ++I; }
            m0 = I * TC_BM;
            n0 = (I + q) * TC_BN;
        } else {
            m0 = (q / TN) * TC_BM;
            n0 = (q % TN) * TC_BN;
        }
    };

    // 1024-aligned stage ring, then barriers and the TMEM address slot
    unsigned char *base = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(base + TC_STAGES * TC_STAGE_BYTES);  // FP32 tiles landed
    uint64_t *split = full + TC_STAGES;                                 // hi / lo written
    uint64_t *empty = split + TC_STAGES;                                // products of the stage done
    uint64_t *accf = empty + TC_STAGES;                                 // accumulator holds a tile
    uint64_t *acce = accf + 2;                                          // accumulator free again
    uint32_t *tmem_slot = (uint32_t *)(acce + 2);
    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&split[s], TC_SPLIT_WARPS * 32);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&accf[a], 1);
            mbar_init(&acce[a], 4 * 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
        s_issued = s_consumed = s_committed = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(2 * TC_BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int KT = (K + TC_BK - 1) / TC_BK;
    auto stage_ptr = [&](int s, int which) { return base + s * TC_STAGE_BYTES + which * TC_TILE_BYTES; };
    if (warp == 0) {
        // TMA producer
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
                int m0, n0;
                tile_origin(tile, m0, n0);
                for (int t = 0; t < KT; ++t, ++it) {
                    const int s = it % TC_STAGES, u = it / TC_STAGES;
                    if (u > 0 && !tc_wait(&empty[s], (u - 1) & 1, &s_fail)) { ok = false; break; }
                    mbar_arrive_expect_tx(&full[s], 2 * TC_TILE_BYTES);
                    tma_load_2d(stage_ptr(s, 0), &mapA, &full[s], t * TC_BK, m0);
                    tma_load_2d(stage_ptr(s, 2), &mapB, &full[s], t * TC_BK, n0);
                }
            }
            s_issued = it;
        }
    } else if (warp == 1) {
        // MMA issuer
        if (lane == 0) {
            constexpr uint32_t IDESC = idesc_tf32_128x128();
            int it = 0, lt = 0, committed = 0;
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x, ++lt) {
                const int a = lt & 1, v = lt >> 1;
                if (v > 0 && !tc_wait(&acce[a], (v - 1) & 1, &s_fail)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(a * TC_BN);
                for (int t = 0; t < KT; ++t, ++it) {
                    const int s = it % TC_STAGES;
                    if (!tc_wait(&split[s], (it / TC_STAGES) & 1, &s_fail)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(stage_ptr(s, 0)), al = smem_u32(stage_ptr(s, 1));
                    const uint32_t b0 = smem_u32(stage_ptr(s, 2)), bl = smem_u32(stage_ptr(s, 3));
#pragma unroll
                    for (int kk = 0; kk < TC_BK / 8; ++kk) {
                        const uint32_t off = kk * 32;  // 8 TF32 values = 32 bytes along K
                        const uint32_t acc0 = (t > 0 || kk > 0) ? 1u : 0u;
                        mma_tf32(d, smem_desc_sw128(a0 + off), smem_desc_sw128(b0 + off), IDESC, acc0);
                        mma_tf32(d, smem_desc_sw128(a0 + off), smem_desc_sw128(bl + off), IDESC, 1u);
                        mma_tf32(d, smem_desc_sw128(al + off), smem_desc_sw128(b0 + off), IDESC, 1u);
                    }
                    mma_commit(&empty[s]);
                    committed = it + 1;
                }
                if (ok) mma_commit(&accf[a]);
            }
            s_committed = committed;
        }
    } else if (warp < 2 + TC_SPLIT_WARPS) {
        // split each landed stage into hi = tf32(x) (in place) and
        // lo = tf32(x - hi) (beside it)
        const int st = tid - 64;
        int it = 0;
        bool ok = true;
        for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
            for (int t = 0; t < KT; ++t, ++it) {
                const int s = it % TC_STAGES;
                if (!tc_wait(&full[s], (it / TC_STAGES) & 1, &s_fail)) { ok = false; break; }
                if (st == 0) s_consumed = it + 1;
                float4 *a = (float4 *)stage_ptr(s, 0), *alo = (float4 *)stage_ptr(s, 1);
                float4 *b = (float4 *)stage_ptr(s, 2), *blo = (float4 *)stage_ptr(s, 3);
                constexpr int NV = TC_TILE_BYTES / 16;
#pragma unroll 4
                for (int v = st; v < NV; v += TC_SPLIT_WARPS * 32) {
                    float4 x = a[v], h, l;
                    h.x = to_tf32(x.x); h.y = to_tf32(x.y); h.z = to_tf32(x.z); h.w = to_tf32(x.w);
                    l.x = to_tf32(x.x - h.x); l.y = to_tf32(x.y - h.y); l.z = to_tf32(x.z - h.z); l.w = to_tf32(x.w - h.w);
                    a[v] = h; alo[v] = l;
                    x = b[v];
                    h.x = to_tf32(x.x); h.y = to_tf32(x.y); h.z = to_tf32(x.z); h.w = to_tf32(x.w);
                    l.x = to_tf32(x.x - h.x); l.y = to_tf32(x.y - h.y); l.z = to_tf32(x.z - h.z); l.w = to_tf32(x.w - h.w);
                    b[v] = h; blo[v] = l;
                }
                fence_proxy_async();  // the writes, before the tensor cores read them
                mbar_arrive(&split[s]);
            }
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, i.e. tile rows
        const int qw = warp & 3;
        int lt = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++lt) {
            const int a = lt & 1, v = lt >> 1;
            // every lane waits; the warp leaves together if any lane gave up
            // (the TMEM loads below are warp-collective)
            const bool okw = tc_wait(&accf[a], v & 1, &s_fail);
            if (!__all_sync(0xffffffffu, okw)) break;
            tc_fence_after();
            int m0, n0;
            tile_origin(tile, m0, n0);
            const int row = m0 + 32 * qw + lane;
            for (int c0 = 0; c0 < TC_BN; c0 += 32) {
                uint32_t r[32];
                tmem_ld32(tmem + ((uint32_t)(32 * qw) << 16) + (uint32_t)(a * TC_BN + c0), r);
                if (row < M) tc3_epilogue_chunk<EPI>(r, row, n0, c0, N, ep);
            }
            tc_fence_before();
            mbar_arrive(&acce[a]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (s_fail) {
        // drain what is still in flight (bounded) before shared and tensor
        // memory are released: TMA copies not yet observed, committed MMAs
        if (tid == 0) {
            atomicExch(err, 6);
            for (int t = s_consumed; t < s_issued; ++t) mbar_wait(&full[t % TC_STAGES], (t / TC_STAGES) & 1);
            if (s_committed > 0) mbar_wait(&empty[(s_committed - 1) % TC_STAGES], ((s_committed - 1) / TC_STAGES) & 1);
        }
        __syncthreads();
    }
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TC_BN) : "memory");
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// 2-D map over a K-contiguous operand: dim0 = K (contiguous), dim1 = rows
static bool make_map(CUtensorMap *m, const float *ptr, int64_t kdim, int64_t rows, int64_t ld)
{
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)kdim, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {TC_BK, TC_BM};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)ptr, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool tc_gemm_supported(int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb, const void *A, const void *B)
{
    if (M <= 0 || N <= 0 || K <= 0) return false;
    if ((lda * 4) % 16 || (ldb * 4) % 16) return false;           // TMA global stride rule
    if (((uintptr_t)A) % 16 || ((uintptr_t)B) % 16) return false;  // TMA base alignment
    return encode_fn() != nullptr;
}

template <int EPI>
static cudaError_t launch_epi(int g, const CUtensorMap &ma, const CUtensorMap &mb, int M, int N, int K,
                              const TcEpilogue &ep, int *err, cudaStream_t s)
{
    cudaError_t e;
    if ((e = allow_max_smem((const void *)tc3_gemm_kernel<EPI>))) return e;
    tc3_gemm_kernel<EPI><<<g, TC_THREADS, TC_SMEM, s>>>(ma, mb, M, N, K, ep, err);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_tc3_gemm(int M, int N, int K, const float *A, int lda, const float *B, int ldb, int epi,
                            const TcEpilogue &ep, int *err, cudaStream_t s)
{
    if (M <= 0 || N <= 0) return cudaSuccess;
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, K, M, lda) || !make_map(&mb, B, K, N, ldb)) return cudaErrorInvalidValue;
    // persistent: one CTA per SM (at most one per tile)
    const int64_t TM = cdiv_i(M, TC_BM), TN = cdiv_i(N, TC_BN);
    const int64_t ntiles = epi == TC_EPI_SYM_ADD_F64 ? TN * (TN + 1) / 2 : TM * TN;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, sms));
    cudaError_t e;
    switch (epi) {
    case TC_EPI_CSTORE: return launch_epi<TC_EPI_CSTORE>(g, ma, mb, M, N, K, ep, err, s);
    case TC_EPI_CSTORE_T: return launch_epi<TC_EPI_CSTORE_T>(g, ma, mb, M, N, K, ep, err, s);
    case TC_EPI_RE_F64_STORE: return launch_epi<TC_EPI_RE_F64_STORE>(g, ma, mb, M, N, K, ep, err, s);
    case TC_EPI_RE_F64_ADD: return launch_epi<TC_EPI_RE_F64_ADD>(g, ma, mb, M, N, K, ep, err, s);
    default: break;
    }
    switch (epi) {
    case TC_EPI_STORE:
        if ((e = allow_max_smem((const void *)tc3_gemm_kernel<TC_EPI_STORE>))) return e;
        tc3_gemm_kernel<TC_EPI_STORE><<<g, TC_THREADS, TC_SMEM, s>>>(ma, mb, M, N, K, ep, err); count_launch();
        break;
    case TC_EPI_DIAG_SOLVE:
        if ((e = allow_max_smem((const void *)tc3_gemm_kernel<TC_EPI_DIAG_SOLVE>))) return e;
        tc3_gemm_kernel<TC_EPI_DIAG_SOLVE><<<g, TC_THREADS, TC_SMEM, s>>>(ma, mb, M, N, K, ep, err); count_launch();
        break;
    default:
        if ((e = allow_max_smem((const void *)tc3_gemm_kernel<TC_EPI_SYM_ADD_F64>))) return e;
        tc3_gemm_kernel<TC_EPI_SYM_ADD_F64><<<g, TC_THREADS, TC_SMEM, s>>>(ma, mb, M, N, K, ep, err); count_launch();
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// complex products as real ones
// ---------------------------------------------------------------------------
// B column 2j (and 2j+1 unless re_only) from column j of Y, one thread per
// (l, j): rows 2l, 2l+1
__global__ void tc_relayout_cplx_kernel(const float2 *__restrict__ Y, int64_t ldy, int k, int n, float sa, float sy,
                                        int re_only, float *__restrict__ B, int64_t ldb)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)k * n) return;
    const int l = (int)(t % k), j = (int)(t / k);
    const float2 y = Y[l + (int64_t)j * ldy];
    const int64_t c0 = re_only ? j : 2 * (int64_t)j;
    B[2 * l + c0 * ldb] = y.x;
    B[2 * l + 1 + c0 * ldb] = -sa * sy * y.y;
    if (!re_only) {
        B[2 * l + (c0 + 1) * ldb] = sy * y.y;
        B[2 * l + 1 + (c0 + 1) * ldb] = sa * y.x;
    }
}

__global__ void tc_relayout_real_kernel(const float *__restrict__ Y, int64_t ldy, int k, int n, float sa,
                                        float *__restrict__ B, int64_t ldb)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)k * n) return;
    const int l = (int)(t % k), j = (int)(t / k);
    const float y = Y[l + (int64_t)j * ldy];
    const int64_t c0 = 2 * (int64_t)j;
    B[2 * l + c0 * ldb] = y;
    B[2 * l + 1 + c0 * ldb] = 0.0f;
    B[2 * l + (c0 + 1) * ldb] = 0.0f;
    B[2 * l + 1 + (c0 + 1) * ldb] = sa * y;
}

// Qt = Q^T through 32 x 32 shared-memory tiles
__global__ void ctranspose_kernel(const float2 *__restrict__ Q, float2 *__restrict__ Qt, int n)
{
    __shared__ float2 tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int i = bx + threadIdx.x, j = by + r;
        if (i < n && j < n) tile[r][threadIdx.x] = Q[i + (int64_t)j * n];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int j = by + threadIdx.x, i = bx + r;
        if (i < n && j < n) Qt[j + (int64_t)i * n] = tile[threadIdx.x][r];
    }
}

cudaError_t launch_tc_relayout_cplx(const void *Y, int64_t ldy, int k, int n, float sa, float sy, bool re_only,
                                    float *B, int64_t ldb, cudaStream_t s)
{
    const int64_t tot = (int64_t)k * n;
    if (tot <= 0) return cudaSuccess;
    tc_relayout_cplx_kernel<<<(unsigned)cdiv_i(tot, 256), 256, 0, s>>>((const float2 *)Y, ldy, k, n, sa, sy,
                                                                        re_only ? 1 : 0, B, ldb);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_tc_relayout_real(const float *Y, int64_t ldy, int k, int n, float sa, float *B, int64_t ldb,
                                    cudaStream_t s)
{
    const int64_t tot = (int64_t)k * n;
    if (tot <= 0) return cudaSuccess;
    tc_relayout_real_kernel<<<(unsigned)cdiv_i(tot, 256), 256, 0, s>>>(Y, ldy, k, n, sa, B, ldb);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_ctranspose(const void *Q, void *Qt, int n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    ctranspose_kernel<<<dim3((unsigned)cdiv_i(n, 32), (unsigned)cdiv_i(n, 32)), dim3(32, 8), 0, s>>>(
        (const float2 *)Q, (float2 *)Qt, n);
    count_launch();
    return cudaGetLastError();
}

bool tc_cgemm_supported(int64_t lda_c, int64_t ldb, const void *A, const void *B)
{
    return tc_gemm_supported(1, 1, 1, 2 * lda_c, ldb, A, B);
}

cudaError_t launch_tc_cgemm(int M, int N, int K, const void *A, int lda_c, const float *B, int ldb, int epi,
                            const TcEpilogue &ep, int *err, cudaStream_t s)
{
    const bool cplx_out = epi == TC_EPI_CSTORE || epi == TC_EPI_CSTORE_T;
    return launch_tc3_gemm(M, cplx_out ? 2 * N : N, 2 * K, (const float *)A, 2 * lda_c, B, ldb, epi, ep, err, s);
}

}  // namespace sqm
