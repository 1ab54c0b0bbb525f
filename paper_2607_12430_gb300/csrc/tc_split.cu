// tc_split.cu -- the FP64 residual of the SPD refinement (Algorithm 3,
// steps 4-5), R = (A - X X) 4^-e for symmetric X, with the product X X
// formed on the BF16 tensor cores by error-free splitting (the scheme of
// Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59 (2012)).
//
// Splitting.  Row i of X (= column i) is scaled by 2^-rho_i, the smallest
// power of two above its largest magnitude, and cut into S balanced digits
// of b bits, each rounded to nearest:
//   X(i, k) = 2^rho_i sum_s m_s(i, k) 2^(-b (s + 1)) + r(i, k),
//   m_s integers with |m_s| <= 2^b,  |r(i, k)| <= 2^(rho_i - b S - 1).
// Rounding (not truncation toward zero) leaves remainders of either sign,
// so the left-out parts of a length-n sum do not all pull one way.  Each
// m_s is exact in BF16 (b <= 8).  A product of two digit matrices,
//   P_st(i, j) = sum_k m_s(i, k) m_t(j, k),
// is a sum of n integers of magnitude <= 2^(2b); with n 2^(2b) <= 2^24 every
// partial sum is an integer of at most 24 bits, so the tensor core's FP32
// accumulation is exact whatever its internal order or rounding.  Then
//   (X X)(i, j) = 2^(rho_i + rho_j) sum_{s,t} 2^(-b (s + t + 2)) P_st(i, j)
// up to the terms left out: digits beyond S and pairs with s + t > D.  With
// b (D + 1) >= 56 + log2(D + 2) and S = D + 1 their sum is below
// n 2^(rho_i + rho_j - 56), within the FP64 product's own error bound
// n u sum_k |X(i,k)| |X(k,j)| for u = 2^-53 when one term dominates, and
// far below it otherwise.  The P_st are scaled exactly (powers of two) and
// summed in FP64.
//
// Products.  Pairs with the same s + t carry the same power of two, so
// several of them can share one FP32 accumulator as long as the bounds of
// their integer sums add up to at most 2^24 (|m_0| <= 2^b, |m_s| <= 2^(b-1)
// for s >= 1, so |P_st| <= n 2^b_s 2^b_t): the accumulation stays exact
// and the FP64 epilogue -- which costs as much as the tensor-core work on a
// part with few FP64 units -- runs once per group instead of once per pair.
// One persistent launch per residual: a CTA per SM loops over 128 x 128
// output tiles of the upper block triangle only (R is symmetric) and, for
// each tile, over every group in turn, with warp roles: warp 0 issues the
// TMA loads of both digit tiles (128 rows x 128 bytes, 128-byte swizzle,
// from one map over all digit slices) into a 6-stage ring, K in steps of 64
// BF16 values over each pair of the group; warp 1 issues 4 tcgen05.mma
// (M = N = 128, K = 16) per stage into one of two 128-column TMEM
// accumulators; warps 2-5 run the FP64 epilogue of the previous group (its
// scaled tile added into the tile's FP64 accumulator, which stays in L2
// while the CTA is on the tile; the first group starts it from A, the last
// one writes Rhat = fl32(R 4^-e), mirrored, and per-warp partial sums of
// |R|^2) while the next group's products go to the other accumulator.
// Every mbarrier wait is bounded (status 6 on timeout) and ends early once
// another role has given up.
#include <cuda_bf16.h>

#include <algorithm>

#include "internal.h"
#include "spd_internal.h"
#include "tc_common.cuh"

namespace sqm {

// output tiles of (128 MH) x 128: with MH = 2 two M = 128 MMAs share the B
// tile (a quarter less operand traffic per flop), used where there are at
// least as many such tiles as SMs; TMA boxes of 128 rows; 192 KB of stages
static constexpr int SP_BR = 128, SP_BN = 128, SP_BK = 64;
template <int MH> struct SpCfg {
    static constexpr int BM = SP_BR * MH, STAGES = MH == 1 ? 6 : 4;
};
static constexpr int SP_THREADS = 192;  // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
static constexpr int SP_TILE_BYTES = SP_BR * SP_BK * 2;  // 16 KB: one box
static constexpr int SP_SMEM = 6 * 2 * SP_TILE_BYTES + 1024 + 256;  // = 4 stages of 3 boxes

// digit width b and pair bound D for an inner dimension n (see above)
void split_plan(int n, int *b, int *D)
{
    int lg = 0;
    while ((1 << lg) < std::max(n, 1)) ++lg;
    int bb = std::max(1, std::min(8, (24 - lg) / 2));
    int dd = 0;
    while (bb * (dd + 1) < 56 + 4) ++dd;  // log2(D + 2) <= 4 for D <= 14
    *b = bb;
    *D = dd;
}

// One warp per row i of X (X symmetric: row i is column i, contiguous).
// Every step of the digit loop
//   t = x 2^b,  m_s = round-half-even(t),  x <- t - m_s
// is exact in FP64, so the digits depend only on the exact value of x; they
// are formed here from that value as a 128-bit fixed-point integer
// X = x 2^124 (exact for every x the digits can see) with integer
// operations -- the same digits, without the ~30 FP64 instructions an entry
// that the FP64 loop costs on a part with few FP64 units:
//   m_s = round-half-even(X / 2^(124 - b (s + 1))),  X -= m_s 2^(124 - b (s + 1)).
// An entry with |x| <= 2^-(b S + 1) has no nonzero digit.
// (b, S compile-time: every shift below is a constant and the digit loop
// unrolls; a run-time shift of a 128-bit value costs tens of instructions)
template <int b, int S>
__global__ void __launch_bounds__(256) split_rows_kernel(const double *__restrict__ X, int64_t ldx, int n, int lds,
                                                         __nv_bfloat16 *__restrict__ Xs, int *__restrict__ rho)
{
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;  // whole warps
    const double *col = X + (int64_t)i * ldx;
    // rho_i: the smallest r with max |x_ik| < 2^r (frexp's exponent), from the bits
    unsigned long long mx = 0;
    for (int k = lane; k < n; k += 32)
        mx = max(mx, (unsigned long long)__double_as_longlong(col[k]) & 0x7FFFFFFFFFFFFFFFull);
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, m));
    int r = 0;
    if (mx != 0) {
        const int ef = (int)(mx >> 52);
        r = ef > 0 ? ef - 1022 : 64 - __clzll((long long)mx) - 1074;
    }
    if (lane == 0) rho[i] = r;
    for (int k = lane; k < lds; k += 32) {
        const long long vb = k < n ? __double_as_longlong(col[k]) : 0ll;
        const int ef = (int)((vb >> 52) & 0x7FF);
        const long long mant = (vb & 0x000FFFFFFFFFFFFFll) | (ef ? (1ll << 52) : 0ll);
        // |v| = mant 2^(e2), e2 = max(ef, 1) - 1075; x 2^124 = mant 2^(e2 + 124 - r)
        const int sh = (ef ? ef : 1) - 1075 + 124 - r;
        // |x| <= 2^-(b S + 1), i.e. mant 2^sh <= 2^(123 - b S): no digit
        const bool zero = mant == 0 || sh < 0 || (sh + (63 - __clzll(mant)) < 123 - b * S) ||
                          (sh + (63 - __clzll(mant)) == 123 - b * S && (mant & (mant - 1)) == 0);
        __int128 rem = zero ? (__int128)0 : ((__int128)mant << sh);
        if (vb < 0) rem = -rem;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int shift = 124 - b * (s + 1);
            __int128 q = rem >> shift;  // floor
            const __int128 frac = rem - (q << shift), half = (__int128)1 << (shift - 1);
            if (frac > half || (frac == half && (q & 1))) q += 1;
            rem -= q << shift;
            Xs[((int64_t)s * n + i) * lds + k] = __float2bfloat16_rn((float)(int)q);  // |m| <= 2^b: exact
        }
    }
}

static constexpr int SP_MAXG = 16;  // pairs per group

static constexpr int SP_MAXP = SP_MAXG * (SP_MAXG + 1) / 2;  // pairs s + t <= D < SP_MAXG

// the digit pairs of a residual, grouped: group q holds pairs
// gstart[q] .. gstart[q+1]-1 (all with the same s + t) and its products carry
// the power of two 2^-shift[q]
struct SplitPlan {
    int ng;
    unsigned char ps[SP_MAXP], pt[SP_MAXP];
    short gstart[SP_MAXP + 1];
    short shift[SP_MAXP];
};

struct SplitEpi {
    const double *A;
    int64_t lda;
    double *Racc;
    int64_t ldr;
    const int *rho;   // scaling exponents of the left operand's rows
    const int *rhoB;  // of the right operand's rows (the same array for X X^T)
    float *Rhat;
    int64_t ldh;
    double sc;      // 4^-e
    double *partials;
};

// bounded mbarrier wait that also ends once another role has failed (the
// role that times out raises the flag)
__device__ __forceinline__ bool sp_wait(uint64_t *bar, uint32_t parity, volatile int *fail)
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

// 2^e as a double (exact in the normal range)
__device__ __forceinline__ double sp_pow2(int e)
{
    return (e >= -1022 && e <= 1023) ? __longlong_as_double((long long)(e + 1023) << 52) : ldexp(1.0, e);
}

// GEN = false: R = A - X X for symmetric X, both operands the digit slices of
// X (mapX), output tiles of the upper block triangle, R mirrored.  GEN = true:
// R = A - X Y^T for the row digits of X (mapX, exponents ep.rho) and of Y
// (mapB, ep.rhoB) -- with Y = X^T the residual of a general X -- over every
// output tile (T column blocks per row block, row-major).
template <int SP_MH, bool GEN>
__global__ void __launch_bounds__(SP_THREADS, 1)
split_gemm_kernel(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapB,
                  const __grid_constant__ SplitPlan plan, int n, int KT, int T, int ntiles, SplitEpi ep, int *err)
{
    constexpr int SP_BM = SpCfg<SP_MH>::BM, SP_STAGES = SpCfg<SP_MH>::STAGES;
    constexpr int SP_STAGE_BYTES = (SP_MH + 1) * SP_TILE_BYTES;  // the A boxes, then B
    constexpr int SP_TMEM_COLS = 2 * SP_MH * SP_BN;              // two accumulators of SP_MH halves
    extern __shared__ unsigned char smraw[];
    __shared__ volatile int s_fail;
    __shared__ int s_issued, s_consumed, s_committed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char *base = (unsigned char *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(base + SP_STAGES * SP_STAGE_BYTES);
    uint64_t *empty = full + SP_STAGES;
    uint64_t *accf = empty + SP_STAGES;  // accumulator a holds a finished group of a tile
    uint64_t *acce = accf + 2;           // accumulator a is free again
    uint32_t *tmem_slot = (uint32_t *)(acce + 2);
    if (tid == 0) {
        for (int s = 0; s < SP_STAGES; ++s) {
            mbar_init(&full[s], 1);
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
                     "r"(SP_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    auto stage_ptr = [&](int s, int which) { return base + s * SP_STAGE_BYTES + which * SP_TILE_BYTES; };
    // tiles meeting the upper triangle: row block I (128 MH rows), column
    // blocks J >= MH I (128 columns; T of them), row-major over I
    auto tile_origin = [&](int q, int &m0, int &n0) {
        if (GEN) {
            m0 = (q / T) * SP_BM;
            n0 = (q % T) * SP_BN;
            return;
        }
        int I = 0;
        while (q >= T - SP_MH * I) { q -= T - SP_MH * I; ++I; }
        m0 = I * SP_BM;
        n0 = (SP_MH * I + q) * SP_BN;
    };
    const int ng = plan.ng;
    if (warp == 0) {
        if (lane == 0) {
            // step t of a group: its pair gstart + t / KT, K block t % KT;
            // digit slice q starts at row q n of the map (rows past n of a
            // tile read the next slice or the zero fill; they only reach
            // output rows / columns >= n, never stored)
            int it = 0;
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
                int m0, n0;
                tile_origin(tile, m0, n0);
                for (int q = 0; ok && q < ng; ++q) {
                    const int p0 = plan.gstart[q], steps = KT * (plan.gstart[q + 1] - p0);
                    for (int t = 0; t < steps; ++t) {
                        const int s = it % SP_STAGES, u = it / SP_STAGES;
                        if (u > 0 && !sp_wait(&empty[s], (u - 1) & 1, &s_fail)) { ok = false; break; }
                        const int pr = p0 + t / KT, kb = t % KT;
                        mbar_arrive_expect_tx(&full[s], (SP_MH + 1) * SP_TILE_BYTES);
#pragma unroll
                        for (int h = 0; h < SP_MH; ++h)
                            tma_load_2d(stage_ptr(s, h), &mapX, &full[s], kb * SP_BK, plan.ps[pr] * n + m0 + h * SP_BR);
                        tma_load_2d(stage_ptr(s, SP_MH), GEN ? &mapB : &mapX, &full[s], kb * SP_BK, plan.pt[pr] * n + n0);
                        ++it;
                    }
                }
            }
            s_issued = it;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t IDESC = idesc_bf16_128x128();
            int it = 0, lt = 0, consumed = 0, committed = 0;
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
                for (int q = 0; ok && q < ng; ++q, ++lt) {
                    const int a = lt & 1, v = lt >> 1;
                    if (v > 0 && !sp_wait(&acce[a], (v - 1) & 1, &s_fail)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(a * SP_MH * SP_BN);
                    const int steps = KT * (plan.gstart[q + 1] - plan.gstart[q]);
                    for (int t = 0; t < steps; ++t, ++it) {
                        const int s = it % SP_STAGES;
                        if (!sp_wait(&full[s], (it / SP_STAGES) & 1, &s_fail)) { ok = false; break; }
                        consumed = it + 1;
                        tc_fence_after();
                        const uint32_t b0 = smem_u32(stage_ptr(s, SP_MH));
#pragma unroll
                        for (int h = 0; h < SP_MH; ++h) {
                            const uint32_t a0 = smem_u32(stage_ptr(s, h));
#pragma unroll
                            for (int kk = 0; kk < SP_BK / 16; ++kk) {
                                const uint32_t off = kk * 32;  // 16 BF16 values = 32 bytes along K
                                mma_bf16(d + (uint32_t)(h * SP_BN), smem_desc_sw128(a0 + off), smem_desc_sw128(b0 + off),
                                         IDESC, (t > 0 || kk > 0) ? 1u : 0u);
                            }
                        }
                        mma_commit(&empty[s]);  // the stage is free once these products are done
                        committed = it + 1;
                    }
                    if (ok) mma_commit(&accf[a]);
                }
            }
            s_consumed = consumed;
            s_committed = committed;
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, i.e. tile rows
        const int qw = warp & 3;
        int lt = 0;
        bool ok = true;
        for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
            int m0, n0;
            tile_origin(tile, m0, n0);
            int rho_h[SP_MH];
#pragma unroll
            for (int h = 0; h < SP_MH; ++h) {
                const int row = m0 + h * SP_BR + 32 * qw + lane;
                rho_h[h] = row < n ? ep.rho[row] : 0;
            }
            for (int q = 0; q < ng; ++q, ++lt) {
                const int a = lt & 1, v = lt >> 1;
                const bool first = q == 0, last = q == ng - 1;
                // every lane waits; the warp leaves together if any lane gave
                // up (the TMEM loads below are warp-collective)
                const bool okw = sp_wait(&accf[a], v & 1, &s_fail);
                if (!__all_sync(0xffffffffu, okw)) { ok = false; break; }
                tc_fence_after();
                const int shift = plan.shift[q];
                double ss = 0.0;
                for (int h = 0; h < SP_MH; ++h) {
                    const int row = m0 + h * SP_BR + 32 * qw + lane;
                    const int rho_i = rho_h[h];
                    for (int c0 = 0; c0 < SP_BN; c0 += 32) {
                        uint32_t r[32];
                        tmem_ld32(tmem + ((uint32_t)(32 * qw) << 16) + (uint32_t)((a * SP_MH + h) * SP_BN + c0), r);
                        if (row < n) {
                            // all loads of the chunk first: the stores below go
                            // to the same arrays, so loads issued after them
                            // would each wait out a full memory round trip
                            double old[32];
                            int rj[32];
#pragma unroll
                            for (int j = 0; j < 32; ++j) {
                                const int col = n0 + c0 + j;
                                const bool in = col < n && (GEN || row <= col);
                                old[j] = in ? (first ? ep.A[row + (int64_t)col * ep.lda]
                                                     : ep.Racc[row + (int64_t)col * ep.ldr])
                                            : 0.0;
                                rj[j] = col < n ? (GEN ? ep.rhoB[col] : ep.rho[col]) : 0;
                            }
#pragma unroll
                            for (int j = 0; j < 32; ++j) {
                                const int col = n0 + c0 + j;
                                if (col >= n || (!GEN && row > col)) continue;
                                // old - P 2^(rho_i + rho_j - shift): the product
                                // is exact, so one rounding as in old - ldexp(P, ...)
                                const double v2 =
                                    fma(-(double)__uint_as_float(r[j]), sp_pow2(rho_i + rj[j] - shift), old[j]);
                                if (last) {
                                    const double rs = v2 * ep.sc;
                                    const float rf = (float)rs;
                                    ep.Rhat[row + (int64_t)col * ep.ldh] = rf;
                                    if (!GEN) ep.Rhat[col + (int64_t)row * ep.ldh] = rf;
                                    ss = fma(rs, rs, ss);
                                    if (!GEN && row != col) ss = fma(rs, rs, ss);  // mirrored entry
                                } else {
                                    ep.Racc[row + (int64_t)col * ep.ldr] = v2;
                                }
                            }
                        }
                    }
                }
                tc_fence_before();
                mbar_arrive(&acce[a]);
                if (last) {
#pragma unroll
                    for (int m = 16; m > 0; m >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, m);
                    if (lane == 0) ep.partials[4 * tile + qw] = ss;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (s_fail) {
        // wait (bounded) for the loads and products still in flight before
        // the shared memory and TMEM are released
        if (tid == 0) {
            atomicExch(err, 6);
            for (int t = s_consumed; t < s_issued; ++t) mbar_wait(&full[t % SP_STAGES], (t / SP_STAGES) & 1);
            if (s_committed > 0) mbar_wait(&empty[(s_committed - 1) % SP_STAGES], ((s_committed - 1) / SP_STAGES) & 1);
        }
        __syncthreads();
    }
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(SP_TMEM_COLS) : "memory");
}

static bool make_bf16_map(CUtensorMap *m, const void *ptr, int64_t kdim, int64_t rows, int64_t ld)
{
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)kdim, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {SP_BK, SP_BR};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

int split_lds(int n) { return (int)cdiv_i(std::max(n, 1), SP_BK) * SP_BK; }

size_t split_digit_elems(int n)
{
    int b, D;
    split_plan(n, &b, &D);
    return (size_t)(D + 1) * (size_t)n * (size_t)split_lds(n);
}

bool split_residual_supported(int n)
{
    int b, D;
    split_plan(n, &b, &D);
    return n >= 1 && (int64_t)n * (1 << (2 * b)) <= (1 << 24) && encode_fn() != nullptr;
}

// digit slices of the rows i of X (column i in storage: X(k, i) for k < n);
// the (b, S) pairs split_plan can give: S = ceil(60 / b) digits of b bits
static cudaError_t launch_split_rows(const double *X, int64_t ldx, int n, int lds, __nv_bfloat16 *Xs, int *rho,
                                     int b, int S, cudaStream_t s)
{
    const unsigned g = (unsigned)cdiv_i((int64_t)n * 32, 256);
    if (b == 8 && S == 8) split_rows_kernel<8, 8><<<g, 256, 0, s>>>(X, ldx, n, lds, Xs, rho);
    else if (b == 7 && S == 9) split_rows_kernel<7, 9><<<g, 256, 0, s>>>(X, ldx, n, lds, Xs, rho);
    else if (b == 6 && S == 10) split_rows_kernel<6, 10><<<g, 256, 0, s>>>(X, ldx, n, lds, Xs, rho);
    else if (b == 5 && S == 12) split_rows_kernel<5, 12><<<g, 256, 0, s>>>(X, ldx, n, lds, Xs, rho);
    else if (b == 4 && S == 15) split_rows_kernel<4, 15><<<g, 256, 0, s>>>(X, ldx, n, lds, Xs, rho);
    else return cudaErrorInvalidValue;
    count_launch();
    return cudaGetLastError();
}

// groups of digit pairs with the same s + t whose integer bounds sum to <= 2^24
static SplitPlan make_split_plan(int n, int b, int D)
{
    SplitPlan plan{};
    int np = 0;
    for (int d = 0; d <= D; ++d) {
        double used = 0.0;
        bool open = false;
        for (int si = 0; si <= d; ++si) {
            const int ti = d - si;
            const double pb = (double)n * ldexp(1.0, si == 0 ? b : b - 1) * ldexp(1.0, ti == 0 ? b : b - 1);
            if (!open || used + pb > 16777216.0 || np - plan.gstart[plan.ng - 1] == SP_MAXG) {
                plan.gstart[plan.ng] = (short)np;
                plan.shift[plan.ng] = (short)(b * (d + 2));
                ++plan.ng;
                used = 0.0;
                open = true;
            }
            plan.ps[np] = (unsigned char)si;
            plan.pt[np] = (unsigned char)ti;
            ++np;
            used += pb;
        }
    }
    plan.gstart[plan.ng] = (short)np;
    return plan;
}

static int sm_count()
{
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

cudaError_t launch_residual_sym_split(const double *A, int64_t lda, const double *X, int64_t ldx, int n, int e,
                                      float *Rhat, int ldr, double *Racc, void *digits, int *rho,
                                      double *partials, int *nparts, int *err, cudaStream_t s)
{
    if (n <= 0) { *nparts = 0; return cudaSuccess; }
    int b, D;
    split_plan(n, &b, &D);
    const int S = D + 1, lds = split_lds(n);
    if (S > SP_MAXG) return cudaErrorInvalidValue;
    __nv_bfloat16 *Xs = (__nv_bfloat16 *)digits;
    cudaError_t er;
    if ((er = launch_split_rows(X, ldx, n, lds, Xs, rho, b, S, s))) return er;
    CUtensorMap mapX;
    if (!make_bf16_map(&mapX, Xs, lds, (int64_t)S * n, lds)) return cudaErrorInvalidValue;
    // T column blocks of 128; row block I (128 MH rows) meets the upper
    // triangle in column blocks MH I .. T-1
    const int T = (int)cdiv_i(n, SP_BN), KT = lds / SP_BK;
    const int sms = sm_count();
    int ntiles2 = 0;
    for (int I = 0; 2 * I < T; ++I) ntiles2 += T - 2 * I;
    const int mh = ntiles2 >= sms ? 2 : 1;
    const int ntiles = mh == 2 ? ntiles2 : T * (T + 1) / 2;
    if ((er = allow_max_smem((const void *)split_gemm_kernel<1, false>)) ||
        (er = allow_max_smem((const void *)split_gemm_kernel<2, false>)))
        return er;
    const SplitPlan plan = make_split_plan(n, b, D);
    const int grid = std::max(1, std::min(ntiles, sms));
    SplitEpi ep{A, lda, Racc, (int64_t)n, rho, rho, Rhat, (int64_t)ldr, ldexp(1.0, -2 * e), partials};
    if (mh == 2) split_gemm_kernel<2, false><<<grid, SP_THREADS, SP_SMEM, s>>>(mapX, mapX, plan, n, KT, T, ntiles, ep, err);
    else split_gemm_kernel<1, false><<<grid, SP_THREADS, SP_SMEM, s>>>(mapX, mapX, plan, n, KT, T, ntiles, ep, err);
    count_launch();
    *nparts = 4 * ntiles;  // a partial sum per epilogue warp and tile
    return cudaGetLastError();
}

// X^T of an n x n FP64 matrix into XT (ld n), 32 x 32 tiles through shared memory
__global__ void __launch_bounds__(256) transpose_f64_kernel(const double *__restrict__ X, int64_t ldx, int n,
                                                           double *__restrict__ XT)
{
    __shared__ double t[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < 32; r += 8) {
        const int i = bx + tx, j = by + r;
        t[r][tx] = (i < n && j < n) ? X[i + (int64_t)j * ldx] : 0.0;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int i = by + tx, j = bx + r;  // XT(i, j) = X(j, i)
        if (i < n && j < n) XT[i + (int64_t)j * n] = t[tx][r];
    }
}

int residual_gen_split_parts(int n)
{
    if (n <= 0) return 0;
    const int T = (int)cdiv_i(n, SP_BN);
    const int mh = (int)cdiv_i(n, 2 * SP_BR) * T >= sm_count() ? 2 : 1;
    return 4 * (int)cdiv_i(n, mh * SP_BR) * T;
}

cudaError_t launch_residual_gen_split(const double *A, int64_t lda, const double *X, int64_t ldx, int n, int e,
                                      float *Rhat, int ldr, double *Racc, double *XT, void *digitsA, void *digitsB,
                                      int *rhoA, int *rhoB, double *partials, int *nparts, int *err, cudaStream_t s)
{
    if (n <= 0) { *nparts = 0; return cudaSuccess; }
    int b, D;
    split_plan(n, &b, &D);
    const int S = D + 1, lds = split_lds(n);
    if (S > SP_MAXG) return cudaErrorInvalidValue;
    cudaError_t er;
    // left operand: the rows of X (columns of X^T); right operand: the
    // columns of X, so that (X X)(i, j) = sum_k X(i, k) X(k, j) pairs row i
    // of the one with row j of the other
    transpose_f64_kernel<<<dim3((unsigned)cdiv_i(n, 32), (unsigned)cdiv_i(n, 32)), 256, 0, s>>>(X, ldx, n, XT);
    count_launch();
    __nv_bfloat16 *Xa = (__nv_bfloat16 *)digitsA, *Xb = (__nv_bfloat16 *)digitsB;
    if ((er = launch_split_rows(XT, n, n, lds, Xa, rhoA, b, S, s))) return er;
    if ((er = launch_split_rows(X, ldx, n, lds, Xb, rhoB, b, S, s))) return er;
    CUtensorMap mapA, mapB;
    if (!make_bf16_map(&mapA, Xa, lds, (int64_t)S * n, lds) || !make_bf16_map(&mapB, Xb, lds, (int64_t)S * n, lds))
        return cudaErrorInvalidValue;
    const int T = (int)cdiv_i(n, SP_BN), KT = lds / SP_BK;
    const int sms = sm_count();
    const int mh = (int)cdiv_i(n, 2 * SP_BR) * T >= sms ? 2 : 1;
    const int ntiles = (int)cdiv_i(n, mh * SP_BR) * T;
    if ((er = allow_max_smem((const void *)split_gemm_kernel<1, true>)) ||
        (er = allow_max_smem((const void *)split_gemm_kernel<2, true>)))
        return er;
    const SplitPlan plan = make_split_plan(n, b, D);
    const int grid = std::max(1, std::min(ntiles, sms));
    SplitEpi ep{A, lda, Racc, (int64_t)n, rhoA, rhoB, Rhat, (int64_t)ldr, ldexp(1.0, -2 * e), partials};
    if (mh == 2) split_gemm_kernel<2, true><<<grid, SP_THREADS, SP_SMEM, s>>>(mapA, mapB, plan, n, KT, T, ntiles, ep, err);
    else split_gemm_kernel<1, true><<<grid, SP_THREADS, SP_SMEM, s>>>(mapA, mapB, plan, n, KT, T, ntiles, ep, err);
    count_launch();
    *nparts = 4 * ntiles;
    return cudaGetLastError();
}

}  // namespace sqm
