// FP32-accurate complex products C = alpha X^H Y + beta C on the BF16 tensor
// cores by exact slicing (the error-free splitting of Ozaki, Ogita, Oishi &
// Rump, Numer. Algorithms 59 (2012), cut to the FP32 significand).  These
// are the dense products of the reduced-precision two-stage reduction
// (paper, section "Performance of the Matrix Diagonalization Algorithm":
// the 2-stage solver's dense trailing updates and the stage-1
// back-transformation): the panel product A22 V, the rank-2b trailing
// update A22 -= V W^H + W V^H and the two products of the back-transform.
//
// Slicing.  X (K x M) and Y (K x N) are complex64, column j of each cut into
// chunks of 64 consecutive k.  Every (column, chunk) gets a power-of-two
// scale 2^e with max |Re|, |Im| < 2^e over the chunk, and each part x of an
// entry is written exactly as
//     x 2^-e = m_1 2^-8 + m_2 2^-16 + m_3 2^-24 + r,   |r| <= 2^-25,
// m_1 in [-256, 256], m_2, m_3 in [-128, 128] (repeated rounding, exact in
// FP32), so every m_s is exact in bf16 and the dropped remainder is below
// half an FP32 ulp of the chunk's largest entry.
//
// Products.  A product of two slices m_a n_b is an integer of magnitude at
// most 2^16.  Pairs (a, b) with the same level q = a + b (0-based slices,
// q = 0, 1, 2; higher levels are below 2^-24 of the leading term and are not
// formed) share one FP32 accumulator in tensor memory; per chunk a level
// sums at most 3 pairs x 64 k x (real, imaginary) = 384 products whose
// magnitudes add up to below 2^24, so the accumulation is exact whatever
// rounding the tensor core applies to partial sums.  After every chunk the
// epilogue warps read the three levels, combine them as
// L0 + 2^-8 L1 + 2^-16 L2 in FP32 (round to nearest) and add the chunk's
// contribution times 2^(e_x + e_y - 16) to FP32 registers.  The result is as
// accurate as an FP32 GEMM with no accumulation bias.
//
// Complex arithmetic (as in the FP64-accurate refinement products): per
// slice a of X, A = Re X_a meets the stack [Re Y_0; Im Y_0; Re Y_1; ...] and
// A = Im X_a meets [Im Y_0; -Re Y_0; ...], N = 2 NT (S - a) rows, so level q
// owns 2 NT accumulator columns [Re | Im] of the NT outputs of the tile.
//
// Kernel: persistent over 128 x 32 output tiles (one CTA per SM, tiles taken
// in a static round robin); warp 0 issues TMA loads, warp 1 the MMAs from
// one thread, warps 2..5 drain the accumulators.  Two accumulator buffers
// alternate between chunks, across tile boundaries, so that the epilogue of
// one chunk overlaps the MMAs of the next.  `lower` computes and writes only
// the tiles and entries with row >= column of a square C.
#include <cudaTypedefs.h>

#include <algorithm>

#include "internal.h"
#include "tc.cuh"

namespace bdg {

int tensor_map_bf16(bdg_ctx *ctx, CUtensorMap *m, const void *ptr, int64_t rows, int64_t kdim, int64_t ld,
                    int box_rows);

namespace xs {

constexpr int S = 3;                               // slices per operand
constexpr int NT = 32;                             // columns of C per tile
constexpr int LEVELS = S;                          // levels q = 0 .. S-1
constexpr int A_STAGES = 4;
constexpr int B_STAGES = 2;
constexpr int A_TILE = tc::BM * tc::BK * 2;        // 16 KB: one plane, 128 rows x 64 k
constexpr int A_STAGE = 2 * A_TILE;                // re + im of one slice
constexpr int B_TILE = NT * tc::BK * 2;            // 4 KB: one plane, 32 rows x 64 k
constexpr int B_STACK = 2 * S * B_TILE;            // one operand stack of 2S tiles
constexpr int B_STAGE = 2 * B_STACK;               // [Re, Im] and [Im, -Re] stacks
constexpr int BUF_COLS = 2 * LEVELS * NT;          // 192 accumulator columns per buffer
constexpr int NPLANES_A = 2 * S;                   // re, im slices
constexpr int NPLANES_B = 3 * S;                   // re, im, -re slices
constexpr int SMEM = A_STAGES * A_STAGE + B_STAGES * B_STAGE + 1024 + 256;
static_assert(SMEM <= 232448, "xs_kernel: shared memory above the 227 KB opt-in limit");
static_assert(tc::BM == 4 * NT, "xs_kernel: the lower-triangle tile map assumes 4 column tiles per row tile");

struct Params {
    CUtensorMap xa[NPLANES_A];      // X slices as the A operand, box 128 rows
    CUtensorMap yb[NPLANES_B];      // Y slices as the B operand, box 32 rows
    int M, N;                       // C is M x N
    int kblocks;                    // K padded to 64, / 64
    int lower;                      // only row >= column (square C)
    int ntm, ntn;                   // row and column tiles
    long long ntiles;
    const int *ex;                  // [kblocks][M] chunk exponents of X's columns
    const int *ey;                  // [kblocks][N] chunk exponents of Y's columns
    float2 *C;
    int64_t ldc;
    float alpha, beta;
    int *err;
    long long wait;                 // cap of every pipeline wait, SM clock cycles
};
static_assert(sizeof(Params) <= 4096, "xs_kernel: parameter block above 4 KB");

// Tile t -> (row tile, column tile).  Full: row-major over the tile grid.
// Lower: row tile r holds the column tiles c <= 4 r + 3 (at most ntn), so the
// tiles before row tile r number P(r) = 2 r^2 + 2 r (every row tile but the
// last has 4 r + 4 <= ntn when C is square).
__device__ __forceinline__ void tile_of(const Params &p, long long t, int &rb, int &cb) {
    if (!p.lower) {
        rb = (int)(t / p.ntn);
        cb = (int)(t % p.ntn);
        return;
    }
    long long r = (long long)((sqrt(1.0 + 2.0 * (double)t) - 1.0) * 0.5);
    while (2 * (r + 1) * (r + 1) + 2 * (r + 1) <= t) ++r;
    while (r > 0 && 2 * r * r + 2 * r > t) --r;
    if (r > p.ntm - 1) r = p.ntm - 1;
    rb = (int)r;
    cb = (int)(t - (2 * r * r + 2 * r));
}

__device__ __forceinline__ float pow2f(int k) {
    k = min(k, 127);
    return k >= -126 ? __int_as_float((k + 127) << 23) : 0.f;
}

__global__ void __launch_bounds__(192, 1) xs_kernel(const __grid_constant__ Params p) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *sA = base;
    unsigned char *sB = base + A_STAGES * A_STAGE;
    uint64_t *afull = (uint64_t *)(sB + B_STAGES * B_STAGE);
    uint64_t *aempty = afull + A_STAGES;
    uint64_t *bfull = aempty + A_STAGES;
    uint64_t *bempty = bfull + B_STAGES;
    uint64_t *accfull = bempty + B_STAGES;   // [2]
    uint64_t *accempty = accfull + 2;        // [2]
    uint64_t *donebar = accempty + 2;        // every MMA of this CTA has completed
    uint32_t *tslot = (uint32_t *)(donebar + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < A_STAGES; ++s) { tc::mbar_init(&afull[s], 1); tc::mbar_init(&aempty[s], 1); }
        for (int s = 0; s < B_STAGES; ++s) { tc::mbar_init(&bfull[s], 1); tc::mbar_init(&bempty[s], 1); }
        for (int s = 0; s < 2; ++s) { tc::mbar_init(&accfull[s], 1); tc::mbar_init(&accempty[s], 128); }
        tc::mbar_init(donebar, 1);
        tc::mbar_fence_init();
    }
    if (warp == 1) tc::tmem_alloc(tslot, 512);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tbase = *tslot;
    const int KB = p.kblocks;

    if (warp == 0 && lane == 0) {
        // ------------------------------------------------------------ producer
        for (int i = 0; i < NPLANES_A; ++i) tc::tma_prefetch_desc(&p.xa[i]);
        for (int i = 0; i < NPLANES_B; ++i) tc::tma_prefetch_desc(&p.yb[i]);
        int ia = 0, ib = 0;
        bool ok = true;
        for (long long t = blockIdx.x; t < p.ntiles && ok; t += gridDim.x) {
            int rb, cb;
            tile_of(p, t, rb, cb);
            const int m0 = rb * tc::BM, n0 = cb * NT;
            for (int kb = 0; kb < KB && ok; ++kb) {
                {
                    const int s = ib % B_STAGES;
                    const uint32_t ph = (ib / B_STAGES) & 1;
                    if (!tc::mbar_wait(&bempty[s], ph ^ 1, p.err, 31, p.wait)) { ok = false; break; }
                    unsigned char *dst = sB + s * B_STAGE;
                    tc::mbar_expect_tx(&bfull[s], B_STAGE);
                    for (int q = 0; q < S; ++q) {
                        // stack 1: Re Y_q, Im Y_q;  stack 2: Im Y_q, -Re Y_q
                        tc::tma_load_2d(dst + (2 * q) * B_TILE, &p.yb[q], kb * tc::BK, n0, &bfull[s]);
                        tc::tma_load_2d(dst + (2 * q + 1) * B_TILE, &p.yb[S + q], kb * tc::BK, n0, &bfull[s]);
                        tc::tma_load_2d(dst + B_STACK + (2 * q) * B_TILE, &p.yb[S + q], kb * tc::BK, n0, &bfull[s]);
                        tc::tma_load_2d(dst + B_STACK + (2 * q + 1) * B_TILE, &p.yb[2 * S + q], kb * tc::BK, n0,
                                        &bfull[s]);
                    }
                    ++ib;
                }
                for (int a = 0; a < S; ++a, ++ia) {
                    const int s = ia % A_STAGES;
                    const uint32_t ph = (ia / A_STAGES) & 1;
                    if (!tc::mbar_wait(&aempty[s], ph ^ 1, p.err, 32, p.wait)) { ok = false; break; }
                    unsigned char *dst = sA + s * A_STAGE;
                    tc::mbar_expect_tx(&afull[s], A_STAGE);
                    tc::tma_load_2d(dst, &p.xa[a], kb * tc::BK, m0, &afull[s]);
                    tc::tma_load_2d(dst + A_TILE, &p.xa[S + a], kb * tc::BK, m0, &afull[s]);
                }
            }
        }
        // every issued load must land before the CTA may exit
        for (int s = 0; s < A_STAGES && s < ia; ++s) {
            const int last = ia - 1 - ((ia - 1 - s) % A_STAGES);
            tc::mbar_drain(&afull[s], (last / A_STAGES) & 1, p.err, 33);
        }
        for (int s = 0; s < B_STAGES && s < ib; ++s) {
            const int last = ib - 1 - ((ib - 1 - s) % B_STAGES);
            tc::mbar_drain(&bfull[s], (last / B_STAGES) & 1, p.err, 34);
        }
    } else if (warp == 1 && lane == 0) {
        // ------------------------------------------------------------ MMA
        int ia = 0, cc = 0;
        bool ok = true;
        for (long long t = blockIdx.x; t < p.ntiles && ok; t += gridDim.x) {
            for (int kb = 0; kb < KB; ++kb, ++cc) {
                const int buf = cc & 1;
                const int use = cc >> 1;   // how many times this buffer was used before
                if (use > 0 && !tc::mbar_wait(&accempty[buf], (use - 1) & 1, p.err, 35, p.wait)) { ok = false; break; }
                tc::tc_fence_after();
                const int sbi = cc % B_STAGES;
                if (!tc::mbar_wait(&bfull[sbi], (cc / B_STAGES) & 1, p.err, 36, p.wait)) { ok = false; break; }
                unsigned char *bst = sB + sbi * B_STAGE;
                const uint64_t db1 = tc::smem_desc_k128(bst);             // [Re Y_b, Im Y_b] stack
                const uint64_t db2 = tc::smem_desc_k128(bst + B_STACK);   // [Im Y_b, -Re Y_b] stack
                const uint32_t acc0 = tbase + (uint32_t)(buf * BUF_COLS);
                for (int a = 0; a < S; ++a, ++ia) {
                    const int s = ia % A_STAGES;
                    if (!tc::mbar_wait(&afull[s], (ia / A_STAGES) & 1, p.err, 37, p.wait)) { ok = false; break; }
                    tc::tc_fence_after();
                    unsigned char *ast = sA + s * A_STAGE;
                    const uint64_t dar = tc::smem_desc_k128(ast), dai = tc::smem_desc_k128(ast + A_TILE);
                    const uint32_t id = tc::idesc_bf16(2 * NT * (S - a), false, false);   // levels a .. S-1
                    const uint32_t d = acc0 + (uint32_t)(a * 2 * NT);
#pragma unroll
                    for (int k = 0; k < tc::BK / tc::UMMA_K; ++k) {
                        const uint64_t o = (uint64_t)(2 * k);
                        const uint32_t first = (a == 0 && k == 0) ? 0u : 1u;
                        tc::mma_bf16(d, dar + o, db1 + o, id, first);   // [Re | Im] += Xr [Yr | Yi]
                        tc::mma_bf16(d, dai + o, db2 + o, id, 1u);      // [Re | Im] += Xi [Yi | -Yr]
                    }
                    tc::mma_commit(&aempty[s]);
                }
                if (!ok) break;
                tc::mma_commit(&bempty[sbi]);
                tc::mma_commit(&accfull[buf]);
            }
        }
        tc::mma_commit(donebar);
    } else if (warp >= 2) {
        // ------------------------------------------------------------ epilogue
        const int lb = 32 * (warp & 3);
        const int row = lb + lane;
        int cc = 0;
        bool ok = true;
        for (long long t = blockIdx.x; t < p.ntiles && ok; t += gridDim.x) {
            int rb, cb;
            tile_of(p, t, rb, cb);
            const int i = rb * tc::BM + row, n0 = cb * NT;
            float accr[NT], acci[NT];
#pragma unroll
            for (int j = 0; j < NT; ++j) { accr[j] = 0.f; acci[j] = 0.f; }
            for (int kb = 0; kb < KB; ++kb, ++cc) {
                const int buf = cc & 1, use = cc >> 1;
                // the row's scale exponent of this chunk, loaded before the wait
                const int er = (i < p.M) ? __ldg(p.ex + (int64_t)kb * p.M + i) : 0;
                if (!tc::mbar_wait(&accfull[buf], use & 1, p.err, 38, p.wait)) { ok = false; break; }
                tc::tc_fence_after();
                const uint32_t t0 = tbase + ((uint32_t)lb << 16) + (uint32_t)(buf * BUF_COLS);
                const int *eyc = p.ey + (int64_t)kb * p.N;
#pragma unroll
                for (int h = 0; h < NT; h += 16) {
                    // levels of columns h .. h+15: L0 + 2^-8 L1 + 2^-16 L2
                    float tr[16], ti[16], v[16];
                    tc::tmem_ld16(t0 + (uint32_t)h, tr);
                    tc::tmem_ld16(t0 + (uint32_t)(NT + h), ti);
#pragma unroll
                    for (int L = 1; L < LEVELS; ++L) {
                        const float sl = __int_as_float((127 - 8 * L) << 23);   // 2^-8L
                        tc::tmem_ld16(t0 + (uint32_t)(L * 2 * NT + h), v);
#pragma unroll
                        for (int j = 0; j < 16; ++j) tr[j] = fmaf(v[j], sl, tr[j]);
                        tc::tmem_ld16(t0 + (uint32_t)(L * 2 * NT + NT + h), v);
#pragma unroll
                        for (int j = 0; j < 16; ++j) ti[j] = fmaf(v[j], sl, ti[j]);
                    }
                    if (h + 16 == NT) {
                        // every level of this buffer has been read
                        tc::tc_fence_before();
                        tc::mbar_arrive(&accempty[buf]);
                    }
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int jj = n0 + h + j;
                        const float sc = pow2f(er + ((jj < p.N) ? __ldg(eyc + jj) : 0) - 16);
                        accr[h + j] = fmaf(tr[j], sc, accr[h + j]);
                        acci[h + j] = fmaf(ti[j], sc, acci[h + j]);
                    }
                }
            }
            if (!ok) break;
            if (i < p.M) {
                const float al = p.alpha, be = p.beta;
                float2 *crow = p.C + i;
#pragma unroll
                for (int h = 0; h < NT; h += 8) {
                    // eight columns at a time: loads first, then the stores
                    float2 q[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int jj = n0 + h + j;
                        q[j] = make_float2(0.f, 0.f);
                        if (be != 0.f && jj < p.N && (!p.lower || i >= jj)) q[j] = crow[(int64_t)jj * p.ldc];
                    }
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int jj = n0 + h + j;
                        if (jj >= p.N || (p.lower && i < jj)) continue;
                        float2 o = make_float2(al * accr[h + j], al * acci[h + j]);
                        if (be != 0.f) { o.x = fmaf(be, q[j].x, o.x); o.y = fmaf(be, q[j].y, o.y); }
                        crow[(int64_t)jj * p.ldc] = o;
                    }
                }
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        // no MMA may still write tensor memory when it is freed
        if (lane == 0) tc::mbar_drain(donebar, 0, p.err, 39);
        __syncwarp();
        tc::tc_fence_after();
        tc::tmem_dealloc(tbase, 512);
    }
}

// ---------------------------------------------------------------------------
// slicing: logical X (K x C, complex64) with element (k, c) at
// src[k sk + c sc]; one CTA per (64-chunk of k, 32 columns).  Planes: q =
// 0..S-1 real slices, S..2S-1 imaginary slices, 2S..3S-1 negated real slices
// (B operand only); element (k, c) of plane q at planes[q pstride + c kp + k].
// The padded tail k >= K is written as zeros; columns c >= C are not touched.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) slice_kernel(int64_t K, int64_t C, const float2 *__restrict__ src, int64_t sk,
                                                    int64_t sc, int conj_, int nplanes,
                                                    __nv_bfloat16 *__restrict__ planes, int64_t kp, int64_t pstride,
                                                    int *__restrict__ eout) {
    __shared__ float2 tile[32][65];
    const int kb = blockIdx.x;
    const int64_t k0 = (int64_t)kb * 64, c0 = (int64_t)blockIdx.y * 32;
    const int tid = threadIdx.x;
    for (int idx = tid; idx < 2048; idx += 256) {
        int k, c;
        if (sk == 1) { k = idx & 63; c = idx >> 6; }      // k contiguous
        else { c = idx & 31; k = idx >> 5; }              // c contiguous (or neither)
        const int64_t gk = k0 + k, gc = c0 + c;
        float2 v = make_float2(0.f, 0.f);
        if (gk < K && gc < C) v = src[gk * sk + gc * sc];
        if (conj_) v.y = -v.y;
        tile[c][k] = v;
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    for (int cc = warp; cc < 32; cc += 8) {
        const int64_t gc = c0 + cc;
        if (gc >= C) continue;
        const float2 v0 = tile[cc][2 * lane], v1 = tile[cc][2 * lane + 1];
        float m = fmaxf(fmaxf(fabsf(v0.x), fabsf(v0.y)), fmaxf(fabsf(v1.x), fabsf(v1.y)));
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        int e = 0;
        if (m > 0.f) frexpf(m, &e);          // m < 2^e
        if (e < -118) e = -118;              // chunks below 2^-118 contribute nothing at FP32 level
        const float s8 = __int_as_float((127 + 8 - e) << 23);   // 2^(8 - e)
        float xr0 = v0.x * s8, xi0 = v0.y * s8, xr1 = v1.x * s8, xi1 = v1.y * s8;   // |x| < 256
        const int64_t o = gc * kp + k0 + 2 * lane;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const float mr0 = rintf(xr0), mi0 = rintf(xi0), mr1 = rintf(xr1), mi1 = rintf(xi1);
            xr0 = (xr0 - mr0) * 256.f; xi0 = (xi0 - mi0) * 256.f;
            xr1 = (xr1 - mr1) * 256.f; xi1 = (xi1 - mi1) * 256.f;
            *(__nv_bfloat162 *)(planes + (int64_t)s * pstride + o) = __floats2bfloat162_rn(mr0, mr1);
            *(__nv_bfloat162 *)(planes + (int64_t)(S + s) * pstride + o) = __floats2bfloat162_rn(mi0, mi1);
            if (nplanes == NPLANES_B)
                *(__nv_bfloat162 *)(planes + (int64_t)(2 * S + s) * pstride + o) = __floats2bfloat162_rn(-mr0, -mr1);
        }
        if (lane == 0) eout[(int64_t)kb * C + gc] = e;
    }
}

}  // namespace xs

int64_t xs_kpad(int64_t K) { return (K + 63) / 64 * 64; }

// bytes of the planes of a K x C operand (A: 2S planes, B: 3S planes) and of its exponents
size_t xs_plane_bytes(int64_t K, int64_t C, bool bop) {
    return (size_t)(bop ? xs::NPLANES_B : xs::NPLANES_A) * (size_t)xs_kpad(K) * (size_t)C * 2;
}
size_t xs_exp_bytes(int64_t K, int64_t C) { return (size_t)(xs_kpad(K) / 64) * (size_t)C * 4; }

// Slice the logical K x C complex64 operand X (element (k, c) at src[k sk + c
// sc], conjugated when conj_) into exact bf16 planes and chunk exponents.
int xs_slice(bdg_ctx *ctx, cudaStream_t st, int64_t K, int64_t C, const float2 *src, int64_t sk, int64_t sc,
             bool conj_, bool bop, __nv_bfloat16 *planes, int *ex) {
    if (K <= 0 || C <= 0) return BDG_OK;
    const int64_t kp = xs_kpad(K);
    dim3 grid((unsigned)(kp / 64), (unsigned)((C + 31) / 32));
    if (grid.y > 65535) return bdg_fail(ctx, BDG_EUNSUPPORTED, "xs_slice: %lld columns", (long long)C);
    xs::slice_kernel<<<grid, 256, 0, st>>>(K, C, src, sk, sc, conj_ ? 1 : 0, bop ? xs::NPLANES_B : xs::NPLANES_A,
                                           planes, kp, kp * C, ex);
    BDG_LAUNCH_CHECK(ctx);
    return BDG_OK;
}

// C (M x N complex64, ldc) <- alpha X^H Y + beta C for sliced X (K x M, A
// planes) and Y (K x N, B planes); with `lower`, M == N and only the entries
// with row >= column are formed and written.
int xs_product(bdg_ctx *ctx, cudaStream_t st, int64_t K, int64_t M, int64_t N, const __nv_bfloat16 *px,
               const int *ex, const __nv_bfloat16 *py, const int *ey, float2 *C, int64_t ldc, float alpha,
               float beta, bool lower) {
    if (M <= 0 || N <= 0) return BDG_OK;
    if (lower && M != N) return bdg_fail(ctx, BDG_EINVAL, "xs_product: lower needs a square result");
    const int64_t kp = xs_kpad(K);
    xs::Params p;
    memset(&p, 0, sizeof(p));
    for (int q = 0; q < xs::NPLANES_A; ++q) {
        int rc = tensor_map_bf16(ctx, &p.xa[q], px + q * kp * M, M, kp, kp, tc::BM);
        if (rc) return rc;
    }
    for (int q = 0; q < xs::NPLANES_B; ++q) {
        int rc = tensor_map_bf16(ctx, &p.yb[q], py + q * kp * N, N, kp, kp, xs::NT);
        if (rc) return rc;
    }
    p.M = (int)M;
    p.N = (int)N;
    p.kblocks = (int)(kp / 64);
    p.lower = lower ? 1 : 0;
    p.ntm = (int)((M + tc::BM - 1) / tc::BM);
    p.ntn = (int)((N + xs::NT - 1) / xs::NT);
    if (lower) {
        const long long r = p.ntm - 1;
        p.ntiles = 2 * r * r + 2 * r + std::min<long long>(4 * (long long)p.ntm, p.ntn);
    } else {
        p.ntiles = (long long)p.ntm * p.ntn;
    }
    p.ex = ex;
    p.ey = ey;
    p.C = C;
    p.ldc = ldc;
    p.alpha = alpha;
    p.beta = beta;
    p.err = ctx->dflags + 6;
    p.wait = ctx->wait_cycles;
    BDG_CUDA_TRY(ctx, cudaFuncSetAttribute(xs::xs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, xs::SMEM));
    const unsigned grid = (unsigned)std::min<long long>(p.ntiles, (long long)ctx->num_sms);
    xs::xs_kernel<<<grid, 192, xs::SMEM, st>>>(p);
    BDG_LAUNCH_CHECK(ctx);
    return BDG_OK;
}

}  // namespace bdg
