// FP64-accurate complex products C = X^H Y on the BF16 tensor cores by
// error-free slicing (the Ozaki scheme: Ozaki, Ogita, Oishi & Rump,
// "Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication and its applications", Numer.
// Algorithms 59 (2012)), used for G = X^H X and S = X^H (H X) of the
// Ogita-Aishima refinement.
//
// Slicing.  Every column j of X (and of Y) gets a power-of-two scale 2^e_j
// with max_k max(|Re X_kj|, |Im X_kj|) < 2^e_j, and
//     X_kj 2^-e_j = sum_{s=1..S} m_s 2^(-8 s),   m_s integer, |m_s| <= 256,
// obtained by repeated rounding (exact in FP64).  Each m_s is exact in bf16.
// Products m_a m_b are integers of magnitude <= 2^16 (<= 2^15 unless both
// are leading slices, <= 2^14 when neither is); a level holds at most S = 6
// pairs, so summed over a chunk of 64 values of k and over the (real,
// imaginary) pair of each output part they stay within 2^24 and the FP32
// accumulation in tensor memory is exact within a chunk.  Pairs (a, b) with
// the same level q = a + b share one accumulator;
// levels 2 .. S+1 are kept (the dropped levels are below 2^(-8(S+1)) of
// the leading term).  After every chunk the epilogue warps read the levels,
// scale level q by 2^(-8(q-2)) (exact) and add them to a double-FP32
// (hi + lo) accumulator.
//
// Tile: 128 rows of C (columns i of X) x NT columns of C (columns j of Y),
// NT = 32, 24, 16 for S = 4, 5, 6 slices.
// Per slice a of X two MMAs cover all levels a+b (b = 0 .. S-1-a) and both
// parts of the complex product: A = Re X_a against the stack
// [Re Y_0, Im Y_0, Re Y_1, Im Y_1, ...] and A = Im X_a against
// [Im Y_0, -Re Y_0, Im Y_1, -Re Y_1, ...] (N = 2 NT (S-a)), so that level q
// owns 2 NT consecutive accumulator columns: [Re | Im] of the NT outputs.
// Negated real slices are stored as planes of their own; the X^T variant
// negates the A operand of the second MMA instead.  Two accumulator
// buffers (S levels x 2 NT columns each) alternate between chunks so that the
// epilogue of chunk c overlaps the MMAs of chunk c+1.
// Only tiles that touch the upper triangle (j >= i) are computed when
// `upper` is set (G and S are Hermitian).
//
// Layout of the contraction index.  The rows of a BdG vector are the u half
// (sites 0 .. V-1) and the v half (V .. 2V-1); the planes store them in a
// K axis of length 2 Vp (Vp = V rounded up to 64): u rows at 0 .. V-1, v rows
// at Vp .. Vp+V-1, zeros elsewhere.  Each 64-wide K chunk then lies in one
// half, which gives two variants at no cost:
//   trans_a: C = X^T Y instead of X^H Y (signs of the Im X terms flip);
//   cswap_b: Y is replaced by C Y with C = [[0, I], [-I, 0]] (the
//            particle-hole partner map without its conjugation): chunk kb
//            reads the chunk of the other half, negated when kb is in the
//            v half.
#include <cudaTypedefs.h>

#include <mutex>

#include "internal.h"
#include "tc.cuh"

namespace bdg {

namespace oz {

constexpr int SMAX = 6;          // slices per operand in the planes; a product may use the first S <= SMAX
constexpr int A_TILE = tc::BM * tc::BK * 2;        // 16 KB (one plane)
constexpr int A_STAGE = 2 * A_TILE;                // re + im of one slice
constexpr int B_STAGES = 2;
constexpr int NPLANES_B = 3 * SMAX;                // Re, Im, -Re slices

// Tile width and pipeline depth by slice count.  The A tiles (128 rows of X,
// S slices) are re-read for every column tile, so the tile is as wide as two
// accumulator buffers of S levels x 2 NT columns allow in the 512 columns of
// tensor memory: NT = 32, 24, 16 for S = 4, 5, 6.
template <int S> struct Cfg;
// EPI drain warps: 4 (one per 32-lane quadrant of tensor memory) or 8 (two per
// quadrant, each taking half of the tile's columns, which halves the
// double-FP32 accumulators a thread holds).
template <> struct Cfg<4> { static constexpr int NT = 32, A_STAGES = 3, EPI = 8; };
template <> struct Cfg<5> { static constexpr int NT = 24, A_STAGES = 3, EPI = 4; };
template <> struct Cfg<6> { static constexpr int NT = 16, A_STAGES = 4, EPI = 4; };
template <int S> struct Geom {
    static constexpr int NT = Cfg<S>::NT;
    static constexpr int A_STAGES = Cfg<S>::A_STAGES;
    static constexpr int EPI = Cfg<S>::EPI;
    static constexpr int THREADS = 64 + 32 * EPI;            // producer warp, MMA warp, drain warps
    static constexpr int NTE = NT * 4 / EPI;                 // columns per drain thread
    static_assert(NTE % 8 == 0, "ozaki_kernel: columns per drain thread must be a multiple of 8");
    static constexpr int B_TILE = NT * tc::BK * 2;           // one slice, one plane
    static constexpr int B_STACK = 2 * S * B_TILE;           // [Re Y_0, Im Y_0, Re Y_1, ...]
    static constexpr int B_STAGE = 2 * B_STACK;              // and [Im Y_0, -Re Y_0, ...]
    static constexpr int BUF_COLS = 2 * S * NT;              // one accumulator buffer: S levels x [Re | Im]
    static constexpr int SMEM = A_STAGES * A_STAGE + B_STAGES * B_STAGE + 1024 + 256;
    static_assert(SMEM <= 232448, "ozaki_kernel: shared memory above the 227 KB opt-in limit");
    static_assert(2 * BUF_COLS <= 512, "ozaki_kernel: two accumulator buffers above 512 TMEM columns");
    static_assert(2 * NT * S <= 256 && (2 * NT * S) % 16 == 0, "ozaki_kernel: MMA N out of range");
    static_assert(B_TILE % 1024 == 0, "ozaki_kernel: B tiles must keep the 1024-byte swizzle alignment");
};

inline int tile_width(int slices) { return slices == 4 ? 32 : slices == 5 ? 24 : 16; }

struct Params {
    CUtensorMap xa[2 * SMAX];       // X slices as the A operand: [re slices, im slices], box 128 rows
    CUtensorMap yb[NPLANES_B];      // Y slices as the B operand: [re, im, -re], box NT rows
    int m;                   // rows of C = columns of X
    int nc;                  // columns of C = columns of Y
    int kblocks;             // 2 Vp / 64
    int vpb;                 // Vp / 64 (chunks per half)
    int upper;
    int trans_a;             // X^T Y instead of X^H Y
    int cswap_b;             // Y -> C Y
    int ntiles_n;            // number of NT-column tiles
    const int *ex;           // column exponents of X
    const int *ey;           // column exponents of Y
    double2 *C;
    int64_t ldc;
    int *err;
    long long wait;          // cap of every pipeline wait, SM clock cycles
};

static_assert(sizeof(Params) <= 4096, "ozaki_kernel: parameter block above 4 KB");

__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float v) {
    float s = hi + v;
    float bb = s - hi;
    float e = (hi - (s - bb)) + (v - bb);
    hi = s;
    lo += e;
}

// S: slices per operand used by this product (levels 2 .. S+1 are kept)
template <int S>
__global__ void __launch_bounds__(Geom<S>::THREADS, 1) ozaki_kernel(const __grid_constant__ Params p) {
    using G = Geom<S>;
    constexpr int LEVELS = S, NT = G::NT, A_STAGES = G::A_STAGES, B_TILE = G::B_TILE, B_STACK = G::B_STACK,
                  B_STAGE = G::B_STAGE, BUF_COLS = G::BUF_COLS, NTE = G::NTE;
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
    const int m0 = blockIdx.y * tc::BM;
    const int n0 = blockIdx.x * NT;
    if (p.upper && n0 + NT - 1 < m0) return;   // tile entirely below the diagonal

    if (threadIdx.x == 0) {
        for (int s = 0; s < A_STAGES; ++s) { tc::mbar_init(&afull[s], 1); tc::mbar_init(&aempty[s], 1); }
        for (int s = 0; s < B_STAGES; ++s) { tc::mbar_init(&bfull[s], 1); tc::mbar_init(&bempty[s], 1); }
        for (int s = 0; s < 2; ++s) { tc::mbar_init(&accfull[s], 1); tc::mbar_init(&accempty[s], 32 * G::EPI); }
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
        int ia = 0, ib = 0;
        bool ok = true;
        for (int kb = 0; kb < KB && ok; ++kb) {
            {
                const int s = ib % B_STAGES;
                const uint32_t ph = (ib / B_STAGES) & 1;
                if (!tc::mbar_wait(&bempty[s], ph ^ 1, p.err, 21, p.wait)) { ok = false; break; }
                unsigned char *dst = sB + s * B_STAGE;
                const int kbs = !p.cswap_b ? kb : (kb < p.vpb ? kb + p.vpb : kb - p.vpb);
                tc::mbar_expect_tx(&bfull[s], 4 * S * B_TILE);
                for (int q = 0; q < S; ++q) {
                    // stack 1: Re Y_q, Im Y_q;  stack 2: Im Y_q, -Re Y_q
                    tc::tma_load_2d(dst + (2 * q) * B_TILE, &p.yb[q], kbs * tc::BK, n0, &bfull[s]);
                    tc::tma_load_2d(dst + (2 * q + 1) * B_TILE, &p.yb[SMAX + q], kbs * tc::BK, n0, &bfull[s]);
                    tc::tma_load_2d(dst + B_STACK + (2 * q) * B_TILE, &p.yb[SMAX + q], kbs * tc::BK, n0, &bfull[s]);
                    tc::tma_load_2d(dst + B_STACK + (2 * q + 1) * B_TILE, &p.yb[2 * SMAX + q], kbs * tc::BK, n0,
                                    &bfull[s]);
                }
                ++ib;
            }
            for (int a = 0; a < S; ++a, ++ia) {
                const int s = ia % A_STAGES;
                const uint32_t ph = (ia / A_STAGES) & 1;
                if (!tc::mbar_wait(&aempty[s], ph ^ 1, p.err, 22, p.wait)) { ok = false; break; }
                unsigned char *dst = sA + s * A_STAGE;
                tc::mbar_expect_tx(&afull[s], A_STAGE);
                tc::tma_load_2d(dst, &p.xa[a], kb * tc::BK, m0, &afull[s]);
                tc::tma_load_2d(dst + A_TILE, &p.xa[SMAX + a], kb * tc::BK, m0, &afull[s]);
            }
        }
        // drain loads in flight
        for (int s = 0; s < A_STAGES && s < ia; ++s) {
            const int last = ia - 1 - ((ia - 1 - s) % A_STAGES);
            tc::mbar_drain(&afull[s], (last / A_STAGES) & 1, p.err, 23);
        }
        for (int s = 0; s < B_STAGES && s < ib; ++s) {
            const int last = ib - 1 - ((ib - 1 - s) % B_STAGES);
            tc::mbar_drain(&bfull[s], (last / B_STAGES) & 1, p.err, 24);
        }
    } else if (warp == 1 && lane == 0) {
        // ------------------------------------------------------------ MMA
        int ia = 0;
        bool ok = true;
        for (int kb = 0; kb < KB && ok; ++kb) {
            const int buf = kb & 1;
            const int use = kb >> 1;   // how many times this buffer was used before
            if (use > 0 && !tc::mbar_wait(&accempty[buf], (use - 1) & 1, p.err, 25, p.wait)) { ok = false; break; }
            tc::tc_fence_after();
            const int sbi = kb % B_STAGES;
            if (!tc::mbar_wait(&bfull[sbi], (kb / B_STAGES) & 1, p.err, 26, p.wait)) { ok = false; break; }
            unsigned char *bst = sB + sbi * B_STAGE;
            const uint64_t db1 = tc::smem_desc_k128(bst);             // [Re Y_b, Im Y_b] stack
            const uint64_t db2 = tc::smem_desc_k128(bst + B_STACK);   // [Im Y_b, -Re Y_b] stack
            const uint32_t acc0 = tbase + (uint32_t)(buf * BUF_COLS);
            for (int a = 0; a < S; ++a, ++ia) {
                const int s = ia % A_STAGES;
                if (!tc::mbar_wait(&afull[s], (ia / A_STAGES) & 1, p.err, 27, p.wait)) { ok = false; break; }
                tc::tc_fence_after();
                unsigned char *ast = sA + s * A_STAGE;
                const uint64_t dar = tc::smem_desc_k128(ast), dai = tc::smem_desc_k128(ast + A_TILE);
                const int nb = S - a;                     // slices b = 0 .. S-1-a (levels a+b+2 <= S+1)
                const uint32_t id1 = tc::idesc_bf16(2 * NT * nb, false, false);
                // X^H Y: Im X enters with +; X^T Y: with - (Re -= Xi Yi, Im += Xi Yr via the -Re Y slices)
                const uint32_t id2 = tc::idesc_bf16(2 * NT * nb, p.trans_a != 0, false);
                const uint32_t d = acc0 + (uint32_t)(a * 2 * NT);
#pragma unroll
                for (int k = 0; k < tc::BK / tc::UMMA_K; ++k) {
                    const uint64_t o = (uint64_t)(2 * k);
                    const uint32_t first = (a == 0 && k == 0) ? 0u : 1u;
                    tc::mma_bf16(d, dar + o, db1 + o, id1, first);   // [Re | Im] += Xr [Yr | Yi]
                    tc::mma_bf16(d, dai + o, db2 + o, id2, 1u);      // [Re | Im] += (+-Xi) [Yi | -Yr]
                }
                tc::mma_commit(&aempty[s]);
            }
            if (!ok) break;
            tc::mma_commit(&bempty[sbi]);
            tc::mma_commit(&accfull[buf]);
        }
        // make sure every issued MMA has completed before the CTA tears down
        tc::mma_commit(donebar);
    } else if (warp >= 2) {
        // ------------------------------------------------------------ epilogue
        const int lb = 32 * (warp & 3);                  // the warp's quadrant of tensor-memory lanes
        const int row = lb + lane;
        const int cb = ((warp - 2) >> 2) * NTE;          // first tile column this thread drains
        float hr[NTE], lr[NTE], hi_[NTE], li[NTE];
#pragma unroll
        for (int j = 0; j < NTE; ++j) { hr[j] = 0.f; lr[j] = 0.f; hi_[j] = 0.f; li[j] = 0.f; }
        bool ok = true;
        for (int kb = 0; kb < KB; ++kb) {
            const int buf = kb & 1, use = kb >> 1;
            if (!tc::mbar_wait(&accfull[buf], use & 1, p.err, 28, p.wait)) { ok = false; break; }
            tc::tc_fence_after();
            const uint32_t t0 = tbase + ((uint32_t)lb << 16) + (uint32_t)(buf * BUF_COLS);
            const float sgn = (p.cswap_b && kb >= p.vpb) ? -1.f : 1.f;   // C Y: the v half enters negated
            float v[NTE];
#pragma unroll
            for (int L = 0; L < LEVELS; ++L) {
                // level L: [Re NT | Im NT]; this thread's columns cb .. cb + NTE - 1 of each
                const float sc = sgn * __int_as_float((127 - 8 * L) << 23);
                tc::tmem_ld_cols<NTE>(t0 + (uint32_t)(L * 2 * NT + cb), v);
#pragma unroll
                for (int j = 0; j < NTE; ++j) two_sum_acc(hr[j], lr[j], v[j] * sc);
                tc::tmem_ld_cols<NTE>(t0 + (uint32_t)(L * 2 * NT + NT + cb), v);
#pragma unroll
                for (int j = 0; j < NTE; ++j) two_sum_acc(hi_[j], li[j], v[j] * sc);
            }
            tc::tc_fence_before();
            tc::mbar_arrive(&accempty[buf]);
            if ((kb & 15) == 15) {
#pragma unroll
                for (int j = 0; j < NTE; ++j) {   // renormalise (hi, lo)
                    float s = hr[j] + lr[j]; lr[j] = lr[j] - (s - hr[j]); hr[j] = s;
                    s = hi_[j] + li[j]; li[j] = li[j] - (s - hi_[j]); hi_[j] = s;
                }
            }
        }
        if (ok) {
            const int i = m0 + row;
            if (i < p.m) {
                const int exi = p.ex[i];
                double2 *crow = p.C + i;
#pragma unroll
                for (int h = 0; h < NTE; h += 8) {
#pragma unroll
                    for (int j = h; j < h + 8; ++j) {   // unrolled: the accumulators stay in registers
                        const int jj = n0 + cb + j;
                        if (jj >= p.nc) continue;
                        // level 2 carries 2^-16 of the scaled product
                        const double sc = ldexp(1.0, exi + __ldg(p.ey + jj) - 16);
                        const double re = ((double)hr[j] + (double)lr[j]) * sc;
                        const double im = ((double)hi_[j] + (double)li[j]) * sc;
                        crow[(int64_t)jj * p.ldc] = make_double2(re, im);
                    }
                }
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        // the final commit above tracks every MMA; wait for it before freeing TMEM
        if (lane == 0) tc::mbar_drain(donebar, 0, p.err, 29);
        __syncwarp();
        tc::tc_fence_after();
        tc::tmem_dealloc(tbase, 512);
    }
}

// ---------------------------------------------------------------------------
// slicing: per column exponent, then S integer slices per real/imag part
// ---------------------------------------------------------------------------
__global__ void col_exponent_kernel(int64_t rows, int64_t cols, const double2 *__restrict__ X, int64_t ldx,
                                    int *__restrict__ ex) {
    __shared__ double s[256];
    const int64_t c = blockIdx.x;
    double m = 0.0;
    for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) {
        double2 v = X[r + c * ldx];
        m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
    }
    s[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] = fmax(s[threadIdx.x], s[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int e = 0;
        if (s[0] > 0.0) frexp(s[0], &e);   // s < 2^e
        ex[c] = e;
    }
}

// The first `stored` slices of every element.  Plane q: real slices
// (q = s), imaginary slices (q = stored + s) and negated real slices
// (q = 2 stored + s); element (row r, column c) at
// planes[q * pstride + c * kp + kr], kr = r (u half) or vp + r - V (v half);
// kp = 2 vp
__global__ void slice_kernel(int64_t rows, int64_t cols, int64_t V, int64_t vp, const double2 *__restrict__ X,
                             int64_t ldx, const int *__restrict__ ex, __nv_bfloat16 *__restrict__ planes,
                             int64_t pstride, int stored) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    const int64_t r = idx % rows, c = idx / rows;
    const double2 v = X[r + c * ldx];
    const int e = ex[c];
    const int64_t kr = r < V ? r : vp + (r - V);
    const int64_t o = c * 2 * vp + kr;
    double xr = ldexp(v.x, -e), xi = ldexp(v.y, -e);   // |x| < 1
#pragma unroll
    for (int s = 0; s < SMAX; ++s) {
        if (s >= stored) break;
        xr *= 256.0; xi *= 256.0;
        const double mr = rint(xr), mi = rint(xi);
        xr -= mr; xi -= mi;
        planes[(int64_t)s * pstride + o] = __double2bfloat16(mr);
        planes[(int64_t)(stored + s) * pstride + o] = __double2bfloat16(mi);
        planes[(int64_t)(2 * stored + s) * pstride + o] = __double2bfloat16(-mr);
    }
}

}  // namespace oz

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::once_flag g_encode_once;

int tensor_map_bf16(bdg_ctx *ctx, CUtensorMap *m, const void *ptr, int64_t rows, int64_t kdim, int64_t ld,
                    int box_rows) {
    // looked up once per process (the batched solver calls this from several threads)
    std::call_once(g_encode_once, [] {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) == cudaSuccess && fn)
            g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
        else
            cudaGetLastError();
    });
    if (!g_encode) return bdg_fail(ctx, BDG_ECUDA, "cuTensorMapEncodeTiled entry point not found");
    if (((uintptr_t)ptr & 15) || ((ld * 2) & 15))
        return bdg_fail(ctx, BDG_EINVAL, "tensor map: base or stride not 16-byte aligned");
    cuuint64_t dims[2] = {(cuuint64_t)kdim, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return bdg_fail(ctx, BDG_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return BDG_OK;
}

static int64_t half_pad(int64_t rows) { return ((rows / 2) + 63) / 64 * 64; }

size_t ozaki_plane_bytes(int64_t rows, int64_t cols) {
    return (size_t)oz::NPLANES_B * 2 * half_pad(rows) * cols * 2;
}

// Slice X (rows = 2V, cols columns, complex128) into bf16 planes + column
// exponents (layout above): the first `stored` slices of the real and
// imaginary parts and of the negated real parts.
int ozaki_slice(bdg_ctx *ctx, cudaStream_t st, int64_t rows, int64_t cols, const double2 *X, int64_t ldx,
                __nv_bfloat16 *planes, int *ex, int stored) {
    if (rows & 1) return bdg_fail(ctx, BDG_EINVAL, "ozaki_slice: odd row count");
    if (stored < 1 || stored > oz::SMAX) return bdg_fail(ctx, BDG_EINVAL, "ozaki_slice: %d slices", stored);
    const int64_t V = rows / 2, vp = half_pad(rows);
    const int64_t pstride = 2 * vp * cols;
    oz::col_exponent_kernel<<<(unsigned)cols, 256, 0, st>>>(rows, cols, X, ldx, ex);
    BDG_LAUNCH_CHECK(ctx);
    if (vp != V) BDG_CUDA_TRY(ctx, cudaMemsetAsync(planes, 0, (size_t)3 * stored * pstride * 2, st));
    const int64_t tot = rows * cols;
    oz::slice_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(rows, cols, V, vp, X, ldx, ex, planes, pstride,
                                                                   stored);
    BDG_LAUNCH_CHECK(ctx);
    return BDG_OK;
}

// C (m x nc) = op(X)^T-or-H op_C(Y) with X (rows x m) and Y (rows x nc) already
// sliced, each buffer holding `stored` slices per part: trans_a selects X^T
// instead of X^H, cswap_b replaces Y by C Y.  `slices` (4, 5 or 6; at most
// `stored`) are used: the product is accurate to about 2^(-8 slices) of the
// scaled terms (6: FP64 level).
// With `upper`, only the entries C[i][j], j >= i, are guaranteed.
int ozaki_product(bdg_ctx *ctx, cudaStream_t st, int64_t rows, int64_t m, int64_t nc, const __nv_bfloat16 *px,
                  const int *ex, const __nv_bfloat16 *py, const int *ey, double2 *C, int64_t ldc, bool upper,
                  bool trans_a, bool cswap_b, int slices, int stored) {
    const int64_t vp = half_pad(rows), kp = 2 * vp;
    if (slices < 4 || slices > 6) return bdg_fail(ctx, BDG_EINVAL, "ozaki_product: %d slices (4, 5 or 6)", slices);
    if (stored < slices || stored > oz::SMAX)
        return bdg_fail(ctx, BDG_EINVAL, "ozaki_product: %d stored slices for a %d-slice product", stored, slices);
    oz::Params p;
    memset(&p, 0, sizeof(p));
    // maps for the planes that exist: re slices q, im slices stored + q, -re slices 2 stored + q
    for (int q = 0; q < stored; ++q) {
        int rc = tensor_map_bf16(ctx, &p.xa[q], px + q * kp * m, m, kp, kp, tc::BM);
        if (!rc) rc = tensor_map_bf16(ctx, &p.xa[oz::SMAX + q], px + (stored + q) * kp * m, m, kp, kp, tc::BM);
        if (rc) return rc;
    }
    const int nt = oz::tile_width(slices);
    for (int q = 0; q < stored; ++q) {
        for (int part = 0; part < 3; ++part) {
            int rc = tensor_map_bf16(ctx, &p.yb[part * oz::SMAX + q], py + (part * stored + q) * kp * nc, nc, kp,
                                     kp, nt);
            if (rc) return rc;
        }
    }
    p.m = (int)m;
    p.nc = (int)nc;
    p.kblocks = (int)(kp / tc::BK);
    p.vpb = (int)(vp / tc::BK);
    p.upper = upper ? 1 : 0;
    p.trans_a = trans_a ? 1 : 0;
    p.cswap_b = cswap_b ? 1 : 0;
    p.ntiles_n = (int)((nc + nt - 1) / nt);
    p.ex = ex;
    p.ey = ey;
    p.C = C;
    p.ldc = ldc;
    p.err = ctx->dflags + 4;
    p.wait = ctx->wait_cycles;
    dim3 grid((unsigned)p.ntiles_n, (unsigned)((m + tc::BM - 1) / tc::BM));
    auto launch = [&](auto kern, int smem, int threads) -> int {
        BDG_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        kern<<<grid, threads, smem, st>>>(p);
        return BDG_OK;
    };
    int rc = BDG_OK;
    switch (slices) {
    case 4: rc = launch(oz::ozaki_kernel<4>, oz::Geom<4>::SMEM, oz::Geom<4>::THREADS); break;
    case 5: rc = launch(oz::ozaki_kernel<5>, oz::Geom<5>::SMEM, oz::Geom<5>::THREADS); break;
    default: rc = launch(oz::ozaki_kernel<6>, oz::Geom<6>::SMEM, oz::Geom<6>::THREADS); break;
    }
    if (rc) return rc;
    BDG_LAUNCH_CHECK(ctx);
    return BDG_OK;
}

}  // namespace bdg
