// Host side of the multi-term tcgen05 GEMM and the split-precision complex
// products built on it.
//
// "BF16x3" complex product C (+)= A B: every real and imaginary part is
// split into hi = bf16(x) and lo = bf16(x - hi) (about 16 significant bits
// together); the three products hi*hi + hi*lo + lo*hi are accumulated in
// FP32.  Complex arithmetic is expanded into real terms:
//     Re C = Ar Br - Ai Bi,   Im C = Ar Bi + Ai Br,
// i.e. 12 real bf16 products into two FP32 accumulators.
#include <cuda_bf16.h>

#include "internal.h"
#include "tc_gemm.cuh"

namespace bdg {

int tensor_map_bf16(bdg_ctx *ctx, CUtensorMap *m, const void *ptr, int64_t rows, int64_t kdim, int64_t ld,
                    int box_rows);

namespace tc {

// C[m + n ldc] (complex128) += (acc0, acc1)
struct EpiAddZ64 {
    double2 *C;
    int64_t ldc;
    int M, N;
    double alpha;
    __device__ void operator()(int m, int n0, const float *v0, const float *v1) const {
        if (m >= M) return;
#pragma unroll 4
        for (int j = 0; j < 32; ++j) {
            int n = n0 + j;
            if (n >= N) break;
            double2 *c = C + m + (int64_t)n * ldc;
            double2 o = *c;
            o.x += alpha * (double)v0[j];
            o.y += alpha * (double)v1[j];
            *c = o;
        }
    }
};

// C[m + n ldc] (complex64) = alpha * (acc0, acc1) + beta * C
struct EpiZ32 {
    float2 *C;
    int64_t ldc;
    int M, N;
    float alpha, beta;
    __device__ void operator()(int m, int n0, const float *v0, const float *v1) const {
        if (m >= M) return;
#pragma unroll 4
        for (int j = 0; j < 32; ++j) {
            int n = n0 + j;
            if (n >= N) break;
            float2 *c = C + m + (int64_t)n * ldc;
            float2 o = make_float2(alpha * v0[j], alpha * v1[j]);
            if (beta != 0.f) { float2 q = *c; o.x += beta * q.x; o.y += beta * q.y; }
            *c = o;
        }
    }
};

}  // namespace tc

// ---------------------------------------------------------------------------
// hi/lo planes.  Plane order: [re_hi, re_lo, im_hi, im_lo]; each plane holds
// element (c, r) at planes[q * pstride + c * ldp + r] (r contiguous: K-major
// when the contraction runs over r).
// ---------------------------------------------------------------------------
template <typename C>
__global__ void split_hilo_kernel(int64_t rows, int64_t cols, const C *__restrict__ X, int64_t ldx, bool conj_,
                                  __nv_bfloat16 *__restrict__ planes, int64_t ldp, int64_t pstride) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    const int64_t r = idx % rows, c = idx / rows;
    const C v = X[r + c * ldx];
    const float xr = (float)v.x, xi = conj_ ? -(float)v.y : (float)v.y;
    const __nv_bfloat16 rh = __float2bfloat16_rn(xr), ih = __float2bfloat16_rn(xi);
    const __nv_bfloat16 rl = __float2bfloat16_rn((float)((double)v.x - (double)__bfloat162float(rh)));
    const double vi = conj_ ? -(double)v.y : (double)v.y;
    const __nv_bfloat16 il = __float2bfloat16_rn((float)(vi - (double)__bfloat162float(ih)));
    const int64_t o = c * ldp + r;
    planes[o] = rh;
    planes[pstride + o] = rl;
    planes[2 * pstride + o] = ih;
    planes[3 * pstride + o] = il;
}

// transposed: element (r, c) of X goes to plane position (row r, k = c)
template <typename C>
__global__ void split_hilo_t_kernel(int64_t rows, int64_t cols, const C *__restrict__ X, int64_t ldx, bool conj_,
                                    __nv_bfloat16 *__restrict__ planes, int64_t ldp, int64_t pstride) {
    __shared__ C tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int k = 0; k < 32; k += 8) {
        int64_t r = r0 + tx, c = c0 + ty + k;
        if (r < rows && c < cols) tile[ty + k][tx] = X[r + c * ldx];
    }
    __syncthreads();
    for (int k = 0; k < 32; k += 8) {
        int64_t r = r0 + ty + k, c = c0 + tx;
        if (r < rows && c < cols) {
            const C v = tile[tx][ty + k];
            const double vr = (double)v.x, vi = conj_ ? -(double)v.y : (double)v.y;
            const __nv_bfloat16 rh = __float2bfloat16_rn((float)vr), ih = __float2bfloat16_rn((float)vi);
            const __nv_bfloat16 rl = __float2bfloat16_rn((float)(vr - (double)__bfloat162float(rh)));
            const __nv_bfloat16 il = __float2bfloat16_rn((float)(vi - (double)__bfloat162float(ih)));
            const int64_t o = r * ldp + c;
            planes[o] = rh;
            planes[pstride + o] = rl;
            planes[2 * pstride + o] = ih;
            planes[3 * pstride + o] = il;
        }
    }
}

int64_t hilo_ld(int64_t k) { return (k + 63) / 64 * 64; }

template <typename C>
int split_hilo(bdg_ctx *ctx, cudaStream_t st, int64_t rows, int64_t cols, const C *X, int64_t ldx, bool transpose,
               bool conj_, __nv_bfloat16 *planes) {
    // without transpose: plane rows = cols of X, K = rows of X; with: plane rows = rows of X, K = cols of X
    const int64_t kdim = transpose ? cols : rows;
    const int64_t prow = transpose ? rows : cols;
    const int64_t ldp = hilo_ld(kdim);
    const int64_t pstride = ldp * prow;
    if (ldp != kdim) BDG_CUDA_TRY(ctx, cudaMemsetAsync(planes, 0, (size_t)4 * pstride * 2, st));
    if (!transpose) {
        int64_t tot = rows * cols;
        split_hilo_kernel<C><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(rows, cols, X, ldx, conj_, planes, ldp,
                                                                            pstride);
    } else {
        dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
        split_hilo_t_kernel<C><<<grid, dim3(32, 8), 0, st>>>(rows, cols, X, ldx, conj_, planes, ldp, pstride);
    }
    BDG_LAUNCH_CHECK(ctx);
    return BDG_OK;
}

template int split_hilo<double2>(bdg_ctx *, cudaStream_t, int64_t, int64_t, const double2 *, int64_t, bool, bool,
                                 __nv_bfloat16 *);
template int split_hilo<float2>(bdg_ctx *, cudaStream_t, int64_t, int64_t, const float2 *, int64_t, bool, bool,
                                __nv_bfloat16 *);

// Fill the 12 terms of a complex BF16x3 product.  Map indices: A planes 0..3
// (re_hi, re_lo, im_hi, im_lo), B planes 4..7.
static void complex_terms(tc::Params &p, int kblocks) {
    int t = 0;
    auto add = [&](int a, int b, int acc, int neg) { p.terms[t++] = tc::Term{(int8_t)a, (int8_t)b, (int8_t)acc, (int8_t)neg, kblocks}; };
    // Re = Ar Br - Ai Bi
    add(0, 4, 0, 0); add(0, 5, 0, 0); add(1, 4, 0, 0);
    add(2, 6, 0, 1); add(2, 7, 0, 1); add(3, 6, 0, 1);
    // Im = Ar Bi + Ai Br
    add(0, 6, 1, 0); add(0, 7, 1, 0); add(1, 6, 1, 0);
    add(2, 4, 1, 0); add(2, 5, 1, 0); add(3, 4, 1, 0);
    p.nterms = t;
    p.total_kblocks = t * kblocks;
}

template <class Epi>
static int launch_complex(bdg_ctx *ctx, cudaStream_t st, int64_t M, int64_t N, int64_t K, const __nv_bfloat16 *pa,
                          const __nv_bfloat16 *pb, const Epi &epi) {
    constexpr int BN = 128, STAGES = 4;
    const int64_t ldp = hilo_ld(K);
    tc::Params p;
    memset(&p, 0, sizeof(p));
    for (int q = 0; q < 4; ++q) {
        int rc = tensor_map_bf16(ctx, &p.maps[q], pa + q * ldp * M, M, ldp, ldp, tc::BM);
        if (rc) return rc;
        rc = tensor_map_bf16(ctx, &p.maps[4 + q], pb + q * ldp * N, N, ldp, ldp, BN);
        if (rc) return rc;
    }
    complex_terms(p, (int)(ldp / tc::BK));
    p.M = (int)M;
    p.N = (int)N;
    p.err = ctx->dflags + 5;
    const int sm = tc::Smem<BN, STAGES>::TOTAL;
    BDG_CUDA_TRY(ctx, cudaFuncSetAttribute(tc::gemm_kernel<BN, 2, STAGES, Epi>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    dim3 grid((unsigned)((M + tc::BM - 1) / tc::BM), (unsigned)((N + BN - 1) / BN));
    if (grid.y > 65535) return bdg_fail(ctx, BDG_EUNSUPPORTED, "tc gemm: N too large");
    tc::gemm_kernel<BN, 2, STAGES, Epi><<<grid, 192, sm, st>>>(p, epi);
    BDG_LAUNCH_CHECK(ctx);
    return BDG_OK;
}

// C (complex128, M x N, ldc) += alpha * A B where A is given by its hi/lo
// planes with rows = M (K-major) and B by planes with rows = N (K-major).
int zgemm_bf16x3_add64(bdg_ctx *ctx, cudaStream_t st, int64_t M, int64_t N, int64_t K, const __nv_bfloat16 *pa,
                       const __nv_bfloat16 *pb, double2 *C, int64_t ldc, double alpha) {
    tc::EpiAddZ64 e{C, ldc, (int)M, (int)N, alpha};
    return launch_complex(ctx, st, M, N, K, pa, pb, e);
}

// C (complex64) = alpha * A B + beta * C
int cgemm_bf16x3(bdg_ctx *ctx, cudaStream_t st, int64_t M, int64_t N, int64_t K, const __nv_bfloat16 *pa,
                 const __nv_bfloat16 *pb, float2 *C, int64_t ldc, float alpha, float beta) {
    tc::EpiZ32 e{C, ldc, (int)M, (int)N, alpha, beta};
    return launch_complex(ctx, st, M, N, K, pa, pb, e);
}

}  // namespace bdg
