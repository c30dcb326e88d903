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
        // issue all loads first so that their latencies overlap
        double2 o[32];
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (n0 + j < N) o[j] = C[m + (int64_t)(n0 + j) * ldc];
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (n0 + j < N)
                C[m + (int64_t)(n0 + j) * ldc] = make_double2(o[j].x + alpha * (double)v0[j], o[j].y + alpha * (double)v1[j]);
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
        float2 q[32];
        if (beta != 0.f) {
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (n0 + j < N) q[j] = C[m + (int64_t)(n0 + j) * ldc];
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            if (n0 + j >= N) continue;
            float2 o = make_float2(alpha * v0[j], alpha * v1[j]);
            if (beta != 0.f) { o.x += beta * q[j].x; o.y += beta * q[j].y; }
            C[m + (int64_t)(n0 + j) * ldc] = o;
        }
    }
};

// split-K partial of layer blockIdx.z: part[z * M * N + m + n * ldp]
struct EpiZ32Split {
    float2 *part;
    int64_t ldp;
    int M, N;
    __device__ void operator()(int m, int n0, const float *v0, const float *v1) const {
        if (m >= M) return;
        float2 *P = part + (int64_t)blockIdx.z * (int64_t)M * N;
#pragma unroll 4
        for (int j = 0; j < 32; ++j) {
            int n = n0 + j;
            if (n >= N) break;
            P[m + (int64_t)n * ldp] = make_float2(v0[j], v1[j]);
        }
    }
};

}  // namespace tc

// ---------------------------------------------------------------------------
// bf16 slice planes.  A value x is written as x = s_0 + s_1 + ... + s_{S-1}
// with s_0 = bf16(x) and s_q = bf16(x - s_0 - ... - s_{q-1}) (8 more
// significant bits per slice; S = 2 gives ~16 bits, S = 3 the full FP32
// significand).  Plane order: [re_0 .. re_{S-1}, im_0 .. im_{S-1}]; each plane
// holds element (c, r) at planes[q * pstride + c * ldp + r] (r contiguous:
// K-major when the contraction runs over r).
// ---------------------------------------------------------------------------
// FP64 input (the refinement's FP64 matrices): residuals in FP64
__device__ __forceinline__ void slice_value(double v, int S, __nv_bfloat16 *out) {
    double r = v;
    for (int q = 0; q < S; ++q) {
        __nv_bfloat16 h = __float2bfloat16_rn((float)r);
        out[q] = h;
        r -= (double)__bfloat162float(h);
    }
}
// FP32 input: x - bf16(x) is exact in FP32, so the residuals stay in FP32
__device__ __forceinline__ void slice_value(float v, int S, __nv_bfloat16 *out) {
    float r = v;
    for (int q = 0; q < S; ++q) {
        __nv_bfloat16 h = __float2bfloat16_rn(r);
        out[q] = h;
        r -= __bfloat162float(h);
    }
}

template <typename C>
__global__ void split_kernel(int64_t rows, int64_t cols, const C *__restrict__ X, int64_t ldx, bool conj_, int S,
                             __nv_bfloat16 *__restrict__ planes, int64_t ldp, int64_t pstride) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    const int64_t r = idx % rows, c = idx / rows;
    const C v = X[r + c * ldx];
    __nv_bfloat16 sr[4], si[4];
    slice_value(v.x, S, sr);
    slice_value(conj_ ? -v.y : v.y, S, si);
    const int64_t o = c * ldp + r;
    for (int q = 0; q < S; ++q) {
        planes[q * pstride + o] = sr[q];
        planes[(S + q) * pstride + o] = si[q];
    }
}

// transposed: element (r, c) of X goes to plane position (row r, k = c)
template <typename C>
__global__ void split_t_kernel(int64_t rows, int64_t cols, const C *__restrict__ X, int64_t ldx, bool conj_, int S,
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
            __nv_bfloat16 sr[4], si[4];
            slice_value(v.x, S, sr);
            slice_value(conj_ ? -v.y : v.y, S, si);
            const int64_t o = r * ldp + c;
            for (int q = 0; q < S; ++q) {
                planes[q * pstride + o] = sr[q];
                planes[(S + q) * pstride + o] = si[q];
            }
        }
    }
}

int64_t hilo_ld(int64_t k) { return (k + 63) / 64 * 64; }

template <typename C>
int split_planes(bdg_ctx *ctx, cudaStream_t st, int64_t rows, int64_t cols, const C *X, int64_t ldx, bool transpose,
                 bool conj_, int S, __nv_bfloat16 *planes) {
    // without transpose: plane rows = cols of X, K = rows of X; with: plane rows = rows of X, K = cols of X
    const int64_t kdim = transpose ? cols : rows;
    const int64_t prow = transpose ? rows : cols;
    const int64_t ldp = hilo_ld(kdim);
    const int64_t pstride = ldp * prow;
    if (ldp != kdim) BDG_CUDA_TRY(ctx, cudaMemsetAsync(planes, 0, (size_t)2 * S * pstride * 2, st));
    if (!transpose) {
        int64_t tot = rows * cols;
        split_kernel<C><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(rows, cols, X, ldx, conj_, S, planes, ldp,
                                                                       pstride);
    } else {
        dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
        split_t_kernel<C><<<grid, dim3(32, 8), 0, st>>>(rows, cols, X, ldx, conj_, S, planes, ldp, pstride);
    }
    BDG_LAUNCH_CHECK(ctx);
    return BDG_OK;
}

template <typename C>
int split_hilo(bdg_ctx *ctx, cudaStream_t st, int64_t rows, int64_t cols, const C *X, int64_t ldx, bool transpose,
               bool conj_, __nv_bfloat16 *planes) {
    return split_planes<C>(ctx, st, rows, cols, X, ldx, transpose, conj_, 2, planes);
}

template int split_planes<double2>(bdg_ctx *, cudaStream_t, int64_t, int64_t, const double2 *, int64_t, bool, bool,
                                   int, __nv_bfloat16 *);
template int split_planes<float2>(bdg_ctx *, cudaStream_t, int64_t, int64_t, const float2 *, int64_t, bool, bool,
                                  int, __nv_bfloat16 *);
template int split_hilo<double2>(bdg_ctx *, cudaStream_t, int64_t, int64_t, const double2 *, int64_t, bool, bool,
                                 __nv_bfloat16 *);

// Terms of a complex product with S slices per operand, keeping the slice
// pairs (a, b) with a + b <= S - 1 (S = 2: 3 pairs, S = 3: 6 pairs).  Map
// indices: A planes 0 .. 2S-1, B planes 2S .. 4S-1.
static void complex_terms(tc::Params &p, int S, int kblocks) {
    int t = 0;
    auto add = [&](int a, int b, int acc, int neg) {
        p.terms[t++] = tc::Term{(int8_t)a, (int8_t)b, (int8_t)acc, (int8_t)neg, kblocks};
    };
    const int B0 = 2 * S;
    for (int a = 0; a < S; ++a)
        for (int b = 0; a + b <= S - 1; ++b) {
            add(a, B0 + b, 0, 0);              // Re += Ar Br
            add(S + a, B0 + S + b, 0, 1);      // Re -= Ai Bi
            add(a, B0 + S + b, 1, 0);          // Im += Ar Bi
            add(S + a, B0 + b, 1, 0);          // Im += Ai Br
        }
    p.nterms = t;
    p.total_kblocks = t * kblocks;
}

template <int BN, class Epi>
static int launch_complex_bn(bdg_ctx *ctx, cudaStream_t st, int64_t M, int64_t N, int64_t K, int S,
                             const __nv_bfloat16 *pa, const __nv_bfloat16 *pb, const Epi &epi, int splits) {
    constexpr int STAGES = BN >= 128 ? 4 : 6;
    const int64_t ldp = hilo_ld(K);
    tc::Params p;
    memset(&p, 0, sizeof(p));
    for (int q = 0; q < 2 * S; ++q) {
        int rc = tensor_map_bf16(ctx, &p.maps[q], pa + q * ldp * M, M, ldp, ldp, tc::BM);
        if (rc) return rc;
        rc = tensor_map_bf16(ctx, &p.maps[2 * S + q], pb + q * ldp * N, N, ldp, ldp, BN);
        if (rc) return rc;
    }
    const int kb = (int)(ldp / tc::BK);
    complex_terms(p, S, kb);
    p.M = (int)M;
    p.N = (int)N;
    p.err = ctx->dflags + 5;
    p.wait = ctx->wait_cycles;
    if (splits < 1) splits = 1;
    p.kb_per_split = (kb + splits - 1) / splits;
    const int sm = tc::Smem<BN, STAGES>::TOTAL;
    BDG_CUDA_TRY(ctx, cudaFuncSetAttribute(tc::gemm_kernel<BN, 2, STAGES, Epi>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    dim3 grid((unsigned)((M + tc::BM - 1) / tc::BM), (unsigned)((N + BN - 1) / BN), (unsigned)splits);
    if (grid.y > 65535) return bdg_fail(ctx, BDG_EUNSUPPORTED, "tc gemm: N too large");
    tc::gemm_kernel<BN, 2, STAGES, Epi><<<grid, 192, sm, st>>>(p, epi);
    BDG_LAUNCH_CHECK(ctx);
    return BDG_OK;
}

// BN = 64 for skinny outputs (N <= 64), 128 otherwise
template <class Epi>
static int launch_complex(bdg_ctx *ctx, cudaStream_t st, int64_t M, int64_t N, int64_t K, int S,
                          const __nv_bfloat16 *pa, const __nv_bfloat16 *pb, const Epi &epi, int splits = 1) {
    if (N <= 64) return launch_complex_bn<64>(ctx, st, M, N, K, S, pa, pb, epi, splits);
    return launch_complex_bn<128>(ctx, st, M, N, K, S, pa, pb, epi, splits);
}

// split-K partials: part[z][m + n M] (complex64) reduced into C = alpha sum_z part + beta C
__global__ void splitk_sum_z32_kernel(int64_t M, int64_t N, int splits, const float2 *__restrict__ part, float alpha,
                                      float beta, float2 *__restrict__ C, int64_t ldc) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= M * N) return;
    int64_t m = idx % M, n = idx / M;
    float2 s = make_float2(0.f, 0.f);
    for (int z = 0; z < splits; ++z) {
        float2 v = part[(int64_t)z * M * N + idx];
        s.x += v.x; s.y += v.y;
    }
    float2 o = make_float2(alpha * s.x, alpha * s.y);
    if (beta != 0.f) { float2 q = C[m + n * ldc]; o.x += beta * q.x; o.y += beta * q.y; }
    C[m + n * ldc] = o;
}

// C (complex128, M x N, ldc) += alpha * A B where A is given by its hi/lo
// planes with rows = M (K-major) and B by planes with rows = N (K-major).
int zgemm_bf16x3_add64(bdg_ctx *ctx, cudaStream_t st, int64_t M, int64_t N, int64_t K, const __nv_bfloat16 *pa,
                       const __nv_bfloat16 *pb, double2 *C, int64_t ldc, double alpha) {
    tc::EpiAddZ64 e{C, ldc, (int)M, (int)N, alpha};
    // wide outputs: 128 x 256 tiles (the Re and Im accumulators fill the 512
    // tensor-memory columns), so each A tile feeds twice the MMA work of a
    // 128 x 128 tile and the operand bytes per flop fall by a quarter
    if (N >= 256) return launch_complex_bn<256>(ctx, st, M, N, K, 2, pa, pb, e, 1);
    return launch_complex(ctx, st, M, N, K, 2, pa, pb, e);
}

// C (complex64) = alpha * A B + beta * C with S slices per operand.  When the
// output is narrow and K long, the K dimension is split over `splits` CTA
// layers whose partial products go through `part` (splits * M * N complex64)
// and are summed deterministically.
int cgemm_bf16(bdg_ctx *ctx, cudaStream_t st, int S, int64_t M, int64_t N, int64_t K, const __nv_bfloat16 *pa,
               const __nv_bfloat16 *pb, float2 *C, int64_t ldc, float alpha, float beta, float2 *part, int splits) {
    if (splits > 1) {
        // no empty layer: every layer must own at least one K block
        const int kb = (int)(hilo_ld(K) / tc::BK);
        const int per = (kb + splits - 1) / splits;
        splits = (kb + per - 1) / per;
    }
    if (splits > 1 && part) {
        tc::EpiZ32Split e{part, M, (int)M, (int)N};
        int rc = launch_complex(ctx, st, M, N, K, S, pa, pb, e, splits);
        if (rc) return rc;
        int64_t tot = M * N;
        splitk_sum_z32_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(M, N, splits, part, alpha, beta, C, ldc);
        BDG_LAUNCH_CHECK(ctx);
        return BDG_OK;
    }
    tc::EpiZ32 e{C, ldc, (int)M, (int)N, alpha, beta};
    return launch_complex(ctx, st, M, N, K, S, pa, pb, e);
}

}  // namespace bdg
