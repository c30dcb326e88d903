// SIMT complex GEMM (FP64 and FP32), column-major:
//     C = alpha * op(A) * op(B) + beta * C,   op in {N (as is), C (conjugate transpose), T (transpose)}.
//
// Used for the FP64 path (B300's FP64 rate is ~1 TFLOP/s on any unit, so a
// register-tiled SIMT kernel reaches it) and for the small/skinny products of
// the reduced-precision path.  64x64 output tile per CTA, 256 threads, 4x4
// complex outputs per thread with a stride of 16 so that shared-memory reads
// broadcast.  A deterministic split-K variant handles the b x b reductions
// over the long dimension (V^H X with K = N).
#include "internal.h"

namespace bdg {

template <typename R> struct GemmCfg;
template <> struct GemmCfg<float> { static constexpr int BK = 16; };
template <> struct GemmCfg<double> { static constexpr int BK = 8; };

// op codes: 0 = as is, 1 = conjugate transpose, 2 = transpose
template <typename R>
__device__ __forceinline__ cplx<R> load_op(const cplx<R> *__restrict__ P, int64_t ld, int op,
                                            int64_t r, int64_t c, int64_t nr, int64_t nc) {
    // element (r, c) of op(P), where op(P) is nr x nc
    if (r >= nr || c >= nc) return czero<cplx<R>>();
    if (op == 0) return P[r + c * ld];
    cplx<R> v = P[c + r * ld];
    if (op == 1) v.y = -v.y;
    return v;
}
static inline int op_code(char o) { return o == 'C' ? 1 : (o == 'T' ? 2 : 0); }

// Computes a 64x64 tile of op(A)[m0:, k0:k1] * op(B)[k0:k1, n0:] and writes
// alpha*acc + beta*C (or, with `partial`, the raw acc into partial[z]).
template <typename R>
__global__ void __launch_bounds__(256) gemm_kernel(int ca, int cb, int64_t M, int64_t N, int64_t K,
                                                   cplx<R> alpha, const cplx<R> *__restrict__ A, int64_t lda,
                                                   const cplx<R> *__restrict__ B, int64_t ldb, cplx<R> beta,
                                                   cplx<R> *__restrict__ C, int64_t ldc, int64_t kchunk,
                                                   cplx<R> *__restrict__ partial) {
    constexpr int BK = GemmCfg<R>::BK;
    using Cx = cplx<R>;
    __shared__ Cx As[BK][64];
    __shared__ Cx Bs[BK][64];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t m0 = (int64_t)blockIdx.x * 64, n0 = (int64_t)blockIdx.y * 64;
    const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
    const int64_t kend = min(K, kbeg + kchunk);
    Cx acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = czero<Cx>();

    for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
        // load tiles: 64*BK elements each, 256 threads
#pragma unroll
        for (int e = threadIdx.x; e < 64 * BK; e += 256) {
            int r, c;
            if (!ca) { r = e & 63; c = e >> 6; }      // consecutive threads -> consecutive rows
            else { c = e % BK; r = e / BK; }          // consecutive threads -> consecutive k
            As[c][r] = (k0 + c < kend) ? load_op<R>(A, lda, ca, m0 + r, k0 + c, M, K) : czero<Cx>();
        }
#pragma unroll
        for (int e = threadIdx.x; e < 64 * BK; e += 256) {
            int r, c;  // r = k index, c = column of op(B)
            if (!cb) { r = e % BK; c = e / BK; }
            else { c = e & 63; r = e >> 6; }
            Bs[r][c] = (k0 + r < kend) ? load_op<R>(B, ldb, cb, k0 + r, n0 + c, K, N) : czero<Cx>();
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            Cx a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t r = m0 + ty + 16 * i;
        if (r >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t c = n0 + tx + 16 * j;
            if (c >= N) continue;
            if (partial) {
                partial[(int64_t)blockIdx.z * M * N + r + c * M] = acc[i][j];
            } else {
                Cx out = cmul(alpha, acc[i][j]);
                if (beta.x != 0 || beta.y != 0) out = cadd(out, cmul(beta, C[r + c * ldc]));
                C[r + c * ldc] = out;
            }
        }
    }
}

template <typename R>
__global__ void splitk_reduce_kernel(int64_t M, int64_t N, int splits, const cplx<R> *__restrict__ partial,
                                     cplx<R> alpha, cplx<R> beta, cplx<R> *__restrict__ C, int64_t ldc) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= M * N) return;
    int64_t r = idx % M, c = idx / M;
    cplx<R> s = czero<cplx<R>>();
    for (int z = 0; z < splits; ++z) s = cadd(s, partial[(int64_t)z * M * N + idx]);
    cplx<R> out = cmul(alpha, s);
    if (beta.x != 0 || beta.y != 0) out = cadd(out, cmul(beta, C[r + c * ldc]));
    C[r + c * ldc] = out;
}

template <typename R>
int gemm(bdg_ctx *ctx, cudaStream_t st, char opA, char opB, int64_t M, int64_t N, int64_t K,
         cplx<R> alpha, const cplx<R> *A, int64_t lda, const cplx<R> *B, int64_t ldb,
         cplx<R> beta, cplx<R> *C, int64_t ldc) {
    if (M <= 0 || N <= 0) return BDG_OK;
    if (K <= 0) {
        // C = beta * C
        alpha = czero<cplx<R>>();
        K = 0;
    }
    dim3 grid((unsigned)((M + 63) / 64), (unsigned)((N + 63) / 64), 1);
    if (grid.y > 65535) return bdg_fail(ctx, BDG_EUNSUPPORTED, "gemm: N too large");
    gemm_kernel<R><<<grid, 256, 0, st>>>(op_code(opA), op_code(opB), M, N, K, alpha, A, lda, B, ldb, beta,
                                         C, ldc, K > 0 ? K : 1, nullptr);
    BDG_LAUNCH_CHECK(ctx);
    return BDG_OK;
}

template <typename R>
int gemm_splitk(bdg_ctx *ctx, cudaStream_t st, char opA, char opB, int64_t M, int64_t N, int64_t K,
                cplx<R> alpha, const cplx<R> *A, int64_t lda, const cplx<R> *B, int64_t ldb,
                cplx<R> beta, cplx<R> *C, int64_t ldc, int splits, cplx<R> *partial) {
    if (M <= 0 || N <= 0) return BDG_OK;
    constexpr int BK = GemmCfg<R>::BK;
    int64_t kchunk = (K + splits - 1) / splits;
    kchunk = (kchunk + BK - 1) / BK * BK;
    if (kchunk < BK) kchunk = BK;
    int z = (int)((K + kchunk - 1) / kchunk);
    if (z < 1) z = 1;
    dim3 grid((unsigned)((M + 63) / 64), (unsigned)((N + 63) / 64), (unsigned)z);
    gemm_kernel<R><<<grid, 256, 0, st>>>(op_code(opA), op_code(opB), M, N, K, alpha, A, lda, B, ldb, beta,
                                         C, ldc, kchunk, partial);
    BDG_LAUNCH_CHECK(ctx);
    int64_t tot = M * N;
    splitk_reduce_kernel<R><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(M, N, z, partial, alpha, beta,
                                                                           C, ldc);
    BDG_LAUNCH_CHECK(ctx);
    return BDG_OK;
}

template int gemm<float>(bdg_ctx *, cudaStream_t, char, char, int64_t, int64_t, int64_t, float2,
                         const float2 *, int64_t, const float2 *, int64_t, float2, float2 *, int64_t);
template int gemm<double>(bdg_ctx *, cudaStream_t, char, char, int64_t, int64_t, int64_t, double2,
                          const double2 *, int64_t, const double2 *, int64_t, double2, double2 *, int64_t);
template int gemm_splitk<float>(bdg_ctx *, cudaStream_t, char, char, int64_t, int64_t, int64_t, float2,
                                const float2 *, int64_t, const float2 *, int64_t, float2, float2 *, int64_t,
                                int, float2 *);
template int gemm_splitk<double>(bdg_ctx *, cudaStream_t, char, char, int64_t, int64_t, int64_t, double2,
                                 const double2 *, int64_t, const double2 *, int64_t, double2, double2 *,
                                 int64_t, int, double2 *);

}  // namespace bdg
