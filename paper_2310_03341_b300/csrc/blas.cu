// Plain complex FP32 GEMMs through cuBLAS with the BF16x9 emulated FP32
// compute type (each FP32 operand split into three bf16 values, products on
// the tensor cores, FP32-accurate results).  Used by the BDG_PREC_BF16X9 mode
// for the plain GEMMs of stage 1 (A22 V and the rank-2b trailing update) and
// of the stage-1 back-transformation; every fused or special product of the
// solver is a kernel of this library.
#include <cublas_v2.h>

#include "internal.h"

namespace bdg {

static cublasOperation_t to_op(char o) {
    return o == 'C' ? CUBLAS_OP_C : (o == 'T' ? CUBLAS_OP_T : CUBLAS_OP_N);
}

int blas_cgemm_emu(bdg_ctx *ctx, cudaStream_t st, char opA, char opB, int64_t M, int64_t N, int64_t K, float2 alpha,
                   const float2 *A, int64_t lda, const float2 *B, int64_t ldb, float2 beta, float2 *C, int64_t ldc) {
    if (M <= 0 || N <= 0) return BDG_OK;
    if (!ctx->blas) {
        cublasHandle_t h;
        if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) return bdg_fail(ctx, BDG_ECUDA, "cublasCreate failed");
        ctx->blas = (void *)h;
    }
    cublasHandle_t h = (cublasHandle_t)ctx->blas;
    if (cublasSetStream(h, st) != CUBLAS_STATUS_SUCCESS) return bdg_fail(ctx, BDG_ECUDA, "cublasSetStream failed");
    cuComplex a = make_cuComplex(alpha.x, alpha.y), b = make_cuComplex(beta.x, beta.y);
    cublasStatus_t s = cublasGemmEx(h, to_op(opA), to_op(opB), (int)M, (int)N, (int)K, &a, A, CUDA_C_32F, (int)lda,
                                    B, CUDA_C_32F, (int)ldb, &b, C, CUDA_C_32F, (int)ldc,
                                    CUBLAS_COMPUTE_32F_EMULATED_16BFX9, CUBLAS_GEMM_DEFAULT);
    if (s != CUBLAS_STATUS_SUCCESS) return bdg_fail(ctx, BDG_ECUDA, "cublasGemmEx (bf16x9 emulation) failed: %d", (int)s);
    // library kernels: not counted by bdg_launch_count, which counts this library's own kernels
    return BDG_OK;
}

// C = alpha A B^H + conj(alpha) B A^H + beta C on the lower triangle of the Hermitian C
// (FP32, the rank-2k update of stage 1; the upper triangle is left untouched)
int blas_cher2k_lower(bdg_ctx *ctx, cudaStream_t st, int64_t n, int64_t k, float2 alpha, const float2 *A,
                      int64_t lda, const float2 *B, int64_t ldb, float beta, float2 *C, int64_t ldc) {
    if (n <= 0) return BDG_OK;
    if (!ctx->blas) {
        cublasHandle_t h;
        if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) return bdg_fail(ctx, BDG_ECUDA, "cublasCreate failed");
        ctx->blas = (void *)h;
    }
    cublasHandle_t h = (cublasHandle_t)ctx->blas;
    if (cublasSetStream(h, st) != CUBLAS_STATUS_SUCCESS) return bdg_fail(ctx, BDG_ECUDA, "cublasSetStream failed");
    cuComplex a = make_cuComplex(alpha.x, alpha.y);
    cublasStatus_t s = cublasCher2k(h, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N, (int)n, (int)k, &a,
                                    reinterpret_cast<const cuComplex *>(A), (int)lda,
                                    reinterpret_cast<const cuComplex *>(B), (int)ldb, &beta,
                                    reinterpret_cast<cuComplex *>(C), (int)ldc);
    if (s != CUBLAS_STATUS_SUCCESS) return bdg_fail(ctx, BDG_ECUDA, "cublasCher2k failed: %d", (int)s);
    return BDG_OK;
}

void blas_destroy(bdg_ctx *ctx) {
    if (ctx->blas) cublasDestroy((cublasHandle_t)ctx->blas);
    ctx->blas = nullptr;
}

}  // namespace bdg
