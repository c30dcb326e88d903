// Shared device helpers of libbdg: complex arithmetic templated on the real
// type, launch/error plumbing and a bounded software grid barrier.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/bdg.h"

namespace bdg {

// ---------------------------------------------------------------------------
// complex numbers: float2 / double2 with .x = real, .y = imaginary
// ---------------------------------------------------------------------------
template <typename R> struct CT;
template <> struct CT<double> { using T = double2; };
template <> struct CT<float> { using T = float2; };
template <typename R> using cplx = typename CT<R>::T;

template <typename R> __host__ __device__ __forceinline__ cplx<R> mk(R a, R b) { cplx<R> z; z.x = a; z.y = b; return z; }
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) { C z; z.x = a.x * b.x - a.y * b.y; z.y = a.x * b.y + a.y * b.x; return z; }
// conj(a) * b
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) { C z; z.x = a.x * b.x + a.y * b.y; z.y = a.x * b.y - a.y * b.x; return z; }
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
template <typename C, typename R> __host__ __device__ __forceinline__ C cscale(C a, R s) { a.x *= s; a.y *= s; return a; }
template <typename C> __host__ __device__ __forceinline__ auto cabs2(C a) -> decltype(a.x) { return a.x * a.x + a.y * a.y; }
// acc += a * b
template <typename C> __host__ __device__ __forceinline__ void cfma(C &acc, C a, C b) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename C> __host__ __device__ __forceinline__ void cfmac(C &acc, C a, C b) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}
template <typename C> __host__ __device__ __forceinline__ C czero() { C z; z.x = 0; z.y = 0; return z; }

// L2-only loads/stores (bypass L1) for data that other CTAs write concurrently.
__device__ __forceinline__ float2 ldcg(const float2 *p) { return __ldcg(p); }
__device__ __forceinline__ double2 ldcg(const double2 *p) { return __ldcg(p); }
__device__ __forceinline__ void stcg(float2 *p, float2 v) { __stcg(p, v); }
__device__ __forceinline__ void stcg(double2 *p, double2 v) { __stcg(p, v); }

// ---------------------------------------------------------------------------
// block reductions
// ---------------------------------------------------------------------------
template <typename R> __device__ __forceinline__ R warp_sum(R v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block; every thread receives the result.  `scratch` needs
// blockDim.x/32 entries.  Contains __syncthreads().
template <typename R> __device__ R block_sum(R v, R *scratch) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    R t = 0;
    for (int i = 0; i < nw; ++i) t += scratch[i];
    return t;
}

// ---------------------------------------------------------------------------
// bounded waits
// ---------------------------------------------------------------------------
// Every device-side spin has an iteration cap; on expiry it raises `err`
// (read by the host and reported as BDG_ETIMEOUT) and gives up.
constexpr long long kSpinLimit = 40000000;  // ~2-4 s with the back-off below

struct GridBarrier {
    unsigned int count;
    unsigned int gen;
    int err;
    int pad;
};

// Software barrier across all CTAs of a cooperative launch (all CTAs are
// co-resident).  Returns false if the wait gave up; the caller must then
// return.  Contains __syncthreads().
__device__ __forceinline__ bool grid_sync(GridBarrier *gb) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *vgen = &gb->gen;
        volatile int *verr = &gb->err;
        unsigned int g = *vgen;
        __threadfence();
        unsigned int arrived = atomicAdd(&gb->count, 1u);
        int ok = 1;
        if (arrived == gridDim.x * gridDim.y * gridDim.z - 1) {
            atomicExch(&gb->count, 0u);
            __threadfence();
            atomicAdd(&gb->gen, 1u);
        } else {
            long long it = 0;
            while (*vgen == g) {
                if (*verr) { ok = 0; break; }
                if (++it > kSpinLimit) { atomicExch(&gb->err, 1); ok = 0; break; }
                __nanosleep(40);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---------------------------------------------------------------------------
// host-side error plumbing
// ---------------------------------------------------------------------------
struct Status {
    int code = BDG_OK;
    char msg[512] = {0};
};

}  // namespace bdg

#define BDG_CUDA_TRY(ctxp, call)                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            return bdg_fail((ctxp), BDG_ECUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call,      \
                            cudaGetErrorString(e_));                                          \
        }                                                                                     \
    } while (0)

#define BDG_LAUNCH_CHECK(ctxp)          \
    do {                                \
        bdg_count_launch(ctxp);         \
        BDG_CUDA_TRY(ctxp, cudaGetLastError()); \
    } while (0)
