// Multi-term tcgen05 GEMM:   D_acc[m, n] = sum over terms t with acc_t = acc of
//                                 (+/-) sum_k A_t[m, k] B_t[n, k]
// with every A_t, B_t a bf16 K-major matrix described by a TMA tensor map.
// Complex and split-precision products are expressed as lists of real
// terms (e.g. Re C = Ar Br^T + Ai Bi^T summed over hi/lo slices), all
// accumulated in FP32 in tensor memory; up to two accumulators per tile
// (real and imaginary part).  The epilogue functor receives, per thread, one
// output row and 32 consecutive columns of each accumulator.
//
// Warp roles (192 threads): warp 0 issues TMA loads, warp 1 owns TMEM and
// issues tcgen05.mma from one thread, warps 2..5 drain the accumulators.
#pragma once

#include "tc.cuh"

namespace bdg {
namespace tc {

constexpr int kMaxMaps = 12;
constexpr int kMaxTerms = 24;

struct Term {
    int8_t a, b;      // tensor-map indices
    int8_t acc;       // accumulator 0 or 1
    int8_t neg;       // subtract this term
    int32_t kblocks;  // number of 64-wide K blocks
};

struct Params {
    CUtensorMap maps[kMaxMaps];
    Term terms[kMaxTerms];
    int nterms;
    int total_kblocks;
    int M, N;
    int kb_per_split;   // K blocks per blockIdx.z layer (split-K); >= every term's kblocks when unsplit
    int *err;
    long long wait;     // cap of every pipeline wait, SM clock cycles
};

template <int BN, int STAGES>
struct Smem {
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int TOTAL = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
    static_assert(8 * (2 * STAGES + 2) + 4 <= 256, "gemm_kernel: barrier area");
};

template <int BN, int NACC, int STAGES, class Epi>
__global__ void __launch_bounds__(192, 1) gemm_kernel(const __grid_constant__ Params p, Epi epi) {
    using S = Smem<BN, STAGES>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned tile area
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(base + STAGES * S::STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *accbar = empty + STAGES;
    uint64_t *donebar = accbar + 1;          // every MMA of this CTA has completed
    uint32_t *tslot = (uint32_t *)(donebar + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    constexpr uint32_t TCOLS = (BN * NACC <= 32) ? 32 : (BN * NACC <= 64) ? 64 : (BN * NACC <= 128) ? 128
                              : (BN * NACC <= 256) ? 256 : 512;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        mbar_init(accbar, 1);
        mbar_init(donebar, 1);
        mbar_fence_init();
    }
    if (warp == 1) tmem_alloc(tslot, TCOLS);
    if (warp == 0 && lane == 0)
        for (int i = 0; i < kMaxMaps; ++i) tma_prefetch_desc(&p.maps[i]);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer
        int it = 0;
        bool ok = true;
        for (int t = 0; t < p.nterms && ok; ++t) {
            const Term tm = p.terms[t];
            const int kb0 = blockIdx.z * p.kb_per_split, kb1 = min(tm.kblocks, kb0 + p.kb_per_split);
            for (int kb = kb0; kb < kb1; ++kb, ++it) {
                const int s = it % STAGES;
                const uint32_t ph = (it / STAGES) & 1;
                if (!mbar_wait(&empty[s], ph ^ 1, p.err, 11, p.wait)) { ok = false; break; }
                unsigned char *sa = base + s * S::STAGE_BYTES;
                unsigned char *sb = sa + S::A_BYTES;
                mbar_expect_tx(&full[s], S::STAGE_BYTES);
                tma_load_2d(sa, &p.maps[tm.a], kb * BK, m0, &full[s]);
                tma_load_2d(sb, &p.maps[tm.b], kb * BK, n0, &full[s]);
            }
        }
        // drain: every issued load must have landed before the CTA may exit
        const int issued = it;
        for (int s = 0; s < STAGES && s < issued; ++s) {
            const int last = issued - 1 - ((issued - 1 - s) % STAGES);
            mbar_drain(&full[s], (last / STAGES) & 1, p.err, 12);
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        int it = 0;
        bool ok = true;
        bool first[2] = {true, true};
        for (int t = 0; t < p.nterms && ok; ++t) {
            const Term tm = p.terms[t];
            const uint32_t idesc = idesc_bf16(BN, tm.neg != 0, false);
            const uint32_t d = tbase + (uint32_t)(tm.acc * BN);
            const int kb0 = blockIdx.z * p.kb_per_split, kb1 = min(tm.kblocks, kb0 + p.kb_per_split);
            for (int kb = kb0; kb < kb1; ++kb, ++it) {
                const int s = it % STAGES;
                const uint32_t ph = (it / STAGES) & 1;
                if (!mbar_wait(&full[s], ph, p.err, 13, p.wait)) { ok = false; break; }
                tc_fence_after();
                unsigned char *sa = base + s * S::STAGE_BYTES;
                unsigned char *sb = sa + S::A_BYTES;
                const uint64_t da = smem_desc_k128(sa), db = smem_desc_k128(sb);
#pragma unroll
                for (int k = 0; k < BK / UMMA_K; ++k) {
                    // advance the start address by k * 32 bytes (encoded >> 4)
                    mma_bf16(d, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), idesc,
                             (first[tm.acc] && k == 0) ? 0u : 1u);
                }
                first[tm.acc] = false;
                mma_commit(&empty[s]);
            }
        }
        mma_commit(accbar);
        mma_commit(donebar);
    } else if (warp >= 2) {
        // ---------------- epilogue
        const bool ok = mbar_wait(accbar, 0, p.err, 14, p.wait);
        tc_fence_after();
        if (ok) {
            const int lb = 32 * (warp & 3);
            const int row = lb + lane;
            float v0[32], v1[32];
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 32) {
                tmem_ld32(tbase + ((uint32_t)lb << 16) + (uint32_t)c0, v0);
                if (NACC == 2) tmem_ld32(tbase + ((uint32_t)lb << 16) + (uint32_t)(BN + c0), v1);
                epi(m0 + row, n0 + c0, v0, v1);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        // no MMA may still write tensor memory when it is freed
        if (lane == 0) mbar_drain(donebar, 0, p.err, 15);
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tbase, TCOLS);
    }
}

// ---- epilogues -------------------------------------------------------------
// real output, column-major: C = alpha * acc0 + beta * C
struct EpiF32 {
    float *C;
    int64_t ldc;
    int M, N;
    float alpha, beta;
    __device__ void operator()(int m, int n0, const float *v0, const float *) const {
        if (m >= M) return;
#pragma unroll 4
        for (int j = 0; j < 32; ++j) {
            int n = n0 + j;
            if (n >= N) break;
            float *c = C + m + (int64_t)n * ldc;
            float o = alpha * v0[j];
            if (beta != 0.f) o += beta * *c;
            *c = o;
        }
    }
};

}  // namespace tc
}  // namespace bdg
