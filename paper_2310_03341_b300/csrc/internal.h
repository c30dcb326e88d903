// Internal declarations shared by the translation units of libbdg.
#pragma once

#include <cuda_bf16.h>
#include <stdarg.h>
#include <stddef.h>
#include <stdint.h>

#include <map>
#include <utility>
#include <vector>

#include "common.cuh"

constexpr long long kDefaultWaitCycles = 4000000000LL;   // ~2 s at 2 GHz

struct bdg_ctx {
    int device = 0;
    int num_sms = 0;
    int smem_optin = 0;
    char err[1024] = {0};
    // workspace arena: one device allocation reused across calls
    char *ws = nullptr;
    size_t ws_bytes = 0;
    size_t ws_top = 0;
    // small persistent device state: barrier + error words
    bdg::GridBarrier *barrier = nullptr;
    int *dflags = nullptr;       // [0]: generic error word of the last kernel group
    // pinned host scalars for results read back
    double *hscal = nullptr;
    int *hflags = nullptr;
    // tuning knobs (set from the environment at creation)
    int band_fp32 = 64;          // stage-1 bandwidth in the FP32/BF16 modes
    int band_fp64 = 32;          // stage-1 bandwidth in the FP64 mode
    int bt2_group = 0;           // sweeps per block reflector in the stage-2 back-transform (0: = band)
    int use_tc = 1;              // tensor-core products in BF16X3 mode
    int last_heev_ph = 0;        // the last bdg_heev used the particle-hole half solve
    int last_heev_prec = -1;     // precision mode of the last bdg_heev (-1: none yet)
    int band_override = 0;       // band width forced by the batched driver (0: default)
    // batched solver: worker contexts (own workspace and stream)
    // and the band width chosen per (precision, order) by its autotuner
    std::vector<bdg_ctx *> workers;
    std::vector<cudaStream_t> worker_streams;
    std::map<std::pair<int, int64_t>, int> batch_band;
    int last_refine_ph = 0;      // the last bdg_refine used the particle-hole reduction
    // cap of every bounded device wait (tensor-core pipeline barriers, the
    // stage-2 sweep dependency), SM clock cycles; bdg_set_wait_limit
    long long wait_cycles = kDefaultWaitCycles;
    // bf16 slices per operand of the refinement's FP64-accurate products, per
    // iteration (the last entry repeats), when set by BDG_REFINE_SLICES
    // (refine_nslices > 0); otherwise the refinement chooses from the target
    // (see refine_impl)
    int refine_slices[8] = {6, 6, 6, 6, 6, 6, 6, 6};
    int refine_nslices = 0;
    // optional per-stage timing (bdg_set_timing): events recorded on the
    // call's stream after each stage, resolved by bdg_stage_times
    int timing = 0;
    long long launches = 0;      // kernel launches issued through this context
    int nstage = 0;
    cudaEvent_t ev[64];
    const char *stage_name[64];
    cudaEvent_t ev0 = nullptr;
};

// record the end of a named stage (no-op unless timing is enabled)
void stage_mark(bdg_ctx *ctx, cudaStream_t st, const char *name);
void stage_begin(bdg_ctx *ctx, cudaStream_t st);

int bdg_fail(bdg_ctx *ctx, int code, const char *fmt, ...);
inline void bdg_count_launch(bdg_ctx *ctx) { if (ctx) ctx->launches++; }

// workspace arena ------------------------------------------------------------
int ws_reserve(bdg_ctx *ctx, size_t bytes);   // grows the arena (synchronises)
void ws_reset(bdg_ctx *ctx);
void *ws_take(bdg_ctx *ctx, size_t bytes);     // 256-byte aligned bump allocation
inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// kernel launchers (return BDG_OK or an error recorded on ctx) ---------------
namespace bdg {

int launch_build(bdg_ctx *ctx, int nx, int ny, int nz, double mu, const double *U,
                 const double2 *Delta, double2 *H, int64_t ldh, double *ktab, cudaStream_t st);
int launch_kinetic_tables(bdg_ctx *ctx, int nx, int ny, int nz, double *ktab, cudaStream_t st);

template <typename R>
int gemm(bdg_ctx *ctx, cudaStream_t st, char opA, char opB, int64_t M, int64_t N, int64_t K,
         cplx<R> alpha, const cplx<R> *A, int64_t lda, const cplx<R> *B, int64_t ldb,
         cplx<R> beta, cplx<R> *C, int64_t ldc);

// C = alpha * op(A) op(B) + beta * C with the K dimension split over `splits`
// CTAs and reduced deterministically through `partial` (splits*M*N entries).
template <typename R>
int gemm_splitk(bdg_ctx *ctx, cudaStream_t st, char opA, char opB, int64_t M, int64_t N,
                int64_t K, cplx<R> alpha, const cplx<R> *A, int64_t lda, const cplx<R> *B,
                int64_t ldb, cplx<R> beta, cplx<R> *C, int64_t ldc, int splits,
                cplx<R> *partial);

struct TriWork {
    double *d, *e, *e2, *w_unsorted, *Y, *Dp, *Dm, *tnorm;
    double2 *Dph;
    int *bstart, *bend, *perm, *pmcount;   // pmcount: 4 ints (the +- counts, the large-cluster count)
    int2 *clist;                           // large clusters (first, end): room for n / 8 + 1
};

// Particle-hole partners: for j < n/2, column n/2-1-j of Z becomes
// (conj v, -conj u) of column n/2+j and w[n/2-1-j] = -w[n/2+j].
template <typename R>
int launch_ph_fill(bdg_ctx *ctx, int64_t n, cplx<R> *Z, int64_t ldz, double *w, cudaStream_t st);

void batch_destroy(bdg_ctx *ctx);

// heev pipeline pieces
template <typename R>
int heev_impl(bdg_ctx *ctx, int64_t n, cplx<R> *A, int64_t lda, double *w, cplx<R> *Z,
              int64_t ldz, int band, int tensor, cudaStream_t st, bool want_ph = false);
size_t heev_workspace_bytes(int64_t n, int band, int elem_bytes, int group, int slices);

int launch_convert_z64_to_z32(bdg_ctx *ctx, int64_t rows, int64_t cols, const double2 *src,
                              int64_t lds, float2 *dst, int64_t ldd, cudaStream_t st);
int launch_convert_z32_to_z64(bdg_ctx *ctx, int64_t rows, int64_t cols, const float2 *src,
                              int64_t lds, double2 *dst, int64_t ldd, cudaStream_t st);

// refinement / densities
size_t refine_workspace_bytes(int64_t n);
int refine_impl(bdg_ctx *ctx, const bdg_grid *g, double mu, const double *U, const double2 *Delta,
                int64_t n, double *w, double2 *Z, int64_t ldz, int max_iter, double tol,
                double *resid_out, double *orth_out, int *iters_out, cudaStream_t st);
int densities_impl(bdg_ctx *ctx, const bdg_grid *g, int64_t n, const double *w, const double2 *Z,
                   int64_t ldz, double T, double Ec, double *n_out, double2 *nu_out,
                   cudaStream_t st);
int tau_j_impl(bdg_ctx *ctx, const bdg_grid *g, int64_t n, const double *w, const double2 *Z,
               int64_t ldz, double T, double Ec, double *tau_out, double *j_out, cudaStream_t st);
int td_evolve_impl(bdg_ctx *ctx, const bdg_grid *g, const bdg_td_params *p, int64_t nq, const double *E0,
                   double2 *Psi, int64_t ldpsi, int nsteps, double *n_out, double2 *nu_out, cudaStream_t st);
int scf_update_impl(bdg_ctx *ctx, int64_t V, const bdg_scf_params *p, const double *n,
                    const double2 *nu, double *U, double2 *Delta, double *dn_max_dev,
                    cudaStream_t st);

// tensor-core products
int tc_available(bdg_ctx *ctx);

// Planes used by the tensor-core products of stage 1 and its
// back-transformation (nullptr members: SIMT path).  S = 2, 3: the
// split-precision products (hi/lo bf16 slices, FP32 accumulation in tensor
// memory); S = kExactSlices: the exact-slice FP32-accurate products
// (xs_slice / xs_product), which also use the chunk exponent arrays.
constexpr int kExactSlices = 9;
struct TcPlanes {
    __nv_bfloat16 *big;    // planes of an n x n (A22) or n x ncols (E slab) operand
    __nv_bfloat16 *skA;    // planes of a narrow A operand
    __nv_bfloat16 *skB;    // planes of a narrow B operand
    float2 *part;          // split-K partials (S = 2, 3)
    int S;
    int num_sms;
    int *ebig, *eA, *eB;   // chunk exponents (exact mode)
    float2 *vagg;          // exact mode: n x 2b block reflector of two stage-1 panels
    float2 *tagg;          // exact mode: its 2b x 2b T factor, then two b x b scratch blocks
};

// exact-slice FP32-accurate complex products on the tensor cores (xs_gemm.cu)
int64_t xs_kpad(int64_t K);
size_t xs_plane_bytes(int64_t K, int64_t C, bool bop);
size_t xs_exp_bytes(int64_t K, int64_t C);
int xs_slice(bdg_ctx *ctx, cudaStream_t st, int64_t K, int64_t C, const float2 *src, int64_t sk, int64_t sc,
             bool conj_, bool bop, __nv_bfloat16 *planes, int *ex);
int xs_product(bdg_ctx *ctx, cudaStream_t st, int64_t K, int64_t M, int64_t N, const __nv_bfloat16 *px,
               const int *ex, const __nv_bfloat16 *py, const int *ey, float2 *C, int64_t ldc, float alpha,
               float beta, bool lower);

}  // namespace bdg
