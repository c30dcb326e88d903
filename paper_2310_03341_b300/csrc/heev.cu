// bdg_heev pipeline: dense -> band (stage 1) -> tridiagonal (stage 2) ->
// FP64 tridiagonal eigenpairs -> back-transformation through stage 2 and
// stage 1 (paper, section "Performance of the Matrix Diagonalization
// Algorithm", the 2-stage solver).
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace bdg {

template <typename R>
int stage1_reduce(bdg_ctx *ctx, cudaStream_t st, int64_t n, int b, cplx<R> *A, int64_t lda, cplx<R> *Bnd,
                  int ldband, cplx<R> *Vst, const int64_t *voff, cplx<R> *Tst, R *taust, cplx<R> *VWV,
                  cplx<R> *Ytmp, cplx<R> *Msmall, cplx<R> *Psmall, cplx<R> *red, cplx<R> *splitws, int npanels,
                  const TcPlanes *tcp);
template <typename R>
int stage1_backtransform(bdg_ctx *ctx, cudaStream_t st, int64_t n, int b, int npanels, const cplx<R> *Vst,
                         const int64_t *voff, const cplx<R> *Tst, cplx<R> *E, int64_t lde, int64_t ncols,
                         cplx<R> *W1, cplx<R> *W2, cplx<R> *splitws, const TcPlanes *tcp);
template <typename R>
int stage2_reduce(bdg_ctx *ctx, cudaStream_t st, int64_t n, int b, int g, cplx<R> *band, int ldband,
                  cplx<R> *refl, R *taus, const int64_t *grp_off_dev, unsigned int *ticket, int *progress,
                  int64_t nrefl_slots);
template <typename R>
int stage2_backtransform(bdg_ctx *ctx, cudaStream_t st, int64_t n, int b, int g, const cplx<R> *refl,
                         const R *taus, const int64_t *grp_off_dev, const int64_t *blk_list_dev, int64_t nblk,
                         const int64_t *blk_off_dev, cplx<R> *Tst, cplx<R> *E, int64_t lde, int64_t ncols);
template <typename R>
int tridiag_solve(bdg_ctx *ctx, cudaStream_t st, int64_t n, const cplx<R> *band, int ldband, const TriWork &tw,
                  double *w_sorted, cplx<R> *E, int64_t lde, double ctol_rel, bool want_ph, int *used_ph);

static inline int64_t steps_of(int64_t n, int b, int64_t s) {
    if (s > n - 3) return 0;
    return (n - s - 3) / b + 1;
}

// Workspace plan shared by the size query and the solver.
struct Plan {
    int64_t n;
    int b, g, ldband, npanels;
    int64_t ngroups, nslots, nblk, vtotal;
    std::vector<int64_t> voff, grp_off, blk_list, blk_off;
    size_t bytes = 0;
    // offsets into the arena
    size_t o_A32, o_Vst, o_Tst, o_tau1, o_VWV, o_Ytmp, o_M, o_P, o_red, o_split, o_band, o_refl, o_tau2,
        o_grpoff, o_blkoff, o_blk, o_bt2T, o_ticket, o_pm, o_prog, o_d, o_e, o_e2, o_wu, o_Dph, o_bs, o_be, o_perm, o_tn, o_cl, o_Y,
        o_Dp, o_Dm, o_E, o_W1, o_W2, o_pbig, o_pska, o_pskb, o_part, o_ebig, o_eA, o_eB, o_vagg, o_tagg;
    int slices = 0;
};

static void make_plan(Plan &p, int64_t n, int b, int g, int elem, bool separate_A, bool separate_E,
                      int num_sms, int slices) {
    p.n = n; p.b = b; p.g = g; p.ldband = 2 * b + 1;
    p.voff.clear(); p.grp_off.clear(); p.blk_list.clear(); p.blk_off.clear();
    p.npanels = 0;
    p.vtotal = 0;
    for (int64_t c0 = 0;; c0 += b) {
        int64_t m = n - c0 - b;
        if (m <= 0) break;
        p.voff.push_back(p.vtotal);
        p.vtotal += m * b;
        p.npanels++;
    }
    p.ngroups = n >= 3 ? (n - 2 + g - 1) / g : 0;
    p.nslots = 0;
    p.nblk = 0;
    for (int64_t J = 0; J < p.ngroups; ++J) {
        p.grp_off.push_back(p.nslots);
        p.blk_off.push_back(p.nblk);
        int64_t ns = steps_of(n, b, J * g);
        p.nslots += ns * g;
        for (int64_t k = 0; k < ns; ++k) { p.blk_list.push_back(J); p.blk_list.push_back(k); }
        p.nblk += ns;
    }
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += align_up(bytes); return o; };
    const size_t nn = (size_t)n * n;
    p.o_A32 = separate_A ? take(nn * elem) : 0;
    p.o_Vst = take((size_t)std::max<int64_t>(p.vtotal, 1) * elem);
    p.o_Tst = take((size_t)std::max(p.npanels, 1) * b * b * elem);
    p.o_tau1 = take((size_t)std::max(p.npanels, 1) * b * (elem / 2));
    p.o_VWV = take((size_t)n * 3 * b * elem);
    p.o_Ytmp = take((size_t)n * b * elem);
    p.o_M = take((size_t)b * b * elem);
    p.o_P = take((size_t)b * b * elem);
    p.o_red = take(((size_t)num_sms * (2 + 2 * (size_t)b + (size_t)b * b) + (size_t)b * b + 2 * (size_t)b + 2) *
                   elem);
    p.o_split = take((size_t)64 * b * b * elem);
    p.o_band = take((size_t)p.ldband * n * elem);
    p.o_refl = take((size_t)std::max<int64_t>(p.nslots, 1) * b * elem);
    p.o_tau2 = take((size_t)std::max<int64_t>(p.nslots, 1) * (elem / 2));
    p.o_grpoff = take((size_t)std::max<int64_t>(p.ngroups, 1) * sizeof(int64_t));
    p.o_blkoff = take((size_t)std::max<int64_t>(p.ngroups, 1) * sizeof(int64_t));
    p.o_blk = take((size_t)std::max<int64_t>(2 * p.nblk, 2) * sizeof(int64_t));
    p.o_bt2T = take((size_t)std::max<int64_t>(p.nblk, 1) * (g + b - 1) * g * elem);
    p.o_ticket = take(sizeof(unsigned int));
    p.o_pm = take(4 * sizeof(int));
    p.o_prog = take((size_t)n * sizeof(int));
    p.o_d = take((size_t)n * 8);
    p.o_e = take((size_t)n * 8);
    p.o_e2 = take((size_t)n * 8);
    p.o_wu = take((size_t)n * 8);
    p.o_Dph = take((size_t)n * 16);
    p.o_bs = take((size_t)n * 4);
    p.o_be = take((size_t)n * 4);
    p.o_perm = take((size_t)n * 4);
    p.o_tn = take(8);
    p.o_cl = take(((size_t)n / 8 + 1) * sizeof(int2));
    p.o_Y = take(nn * 8);
    p.o_Dp = take(nn * 8);
    p.o_Dm = take(nn * 8);
    p.o_E = separate_E ? take(nn * elem) : 0;
    // the exact-slice back-transform applies two panels at a time: W1, W2 hold n x 2b
    const size_t wcols = (slices == kExactSlices) ? 2 * (size_t)b : (size_t)b;
    p.o_W1 = take(wcols * n * elem);
    p.o_W2 = take(wcols * n * elem);
    p.slices = slices;
    if (slices == kExactSlices) {
        // exact-slice products: X planes of A22 (n x n) or of the E slab, the
        // narrow operands of the rank-2b update and of the back-transform
        p.o_pbig = take(xs_plane_bytes(n, n, false));
        p.o_pska = take(std::max(xs_plane_bytes(2 * b, n, false), xs_plane_bytes(b, n, false)));
        p.o_pskb = take(std::max({xs_plane_bytes(n, 2 * b, true), xs_plane_bytes(2 * b, n, true),
                                  xs_plane_bytes(b, n, true)}));
        p.o_ebig = take(xs_exp_bytes(n, n));
        p.o_eA = take(std::max(xs_exp_bytes(2 * b, n), xs_exp_bytes(b, n)));
        p.o_eB = take(std::max({xs_exp_bytes(n, 2 * b), xs_exp_bytes(2 * b, n), xs_exp_bytes(b, n)}));
        p.o_vagg = take((size_t)n * 2 * b * 8);
        p.o_tagg = take((size_t)6 * b * b * 8);
        p.o_part = 0;
    } else if (slices) {
        // up to 3 slices x (re, im) planes
        const size_t npad = (size_t)((n + 63) / 64) * 64 + 64;
        p.o_pbig = take((size_t)6 * npad * n * 2);
        p.o_pska = take((size_t)6 * npad * (2 * b + 64) * 2);
        p.o_pskb = take((size_t)6 * npad * (2 * b + 64) * 2);
        p.o_part = take((size_t)8 * npad * 64 * 8);
    }
    p.bytes = off;
}

size_t heev_workspace_bytes(int64_t n, int band, int elem_bytes, int group, int slices) {
    // the solver may shrink the back-transformation group to fit shared
    // memory; take the largest plan over the candidate group sizes
    size_t best = 0;
    for (int g = std::max(group > 0 ? std::min(group, 64) : band, 8); g >= 8; g /= 2) {
        Plan p;
        make_plan(p, n, band, g, elem_bytes, false, false, 160, slices);
        best = std::max(best, p.bytes);
    }
    return best + 4096;
}

template <typename R>
int heev_impl(bdg_ctx *ctx, int64_t n, cplx<R> *A, int64_t lda, double *w, cplx<R> *Z, int64_t ldz, int band,
              int tensor, cudaStream_t st, bool want_ph) {
    if (sizeof(R) == 8) tensor = 0;   // the FP64 path has no tensor-core products
    using Cx = cplx<R>;
    const int b = band;
    // sweeps per block reflector of the stage-2 back-transformation: the
    // apply kernel keeps V ((g+b-1) x g), T (g x g) and a (g+b-1) x 32 slab
    // of E in shared memory
    int g = ctx->bt2_group > 0 ? std::min(ctx->bt2_group, 64) : b;
    auto bt2_smem = [&](int gg) {
        const size_t mrp = (size_t)((gg + b - 1 + 7) / 8) * 8;
        return (mrp * 64 + (size_t)gg * b + mrp * gg + (size_t)gg * 64) * sizeof(Cx);
    };
    while (g > 8 && bt2_smem(g) > (size_t)ctx->smem_optin) g /= 2;
    Plan p;
    make_plan(p, n, b, g, (int)sizeof(Cx), false, false, ctx->num_sms, tensor);
    int rc = BDG_OK;
    char *base = (char *)ws_take(ctx, p.bytes);
    if (!base) return bdg_fail(ctx, BDG_ENOMEM, "heev: workspace arena too small (%zu bytes needed)", p.bytes);
    auto P_ = [&](size_t o) { return (void *)(base + o); };
    Cx *Vst = (Cx *)P_(p.o_Vst);
    Cx *Tst = (Cx *)P_(p.o_Tst);
    R *tau1 = (R *)P_(p.o_tau1);
    Cx *VWV = (Cx *)P_(p.o_VWV);
    Cx *Ytmp = (Cx *)P_(p.o_Ytmp);
    Cx *Mm = (Cx *)P_(p.o_M);
    Cx *Pm = (Cx *)P_(p.o_P);
    Cx *red = (Cx *)P_(p.o_red);
    Cx *splitws = (Cx *)P_(p.o_split);
    Cx *bandp = (Cx *)P_(p.o_band);
    Cx *refl = (Cx *)P_(p.o_refl);
    R *tau2 = (R *)P_(p.o_tau2);
    int64_t *grpoff = (int64_t *)P_(p.o_grpoff);
    int64_t *blk = (int64_t *)P_(p.o_blk);
    int64_t *blkoff = (int64_t *)P_(p.o_blkoff);
    Cx *bt2T = (Cx *)P_(p.o_bt2T);
    unsigned int *ticket = (unsigned int *)P_(p.o_ticket);
    int *prog = (int *)P_(p.o_prog);
    TriWork tw;
    tw.d = (double *)P_(p.o_d); tw.e = (double *)P_(p.o_e); tw.e2 = (double *)P_(p.o_e2);
    tw.w_unsorted = (double *)P_(p.o_wu); tw.Dph = (double2 *)P_(p.o_Dph);
    tw.bstart = (int *)P_(p.o_bs); tw.bend = (int *)P_(p.o_be); tw.perm = (int *)P_(p.o_perm);
    tw.tnorm = (double *)P_(p.o_tn); tw.Y = (double *)P_(p.o_Y); tw.Dp = (double *)P_(p.o_Dp);
    tw.Dm = (double *)P_(p.o_Dm);
    tw.pmcount = (int *)P_(p.o_pm);
    tw.clist = (int2 *)P_(p.o_cl);
    Cx *W1 = (Cx *)P_(p.o_W1), *W2 = (Cx *)P_(p.o_W2);
    TcPlanes tcp_s{nullptr, nullptr, nullptr, nullptr, 0, ctx->num_sms, nullptr, nullptr, nullptr, nullptr, nullptr};
    const TcPlanes *tcp = nullptr;
    if (tensor) {
        tcp_s.big = (__nv_bfloat16 *)P_(p.o_pbig);
        tcp_s.skA = (__nv_bfloat16 *)P_(p.o_pska);
        tcp_s.skB = (__nv_bfloat16 *)P_(p.o_pskb);
        tcp_s.S = tensor;   // slices per operand, or kExactSlices
        if (tensor == kExactSlices) {
            tcp_s.ebig = (int *)P_(p.o_ebig);
            tcp_s.eA = (int *)P_(p.o_eA);
            tcp_s.eB = (int *)P_(p.o_eB);
            tcp_s.vagg = (float2 *)P_(p.o_vagg);
            tcp_s.tagg = (float2 *)P_(p.o_tagg);
        } else {
            tcp_s.part = (float2 *)P_(p.o_part);
        }
        tcp = &tcp_s;
    }

    if (n == 1) {
        // 1 x 1: eigenvalue Re(a), eigenvector 1
        Cx one = mk<R>(1, 0);
        BDG_CUDA_TRY(ctx, cudaMemcpyAsync(Z, &one, sizeof(Cx), cudaMemcpyHostToDevice, st));
        // w[0] = Re A[0]
        R a[2];
        BDG_CUDA_TRY(ctx, cudaMemcpyAsync(a, A, sizeof(Cx), cudaMemcpyDeviceToHost, st));
        BDG_CUDA_TRY(ctx, cudaStreamSynchronize(st));
        double wv = (double)a[0];
        BDG_CUDA_TRY(ctx, cudaMemcpyAsync(w, &wv, sizeof(double), cudaMemcpyHostToDevice, st));
        BDG_CUDA_TRY(ctx, cudaStreamSynchronize(st));
        return BDG_OK;
    }
    BDG_CUDA_TRY(ctx, cudaMemcpyAsync(grpoff, p.grp_off.data(), p.grp_off.size() * sizeof(int64_t),
                                      cudaMemcpyHostToDevice, st));
    BDG_CUDA_TRY(ctx, cudaMemcpyAsync(blk, p.blk_list.data(), p.blk_list.size() * sizeof(int64_t),
                                      cudaMemcpyHostToDevice, st));
    BDG_CUDA_TRY(ctx, cudaMemcpyAsync(blkoff, p.blk_off.data(), p.blk_off.size() * sizeof(int64_t),
                                      cudaMemcpyHostToDevice, st));
    // ---- stage 1
    rc = stage1_reduce<R>(ctx, st, n, b, A, lda, bandp, p.ldband, Vst, p.voff.data(), Tst, tau1, VWV, Ytmp, Mm,
                          Pm, red, splitws, p.npanels, tcp);
    if (rc) return rc;
    stage_mark(ctx, st, "stage1_band");
    // ---- stage 2
    rc = stage2_reduce<R>(ctx, st, n, b, g, bandp, p.ldband, refl, tau2, grpoff, ticket, prog, p.nslots);
    if (rc) return rc;
    stage_mark(ctx, st, "stage2_bulge");
    // ---- tridiagonal eigenpairs, E = D Y(:, perm) into Z
    // cluster tolerance of the inverse iteration (relative to ||T||): in FP64
    // mode it sets the orthogonality of the result (eps ||T|| / gap for
    // eigenvalues outside clusters); in the reduced-precision modes the
    // refinement restores orthogonality, so only near-coincident eigenvalues
    // are grouped
    const double ctol_rel = (sizeof(R) == 8) ? 1e-6 : 1e-10;
    // particle-hole half solve: the vectors of the upper half of the
    // spectrum go to Z[:, n/2 ..]; the rest follows from the symmetry
    int ph = 0;
    rc = tridiag_solve<R>(ctx, st, n, bandp, p.ldband, tw, w, Z, ldz, ctol_rel, want_ph, &ph);
    if (rc) return rc;
    ctx->last_heev_ph = ph;
    const int64_t c0 = ph ? n / 2 : 0, ncols = n - c0;
    // bounded-wait status of stage 1 and stage 2 (checked after the host sync inside tridiag_solve)
    int flags[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    BDG_CUDA_TRY(ctx, cudaMemcpyAsync(flags, ctx->dflags, sizeof(flags), cudaMemcpyDeviceToHost, st));
    BDG_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    if (flags[0]) return bdg_fail(ctx, BDG_ETIMEOUT, "stage-2 bulge chasing: a bounded wait gave up (code %d)",
                                  flags[0]);
    for (int i = 4; i < 8; ++i)
        if (flags[i])
            return bdg_fail(ctx, BDG_ETIMEOUT, "stage 1: a tensor-core pipeline wait gave up (code %d)", flags[i]);
    stage_mark(ctx, st, "tridiagonal");
    // ---- back-transformation: Z <- Q1 Q2 Z
    Cx *Zc = Z + c0 * ldz;
    rc = stage2_backtransform<R>(ctx, st, n, b, g, refl, tau2, grpoff, blk, p.nblk, blkoff, bt2T, Zc, ldz, ncols);
    if (rc) return rc;
    stage_mark(ctx, st, "backtransform2");
    rc = stage1_backtransform<R>(ctx, st, n, b, p.npanels, Vst, p.voff.data(), Tst, Zc, ldz, ncols, W1, W2,
                                 splitws, tcp);
    if (rc) return rc;
    stage_mark(ctx, st, "backtransform1");
    if (ph) {
        rc = launch_ph_fill<R>(ctx, n, Z, ldz, w, st);
        if (rc) return rc;
        stage_mark(ctx, st, "ph_partners");
    }
    return BDG_OK;
}

template int heev_impl<float>(bdg_ctx *, int64_t, float2 *, int64_t, double *, float2 *, int64_t, int, int,
                              cudaStream_t, bool);
template int heev_impl<double>(bdg_ctx *, int64_t, double2 *, int64_t, double *, double2 *, int64_t, int, int,
                               cudaStream_t, bool);

// ---------------------------------------------------------------------------
// particle-hole partners (see launch_ph_fill)
// ---------------------------------------------------------------------------
template <typename R>
__global__ void ph_fill_kernel(int64_t n, cplx<R> *__restrict__ Z, int64_t ldz, double *__restrict__ w) {
    const int64_t h = n / 2;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * h) return;
    const int64_t r = idx % n, j = idx / n;
    const cplx<R> *src = Z + (h + j) * ldz;
    cplx<R> *dst = Z + (h - 1 - j) * ldz;
    // (u, v) -> (conj v, -conj u)
    if (r < h) {
        const cplx<R> v = src[r + h];
        dst[r] = mk<R>(v.x, -v.y);
    } else {
        const cplx<R> u = src[r - h];
        dst[r] = mk<R>(-u.x, u.y);
    }
    if (r == 0) w[h - 1 - j] = -w[h + j];
}

template <typename R>
int launch_ph_fill(bdg_ctx *ctx, int64_t n, cplx<R> *Z, int64_t ldz, double *w, cudaStream_t st) {
    const int64_t tot = n * (n / 2);
    ph_fill_kernel<R><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, Z, ldz, w);
    BDG_LAUNCH_CHECK(ctx);
    return BDG_OK;
}
template int launch_ph_fill<float>(bdg_ctx *, int64_t, float2 *, int64_t, double *, cudaStream_t);
template int launch_ph_fill<double>(bdg_ctx *, int64_t, double2 *, int64_t, double *, cudaStream_t);

// ---------------------------------------------------------------------------
// precision conversions
// ---------------------------------------------------------------------------
__global__ void z64_to_z32_kernel(int64_t rows, int64_t cols, const double2 *__restrict__ s, int64_t lds,
                                  float2 *__restrict__ d, int64_t ldd) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    int64_t r = idx % rows, c = idx / rows;
    double2 v = s[r + c * lds];
    d[r + c * ldd] = make_float2((float)v.x, (float)v.y);
}
__global__ void z32_to_z64_kernel(int64_t rows, int64_t cols, const float2 *__restrict__ s, int64_t lds,
                                  double2 *__restrict__ d, int64_t ldd) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    int64_t r = idx % rows, c = idx / rows;
    float2 v = s[r + c * lds];
    d[r + c * ldd] = make_double2((double)v.x, (double)v.y);
}
int launch_convert_z64_to_z32(bdg_ctx *ctx, int64_t rows, int64_t cols, const double2 *src, int64_t lds,
                              float2 *dst, int64_t ldd, cudaStream_t st) {
    int64_t tot = rows * cols;
    z64_to_z32_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(rows, cols, src, lds, dst, ldd);
    BDG_LAUNCH_CHECK(ctx);
    return BDG_OK;
}
int launch_convert_z32_to_z64(bdg_ctx *ctx, int64_t rows, int64_t cols, const float2 *src, int64_t lds,
                              double2 *dst, int64_t ldd, cudaStream_t st) {
    int64_t tot = rows * cols;
    z32_to_z64_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(rows, cols, src, lds, dst, ldd);
    BDG_LAUNCH_CHECK(ctx);
    return BDG_OK;
}

}  // namespace bdg
