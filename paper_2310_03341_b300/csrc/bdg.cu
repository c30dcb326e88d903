// C-ABI entry points of libbdg (declared in include/bdg.h): context and
// workspace management, argument checking, precision dispatch.
#include <stdarg.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

int bdg_fail(bdg_ctx *ctx, int code, const char *fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

int ws_reserve(bdg_ctx *ctx, size_t bytes) {
    ctx->ws_top = 0;
    if (bytes <= ctx->ws_bytes) return BDG_OK;
    if (ctx->ws) {
        cudaDeviceSynchronize();
        cudaFree(ctx->ws);
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
    }
    size_t want = align_up(bytes, 1 << 20);
    cudaError_t e = cudaMalloc((void **)&ctx->ws, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->ws = nullptr;
        return bdg_fail(ctx, BDG_ENOMEM, "workspace: cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e));
    }
    ctx->ws_bytes = want;
    return BDG_OK;
}

void ws_reset(bdg_ctx *ctx) { ctx->ws_top = 0; }

void *ws_take(bdg_ctx *ctx, size_t bytes) {
    size_t b = align_up(bytes);
    if (ctx->ws_top + b > ctx->ws_bytes) return nullptr;
    void *p = ctx->ws + ctx->ws_top;
    ctx->ws_top += b;
    return p;
}

void stage_begin(bdg_ctx *ctx, cudaStream_t st) {
    if (!ctx->timing) return;
    ctx->nstage = 0;
    if (!ctx->ev0) {
        cudaEventCreate(&ctx->ev0);
        for (int i = 0; i < 64; ++i) cudaEventCreate(&ctx->ev[i]);
    }
    cudaEventRecord(ctx->ev0, st);
}

void stage_mark(bdg_ctx *ctx, cudaStream_t st, const char *name) {
    if (!ctx->timing || ctx->nstage >= 64) return;
    ctx->stage_name[ctx->nstage] = name;
    cudaEventRecord(ctx->ev[ctx->nstage], st);
    ctx->nstage++;
}

static int env_int(const char *name, int dflt) {
    const char *v = getenv(name);
    return v ? atoi(v) : dflt;
}

extern "C" {

int bdg_create(int device, bdg_ctx **out) {
    if (!out) return BDG_EINVAL;
    *out = nullptr;
    bdg_ctx *ctx = new (std::nothrow) bdg_ctx();
    if (!ctx) return BDG_ENOMEM;
    ctx->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&ctx->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->barrier, sizeof(bdg::GridBarrier));
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->dflags, 16 * sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&ctx->hscal, 64 * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&ctx->hflags, 16 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->dflags, 0, 16 * sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return BDG_ECUDA;
    }
    ctx->band_fp32 = env_int("BDG_BAND_FP32", 64);
    ctx->band_fp64 = env_int("BDG_BAND_FP64", 32);
    ctx->bt2_group = env_int("BDG_BT2_GROUP", 0);
    ctx->use_tc = env_int("BDG_USE_TC", 1);
    if (const char *sl = getenv("BDG_REFINE_SLICES")) {
        // comma-separated slices per refinement iteration, each 4, 5 or 6
        int k = 0;
        for (const char *q = sl; *q && k < 8;) {
            const int v = atoi(q);
            if (v >= 4 && v <= 6) ctx->refine_slices[k++] = v;
            while (*q && *q != ',') ++q;
            if (*q == ',') ++q;
        }
        if (k > 0) ctx->refine_nslices = k;
    }
    *out = ctx;
    return BDG_OK;
}

void bdg_destroy(bdg_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->barrier) cudaFree(ctx->barrier);
    if (ctx->dflags) cudaFree(ctx->dflags);
    if (ctx->hscal) cudaFreeHost(ctx->hscal);
    if (ctx->hflags) cudaFreeHost(ctx->hflags);
    bdg::batch_destroy(ctx);
    delete ctx;
}

const char *bdg_last_error(bdg_ctx *ctx) { return ctx ? ctx->err : "null context"; }

int bdg_last_modes(bdg_ctx *ctx, int *heev_ph, int *refine_ph) {
    if (!ctx) return BDG_EINVAL;
    if (heev_ph) *heev_ph = ctx->last_heev_ph;
    if (refine_ph) *refine_ph = ctx->last_refine_ph;
    return BDG_OK;
}

int bdg_launch_count(bdg_ctx *ctx, long long *count) {
    if (!ctx || !count) return BDG_EINVAL;
    long long sub = 0;
    for (bdg_ctx *wk : ctx->workers) sub += wk->launches;
    *count = ctx->launches + sub;
    return BDG_OK;
}

int bdg_set_wait_limit(bdg_ctx *ctx, long long cycles) {
    if (!ctx || cycles < 0) return BDG_EINVAL;
    ctx->wait_cycles = cycles > 0 ? cycles : kDefaultWaitCycles;
    return BDG_OK;
}

int bdg_set_timing(bdg_ctx *ctx, int enable) {
    if (!ctx) return BDG_EINVAL;
    ctx->timing = enable ? 1 : 0;
    ctx->nstage = 0;
    return BDG_OK;
}

int bdg_stage_times(bdg_ctx *ctx, int max_stages, double *ms, const char **names, int *count) {
    if (!ctx || !count || max_stages < 0) return BDG_EINVAL;
    *count = 0;
    if (!ctx->timing || !ctx->ev0) return BDG_OK;
    cudaEvent_t prev = ctx->ev0;
    int n = ctx->nstage < max_stages ? ctx->nstage : max_stages;
    for (int i = 0; i < n; ++i) {
        float t = 0.f;
        if (cudaEventSynchronize(ctx->ev[i]) != cudaSuccess || cudaEventElapsedTime(&t, prev, ctx->ev[i]) != cudaSuccess) {
            cudaGetLastError();
            return bdg_fail(ctx, BDG_ECUDA, "stage timing: event query failed");
        }
        if (ms) ms[i] = t;
        if (names) names[i] = ctx->stage_name[i];
        prev = ctx->ev[i];
    }
    *count = n;
    return BDG_OK;
}

static int check_grid(bdg_ctx *ctx, const bdg_grid *g) {
    if (!g) return bdg_fail(ctx, BDG_EINVAL, "grid is NULL");
    if (g->nx < 2 || g->ny < 1 || g->nz < 1)
        return bdg_fail(ctx, BDG_EINVAL, "grid %dx%dx%d: sizes must be >= 1 (nx >= 2)", g->nx, g->ny, g->nz);
    if ((g->nx & 1) || (g->ny > 1 && (g->ny & 1)) || (g->nz > 1 && (g->nz & 1)))
        return bdg_fail(ctx, BDG_EINVAL, "grid %dx%dx%d: sizes must be even (or 1)", g->nx, g->ny, g->nz);
    if (g->dx != 1.0) return bdg_fail(ctx, BDG_EINVAL, "grid spacing dx must be 1 (got %g)", g->dx);
    return BDG_OK;
}

int bdg_build(bdg_ctx *ctx, const bdg_grid *grid, double mu, const double *U, const double2 *Delta, double2 *H,
              int64_t ldh, cudaStream_t stream) {
    if (!ctx) return BDG_EINVAL;
    int rc = check_grid(ctx, grid);
    if (rc) return rc;
    const int64_t N = 2LL * grid->nx * grid->ny * grid->nz;
    if (!U || !Delta || !H) return bdg_fail(ctx, BDG_EINVAL, "bdg_build: null pointer");
    if (ldh < N) return bdg_fail(ctx, BDG_EINVAL, "bdg_build: ldh=%lld < N=%lld", (long long)ldh, (long long)N);
    cudaSetDevice(ctx->device);
    rc = ws_reserve(ctx, 4096);
    if (rc) return rc;
    double *ktab = (double *)ws_take(ctx, sizeof(double) * (grid->nx + grid->ny + grid->nz));
    return bdg::launch_build(ctx, grid->nx, grid->ny, grid->nz, mu, U, Delta, H, ldh, ktab, stream);
}

// bf16 slices per operand of the tensor-core products for a precision mode
// (0: SIMT FP32 products)
static int tc_slices(bdg_ctx *ctx, int prec) {
    if (!ctx->use_tc) return 0;
    if (prec == BDG_PREC_BF16X3) return 2;
    if (prec == BDG_PREC_BF16X6) return 3;
    if (prec == BDG_PREC_BF16X9) return bdg::kExactSlices;
    return 0;
}

static int band_for(bdg_ctx *ctx, int prec, int64_t n) {
    int b = (prec == BDG_PREC_FP64) ? ctx->band_fp64 : ctx->band_fp32;
    if (ctx->band_override > 0) b = ctx->band_override;
    if (b > 64) b = 64;
    if (b < 2) b = 2;
    if (n <= 2 * b && n > 4) b = std::max<int>(2, (int)(n / 4));
    return b;
}

int bdg_heev_workspace(bdg_ctx *ctx, int64_t n, int prec, size_t *bytes) {
    if (!ctx || !bytes || n < 1) return BDG_EINVAL;
    int b = band_for(ctx, prec, n);
    if (prec == BDG_PREC_FP64) {
        *bytes = bdg::heev_workspace_bytes(n, b, 16, ctx->bt2_group, 0);
    } else {
        *bytes = bdg::heev_workspace_bytes(n, b, 8, ctx->bt2_group, tc_slices(ctx, prec)) +
                 2 * align_up((size_t)n * n * 8);
    }
    return BDG_OK;
}

int bdg_heev(bdg_ctx *ctx, int64_t n, double2 *A, int64_t lda, double *w, double2 *Z, int64_t ldz, int prec,
             cudaStream_t stream) {
    if (!ctx) return BDG_EINVAL;
    const bool ph = (prec & BDG_HEEV_PH) != 0;
    prec &= ~BDG_HEEV_PH;
    if (ph && (n % 2) != 0) return bdg_fail(ctx, BDG_EINVAL, "bdg_heev: BDG_HEEV_PH needs an even order");
    if (n < 1 || !A || !w || !Z) return bdg_fail(ctx, BDG_EINVAL, "bdg_heev: bad arguments (n=%lld)", (long long)n);
    if (lda < n || ldz < n) return bdg_fail(ctx, BDG_EINVAL, "bdg_heev: lda/ldz < n");
    if (prec != BDG_PREC_FP64 && prec != BDG_PREC_FP32 && prec != BDG_PREC_BF16X3 && prec != BDG_PREC_BF16X6 &&
        prec != BDG_PREC_BF16X9)
        return bdg_fail(ctx, BDG_EINVAL, "bdg_heev: unknown precision %d", prec);
    if (n > 2147483647LL / 2) return bdg_fail(ctx, BDG_EUNSUPPORTED, "bdg_heev: n too large");
    cudaSetDevice(ctx->device);
    ctx->err[0] = 0;
    size_t bytes = 0;
    bdg_heev_workspace(ctx, n, prec, &bytes);
    int rc = ws_reserve(ctx, bytes);
    if (rc) return rc;
    const int b = band_for(ctx, prec, n);
    ctx->last_heev_prec = prec;
    // the error words of the bounded waits start clear for every call
    BDG_CUDA_TRY(ctx, cudaMemsetAsync(ctx->dflags, 0, 16 * sizeof(int), stream));
    stage_begin(ctx, stream);
    if (prec == BDG_PREC_FP64) {
        return bdg::heev_impl<double>(ctx, n, A, lda, w, Z, ldz, b, 0, stream, ph);
    }
    float2 *A32 = (float2 *)ws_take(ctx, (size_t)n * n * 8);
    float2 *E32 = (float2 *)ws_take(ctx, (size_t)n * n * 8);
    rc = bdg::launch_convert_z64_to_z32(ctx, n, n, A, lda, A32, n, stream);
    if (rc) return rc;
    stage_mark(ctx, stream, "convert_in");
    rc = bdg::heev_impl<float>(ctx, n, A32, n, w, E32, n, b, tc_slices(ctx, prec), stream, ph);
    if (rc) return rc;
    rc = bdg::launch_convert_z32_to_z64(ctx, n, n, E32, n, Z, ldz, stream);
    stage_mark(ctx, stream, "convert_out");
    return rc;
}

int bdg_refine(bdg_ctx *ctx, const bdg_grid *grid, double mu, const double *U, const double2 *Delta, int64_t n,
               double *w, double2 *Z, int64_t ldz, int max_iter, double tol, double *resid_out, double *orth_out,
               int *iters_out, cudaStream_t stream) {
    if (!ctx) return BDG_EINVAL;
    int rc = check_grid(ctx, grid);
    if (rc) return rc;
    const int64_t N = 2LL * grid->nx * grid->ny * grid->nz;
    if (n != N) return bdg_fail(ctx, BDG_EINVAL, "bdg_refine: n=%lld but the grid gives N=%lld", (long long)n,
                                (long long)N);
    if (!U || !Delta || !w || !Z || ldz < n || max_iter < 0)
        return bdg_fail(ctx, BDG_EINVAL, "bdg_refine: bad arguments");
    cudaSetDevice(ctx->device);
    ctx->err[0] = 0;
    ws_reset(ctx);
    BDG_CUDA_TRY(ctx, cudaMemsetAsync(ctx->dflags, 0, 16 * sizeof(int), stream));
    stage_begin(ctx, stream);
    return bdg::refine_impl(ctx, grid, mu, U, Delta, n, w, Z, ldz, max_iter, tol, resid_out, orth_out, iters_out,
                            stream);
}

int bdg_densities(bdg_ctx *ctx, const bdg_grid *grid, int64_t n, const double *w, const double2 *Z, int64_t ldz,
                  double T, double Ec, double *n_out, double2 *nu_out, cudaStream_t stream) {
    if (!ctx) return BDG_EINVAL;
    int rc = check_grid(ctx, grid);
    if (rc) return rc;
    const int64_t N = 2LL * grid->nx * grid->ny * grid->nz;
    if (n != N || !w || !Z || ldz < n || !n_out || !nu_out || T < 0)
        return bdg_fail(ctx, BDG_EINVAL, "bdg_densities: bad arguments");
    cudaSetDevice(ctx->device);
    ctx->err[0] = 0;
    ws_reset(ctx);
    return bdg::densities_impl(ctx, grid, n, w, Z, ldz, T, Ec, n_out, nu_out, stream);
}

int bdg_kinetic_current_densities(bdg_ctx *ctx, const bdg_grid *grid, int64_t n, const double *w,
                                  const double2 *Z, int64_t ldz, double T, double Ec, double *tau_out,
                                  double *j_out, cudaStream_t stream) {
    if (!ctx) return BDG_EINVAL;
    int rc = check_grid(ctx, grid);
    if (rc) return rc;
    const int64_t N = 2LL * grid->nx * grid->ny * grid->nz;
    if (n != N || !w || !Z || ldz < n || !tau_out || !j_out || T < 0)
        return bdg_fail(ctx, BDG_EINVAL, "bdg_kinetic_current_densities: bad arguments");
    cudaSetDevice(ctx->device);
    ctx->err[0] = 0;
    ws_reset(ctx);
    return bdg::tau_j_impl(ctx, grid, n, w, Z, ldz, T, Ec, tau_out, j_out, stream);
}

// Contact coupling of the stated substitute functional (host arithmetic, no device): for a
// trial Hartree shift U0 the gap equation fixes g = Delta0 / nu0(U0); the Hartree condition
// phi(U0) = U0 + g n0(U0) / 2 = 0 is then solved by bisection, the bracket [-5, 0] widened
// downwards (x2, down to -5000) while phi has one sign on it (a coarse lattice in scaled units
// shifts the root down).
int bdg_gap_coupling(const bdg_grid *grid, double mu, double Delta0, double Ec, double *g_out, double *U0_out) {
    if (!grid || !g_out || !U0_out || !(Delta0 > 0) || !(Ec > 0) || grid->nx < 1 || grid->ny < 1 || grid->nz < 1 ||
        grid->dx != 1.0 || (grid->nx > 1 && (grid->nx & 1)) || (grid->ny > 1 && (grid->ny & 1)) ||
        (grid->nz > 1 && (grid->nz & 1)))
        return BDG_EINVAL;
    const int dims[3] = {grid->nx, grid->ny, grid->nz};
    std::vector<double> e1[3];
    const double pi = 3.14159265358979323846;
    for (int a = 0; a < 3; ++a) {
        const int n = dims[a];
        for (int m = -(n / 2); m < n - n / 2; ++m) {
            const double k = 2.0 * pi * m / n;
            e1[a].push_back(0.5 * k * k);
        }
    }
    const double V = (double)dims[0] * dims[1] * dims[2];
    auto sums = [&](double U0, double &n0, double &nu0) {
        double sn = 0.0, snu = 0.0;
        for (double ex : e1[0])
            for (double ey : e1[1])
                for (double ez : e1[2]) {
                    const double xi = ex + ey + ez - mu + U0;
                    const double E = std::sqrt(xi * xi + Delta0 * Delta0);
                    if (E < Ec) { sn += 1.0 - xi / E; snu += Delta0 / (2.0 * E); }
                }
        n0 = sn / V;
        nu0 = snu / V;
    };
    bool empty = false;   // no k in the window: the gap equation has no solution
    auto phi = [&](double U0) {
        double n0, nu0;
        sums(U0, n0, nu0);
        if (!(nu0 > 0)) { empty = true; return 0.0; }
        return U0 + (Delta0 / nu0) * n0 / 2.0;
    };
    double lo = -5.0, hi = 0.0, flo = phi(lo), fhi = phi(hi);
    while (flo * fhi > 0 && lo > -5e3) { lo *= 2.0; flo = phi(lo); }
    if (flo * fhi > 0) return BDG_ENOCONV;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi), fm = phi(mid);
        if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else { hi = mid; }
        if (hi - lo < 1e-15) break;
    }
    const double U0 = 0.5 * (lo + hi);
    double n0, nu0;
    sums(U0, n0, nu0);
    if (empty || !(nu0 > 0)) return BDG_ENOCONV;
    *g_out = Delta0 / nu0;
    *U0_out = U0;
    return BDG_OK;
}

int bdg_td_evolve(bdg_ctx *ctx, const bdg_grid *grid, const bdg_td_params *p, int64_t nq, const double *E0,
                  double2 *Psi, int64_t ldpsi, int nsteps, double *n_out, double2 *nu_out, cudaStream_t stream) {
    if (!ctx) return BDG_EINVAL;
    int rc = check_grid(ctx, grid);
    if (rc) return rc;
    const int64_t N = 2LL * grid->nx * grid->ny * grid->nz;
    if (!p || !E0 || !Psi || nq < 1 || ldpsi < N || !(p->dt > 0) || nsteps < 0 || p->T < 0)
        return bdg_fail(ctx, BDG_EINVAL, "bdg_td_evolve: bad arguments");
    cudaSetDevice(ctx->device);
    ctx->err[0] = 0;
    return bdg::td_evolve_impl(ctx, grid, p, nq, E0, Psi, ldpsi, nsteps, n_out, nu_out, stream);
}

int bdg_scf_step(bdg_ctx *ctx, const bdg_grid *grid, const bdg_scf_params *p, double *U, double2 *Delta,
                 double *dn_max_out, cudaStream_t stream) {
    if (!ctx) return BDG_EINVAL;
    int rc = check_grid(ctx, grid);
    if (rc) return rc;
    if (!p || !U || !Delta || !p->n_prev || p->alpha <= 0 || p->alpha > 1 || p->g <= 0)
        return bdg_fail(ctx, BDG_EINVAL, "bdg_scf_step: bad arguments");
    cudaSetDevice(ctx->device);
    ctx->err[0] = 0;
    const int64_t V = (int64_t)grid->nx * grid->ny * grid->nz, N = 2 * V;
    // persistent buffers for this step: H, Z (complex128), w, n, nu, dn
    size_t bytes_heev = 0;
    bdg_heev_workspace(ctx, N, p->prec, &bytes_heev);
    size_t own = 2 * align_up((size_t)N * N * 16) + align_up((size_t)N * 8) + align_up((size_t)V * 8) +
                 align_up((size_t)V * 16) + align_up(64) + align_up(4096);
    // refine needs its own workspace after heev; take the max of the two
    size_t bytes_ref = bdg::refine_workspace_bytes(N);
    rc = ws_reserve(ctx, own + std::max(bytes_heev, bytes_ref));
    if (rc) return rc;
    double2 *H = (double2 *)ws_take(ctx, (size_t)N * N * 16);
    double2 *Zb = (double2 *)ws_take(ctx, (size_t)N * N * 16);
    double *wv = (double *)ws_take(ctx, (size_t)N * 8);
    double *nv = (double *)ws_take(ctx, (size_t)V * 8);
    double2 *nuv = (double2 *)ws_take(ctx, (size_t)V * 16);
    double *dn = (double *)ws_take(ctx, 64);
    double *ktab = (double *)ws_take(ctx, 4096);
    const size_t mark = ctx->ws_top;
    BDG_CUDA_TRY(ctx, cudaMemsetAsync(ctx->dflags, 0, 16 * sizeof(int), stream));
    rc = bdg::launch_build(ctx, grid->nx, grid->ny, grid->nz, p->mu, U, Delta, H, N, ktab, stream);
    if (rc) return rc;
    const int b = band_for(ctx, p->prec, N);
    ctx->last_heev_prec = p->prec;
    if (p->prec == BDG_PREC_FP64) {
        rc = bdg::heev_impl<double>(ctx, N, H, N, wv, Zb, N, b, 0, stream, true);
    } else {
        float2 *A32 = (float2 *)ws_take(ctx, (size_t)N * N * 8);
        float2 *E32 = (float2 *)ws_take(ctx, (size_t)N * N * 8);
        if (!A32 || !E32) return bdg_fail(ctx, BDG_ENOMEM, "scf_step: workspace");
        rc = bdg::launch_convert_z64_to_z32(ctx, N, N, H, N, A32, N, stream);
        if (!rc) rc = bdg::heev_impl<float>(ctx, N, A32, N, wv, E32, N, b, tc_slices(ctx, p->prec), stream, true);
        if (!rc) rc = bdg::launch_convert_z32_to_z64(ctx, N, N, E32, N, Zb, N, stream);
    }
    if (rc) return rc;
    ctx->ws_top = mark;
    if (p->prec != BDG_PREC_FP64 && p->refine_iters > 0) {
        double res = 0;
        int its = 0;
        rc = bdg::refine_impl(ctx, grid, p->mu, U, Delta, N, wv, Zb, N, p->refine_iters,
                              p->refine_tol > 0 ? p->refine_tol : 1e-11, &res, nullptr, &its, stream);
        if (rc && rc != BDG_ENOCONV) return rc;
        ctx->ws_top = mark;
    }
    rc = bdg::densities_impl(ctx, grid, N, wv, Zb, N, p->T, p->Ec, nv, nuv, stream);
    if (rc) return rc;
    rc = bdg::scf_update_impl(ctx, V, p, nv, nuv, U, Delta, dn, stream);
    if (rc) return rc;
    if (dn_max_out) {
        BDG_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->hscal, dn, sizeof(double), cudaMemcpyDeviceToHost, stream));
        BDG_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
        *dn_max_out = ctx->hscal[0];
    }
    return BDG_OK;
}

}  // extern "C"
