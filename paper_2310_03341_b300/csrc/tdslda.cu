// Time evolution of the quasiparticle wavefunctions (paper, Eq. (TDSLDA) and
// "Performance of the Time Evolution Algorithm"):
//
//   i d phi_n / dt = H(t) phi_n,   H = [[h, Delta], [Delta^*, -h^*]],  h = T + U - mu,
//
// for all evolved states at once; H is the same for every state and depends
// on the states only through the local densities n and nu (Eq. (densities2),
// occupation weights f_T(+-E_n) fixed at their initial values), through the
// stated contact functional U = U_ext - g n / 2, Delta = g nu.
//
// Time stepping: fifth-order Adams-Bashforth-Moulton, predict - evaluate -
// correct - evaluate, so H (densities, U, Delta and H Psi) is evaluated twice
// per step as in the paper.  With K = H Psi (so F = -i K):
//   P        = Psi - i dt sum_k b_k K_{n-k},    b = (1901, -2774, 2616, -1274, 251) / 720,
//   Psi_n+1  = Psi - i dt (a_0 K(P) + sum_{k>=1} a_k K_{n+1-k}),
//                                                a = (251, 646, -264, 106, -19) / 720.
// The first four steps are classical RK4 steps, which build the history.
//
// On the GPU one evaluation is: the densities of all states (FP64 partial
// sums per column chunk, reduced deterministically), the functional update,
// and H applied to every state through the Kronecker-sum structure of the
// kinetic operator (the circulant 1-D tables t(d), i.e. the spectral k^2/2
// applied as exact line convolutions, no FFT library).  The step
// combinations are one fused kernel over the state arrays.
#include <algorithm>
#include <initializer_list>
#include <utility>

#include "internal.h"

namespace bdg {

int launch_apply_h(bdg_ctx *ctx, int nx, int ny, int nz, double mu, const double *U, const double2 *Delta,
                   const double *ktab, int64_t ncols, const double2 *X, int64_t ldx, double2 *Y, int64_t ldy,
                   cudaStream_t st);
int launch_column_densities(bdg_ctx *ctx, int64_t V, const double *w, const double2 *Z, int64_t ldz,
                            const int64_t *lohi, double T, int nchunks, double *pn, double2 *pnu, double *n_out,
                            double2 *nu_out, cudaStream_t st);

namespace td {

constexpr double kAB5[5] = {1901.0 / 720.0, -2774.0 / 720.0, 2616.0 / 720.0, -1274.0 / 720.0, 251.0 / 720.0};
constexpr double kAM5[5] = {251.0 / 720.0, 646.0 / 720.0, -264.0 / 720.0, 106.0 / 720.0, -19.0 / 720.0};

struct Combo {
    const double2 *K[5];
    double c[5];
    int m;
    int minus_i;   // 1: out = base - i sum c_j K_j;  0: out = base + sum c_j K_j
};

__global__ void combo_kernel(int64_t count, const double2 *__restrict__ base, double2 *__restrict__ out, Combo cb) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    double sr = 0.0, si = 0.0;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        if (j < cb.m) {
            const double2 k = cb.K[j][i];
            sr = fma(cb.c[j], k.x, sr);
            si = fma(cb.c[j], k.y, si);
        }
    }
    const double2 b = base[i];
    out[i] = cb.minus_i ? make_double2(b.x + si, b.y - sr)    // -i (sr + i si) = si - i sr
                        : make_double2(b.x + sr, b.y + si);
}

// U = U_ext - g n / 2,  Delta = g nu
__global__ void fields_kernel(int64_t V, const double *__restrict__ n, const double2 *__restrict__ nu,
                              const double *__restrict__ U_ext, double g, double *__restrict__ U,
                              double2 *__restrict__ D) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    U[s] = (U_ext ? U_ext[s] : 0.0) - 0.5 * g * n[s];
    const double2 v = nu[s];
    D[s] = make_double2(g * v.x, g * v.y);
}

__global__ void set_range_kernel(int64_t *lohi, int64_t hi) {
    lohi[0] = 0;
    lohi[1] = hi;
}

__global__ void copy_cols_kernel(int64_t rows, int64_t cols, const double2 *__restrict__ src, int64_t lds,
                                 double2 *__restrict__ dst, int64_t ldd) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    const int64_t r = idx % rows, c = idx / rows;
    dst[r + c * ldd] = src[r + c * lds];
}

}  // namespace td

int td_evolve_impl(bdg_ctx *ctx, const bdg_grid *g, const bdg_td_params *p, int64_t nq, const double *E0,
                   double2 *Psi, int64_t ldpsi, int nsteps, double *n_out, double2 *nu_out, cudaStream_t st) {
    const int64_t V = (int64_t)g->nx * g->ny * g->nz, N = 2 * V;
    const int64_t cnt = N * nq;                 // entries of one state array
    const size_t sbytes = (size_t)cnt * 16;
    const int nchunks = (int)std::max<int64_t>(1, std::min<int64_t>(64, (ctx->num_sms * 8 * 256) / V));
    const size_t need = 9 * align_up(sbytes) + 2 * align_up((size_t)V * 8) + 2 * align_up((size_t)V * 16) +
                        align_up((size_t)nchunks * V * 8) + align_up((size_t)nchunks * V * 16) + 2 * align_up(4096);
    int rc = ws_reserve(ctx, need);
    if (rc) return rc;
    double2 *Ps = (double2 *)ws_take(ctx, sbytes);     // the state, contiguous (ld N)
    double2 *X = (double2 *)ws_take(ctx, sbytes);      // stage / predictor input
    double2 *KP = (double2 *)ws_take(ctx, sbytes);     // H at the stage or predicted state
    double2 *Ks = (double2 *)ws_take(ctx, sbytes);     // RK4: k1 + 2 k2 + 2 k3
    double2 *ring[5];
    for (int i = 0; i < 5; ++i) ring[i] = (double2 *)ws_take(ctx, sbytes);   // H Psi_n, H Psi_n-1, ...
    double *nv = (double *)ws_take(ctx, (size_t)V * 8);
    double2 *nuv = (double2 *)ws_take(ctx, (size_t)V * 16);
    double *U = (double *)ws_take(ctx, (size_t)V * 8);
    double2 *D = (double2 *)ws_take(ctx, (size_t)V * 16);
    double *pn = (double *)ws_take(ctx, (size_t)nchunks * V * 8);
    double2 *pnu = (double2 *)ws_take(ctx, (size_t)nchunks * V * 16);
    double *ktab = (double *)ws_take(ctx, 4096);
    int64_t *lohi = (int64_t *)ws_take(ctx, 4096);
    if (!lohi) return bdg_fail(ctx, BDG_ENOMEM, "td_evolve: workspace");
    rc = launch_kinetic_tables(ctx, g->nx, g->ny, g->nz, ktab, st);
    if (rc) return rc;
    td::set_range_kernel<<<1, 1, 0, st>>>(lohi, nq);
    BDG_LAUNCH_CHECK(ctx);
    const unsigned sgrid = (unsigned)((cnt + 255) / 256);
    td::copy_cols_kernel<<<sgrid, 256, 0, st>>>(N, nq, Psi, ldpsi, Ps, N);
    BDG_LAUNCH_CHECK(ctx);

    // K = H[X] X: densities of X, the functional, then H applied to every column
    auto evaluate = [&](const double2 *Xs, double2 *K) -> int {
        int r = launch_column_densities(ctx, V, E0, Xs, N, lohi, p->T, nchunks, pn, pnu, nv, nuv, st);
        if (r) return r;
        td::fields_kernel<<<(unsigned)((V + 255) / 256), 256, 0, st>>>(V, nv, nuv, p->U_ext, p->g, U, D);
        BDG_LAUNCH_CHECK(ctx);
        return launch_apply_h(ctx, g->nx, g->ny, g->nz, p->mu, U, D, ktab, nq, Xs, N, K, N, st);
    };
    auto combo = [&](const double2 *base, double2 *out, bool minus_i,
                     std::initializer_list<std::pair<const double2 *, double>> terms) -> int {
        td::Combo cb;
        cb.m = 0;
        cb.minus_i = minus_i ? 1 : 0;
        for (auto &t : terms) { cb.K[cb.m] = t.first; cb.c[cb.m] = t.second; ++cb.m; }
        for (int j = cb.m; j < 5; ++j) { cb.K[j] = nullptr; cb.c[j] = 0.0; }
        td::combo_kernel<<<sgrid, 256, 0, st>>>(cnt, base, out, cb);
        BDG_LAUNCH_CHECK(ctx);
        return BDG_OK;
    };
    const double dt = p->dt;
    // history: ring[(head - j) mod 5] = H Psi_{n-j} for j < have
    int have = 0, head = 0;
    auto hist = [&](int j) { return ring[((head - j) % 5 + 5) % 5]; };
    rc = evaluate(Ps, ring[0]);
    if (rc) return rc;
    have = 1;
    for (int step = 0; step < nsteps; ++step) {
        if (have < 5) {
            // classical RK4 with k1 = H Psi_n: k2 = H(Psi - i dt/2 k1), k3 = H(Psi - i dt/2 k2),
            // k4 = H(Psi - i dt k3), Psi += -i dt/6 (k1 + 2 k2 + 2 k3 + k4)
            const double2 *k1 = hist(0);
            if ((rc = combo(Ps, X, true, {{k1, 0.5 * dt}}))) return rc;
            if ((rc = evaluate(X, KP))) return rc;
            if ((rc = combo(k1, Ks, false, {{KP, 2.0}}))) return rc;
            if ((rc = combo(Ps, X, true, {{KP, 0.5 * dt}}))) return rc;
            if ((rc = evaluate(X, KP))) return rc;
            if ((rc = combo(Ks, Ks, false, {{KP, 2.0}}))) return rc;
            if ((rc = combo(Ps, X, true, {{KP, dt}}))) return rc;
            if ((rc = evaluate(X, KP))) return rc;
            if ((rc = combo(Ps, Ps, true, {{Ks, dt / 6.0}, {KP, dt / 6.0}}))) return rc;
        } else {
            // predict, evaluate, correct
            if ((rc = combo(Ps, X, true, {{hist(0), dt * td::kAB5[0]}, {hist(1), dt * td::kAB5[1]},
                                          {hist(2), dt * td::kAB5[2]}, {hist(3), dt * td::kAB5[3]},
                                          {hist(4), dt * td::kAB5[4]}})))
                return rc;
            if ((rc = evaluate(X, KP))) return rc;
            if ((rc = combo(Ps, Ps, true, {{KP, dt * td::kAM5[0]}, {hist(0), dt * td::kAM5[1]},
                                           {hist(1), dt * td::kAM5[2]}, {hist(2), dt * td::kAM5[3]},
                                           {hist(3), dt * td::kAM5[4]}})))
                return rc;
        }
        // evaluate at the new state: the newest history entry
        head = (head + 1) % 5;
        if ((rc = evaluate(Ps, ring[head]))) return rc;
        have = std::min(have + 1, 5);
    }
    // results: the state back to the caller's layout, the densities at the final time
    td::copy_cols_kernel<<<sgrid, 256, 0, st>>>(N, nq, Ps, N, Psi, ldpsi);
    BDG_LAUNCH_CHECK(ctx);
    if (n_out || nu_out) {
        rc = launch_column_densities(ctx, V, E0, Ps, N, lohi, p->T, nchunks, pn, pnu, n_out ? n_out : nv,
                                     nu_out ? nu_out : nuv, st);
        if (rc) return rc;
    }
    return BDG_OK;
}

}  // namespace bdg
