// bdg_build: fill the dense BdG matrix of Eq. (stHpsi).
//
// h = T + diag(U) - mu with T the spectral kinetic operator F^-1 (k^2/2) F on
// the periodic grid (paper, "Numerical setup and implementation").  On a
// periodic 1-D grid of n points that operator is the real symmetric
// circulant with first column
//     t(0) = pi^2 (n^2 + 2) / (6 n^2),
//     t(d) = (-1)^d pi^2 / (n^2 sin^2(pi d / n)),   d = 1 .. n-1,
// (the closed-form sum of (1/n) sum_m (k_m^2/2) cos(k_m d) over
// k_m = 2 pi m / n, m = -n/2 .. n/2-1), and in 3-D it is the Kronecker sum
// T = T_x (x) I (x) I + I (x) T_y (x) I + I (x) I (x) T_z.  Each row of h
// therefore has nx + ny + nz - 2 nonzeros and h is real, so the lower-right
// block -h^* equals -h.
//
// The fill is one pass writing N^2 complex128 values: HBM-write bound.
#include "internal.h"

namespace bdg {

__global__ void kinetic_tables_kernel(int nx, int ny, int nz, double *ktab) {
    // ktab = [t_x(0..nx-1), t_y(0..ny-1), t_z(0..nz-1)]
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int total = nx + ny + nz;
    if (i >= total) return;
    int n, d;
    if (i < nx) { n = nx; d = i; }
    else if (i < nx + ny) { n = ny; d = i - nx; }
    else { n = nz; d = i - nx - ny; }
    const double pi2 = 9.869604401089358;  // pi^2
    double nn = (double)n * (double)n;
    double t;
    if (n == 1) {
        t = 0.0;   // a single point carries only the k = 0 mode
    } else if (d == 0) {
        t = pi2 * (nn + 2.0) / (6.0 * nn);
    } else {
        double s = sinpi((double)d / (double)n);
        t = ((d & 1) ? -1.0 : 1.0) * pi2 / (nn * s * s);
    }
    ktab[i] = t;
}

// One thread writes one complex entry; blockIdx.y (and z) index the column.
__global__ void build_kernel(int nx, int ny, int nz, double mu, const double *__restrict__ U,
                             const double2 *__restrict__ Delta, double2 *__restrict__ H,
                             int64_t ldh, const double *__restrict__ ktab) {
    const int64_t V = (int64_t)nx * ny * nz;
    const int64_t N = 2 * V;
    const int64_t j = (int64_t)blockIdx.y + (int64_t)blockIdx.z * gridDim.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N || j >= N) return;
    const double *tx = ktab, *ty = ktab + nx, *tz = ktab + nx + ny;
    const bool iu = i < V, ju = j < V;
    const int64_t s = iu ? i : i - V;
    const int64_t t = ju ? j : j - V;
    double2 out = make_double2(0.0, 0.0);
    if (iu == ju) {
        const int64_t nyz = (int64_t)ny * nz;
        int ix = (int)(s / nyz), iy = (int)((s / nz) % ny), iz = (int)(s % nz);
        int jx = (int)(t / nyz), jy = (int)((t / nz) % ny), jz = (int)(t % nz);
        double h = 0.0;
        if (iy == jy && iz == jz) h += tx[(ix - jx + nx) % nx];
        if (ix == jx && iz == jz) h += ty[(iy - jy + ny) % ny];
        if (ix == jx && iy == jy) h += tz[(iz - jz + nz) % nz];
        if (s == t) h += U[s] - mu;
        out.x = iu ? h : -h;   // lower-right block: -conj(h) = -h (h real)
    } else if (s == t) {
        double2 d = Delta[s];
        out = iu ? d : make_double2(d.x, -d.y);  // upper-right Delta, lower-left Delta^*
    }
    H[i + j * ldh] = out;
}

int launch_kinetic_tables(bdg_ctx *ctx, int nx, int ny, int nz, double *ktab, cudaStream_t st) {
    int total = nx + ny + nz;
    kinetic_tables_kernel<<<(total + 127) / 128, 128, 0, st>>>(nx, ny, nz, ktab);
    BDG_LAUNCH_CHECK(ctx);
    return BDG_OK;
}

int launch_build(bdg_ctx *ctx, int nx, int ny, int nz, double mu, const double *U,
                 const double2 *Delta, double2 *H, int64_t ldh, double *ktab, cudaStream_t st) {
    int rc = launch_kinetic_tables(ctx, nx, ny, nz, ktab, st);
    if (rc) return rc;
    const int64_t N = 2LL * nx * ny * nz;
    dim3 block(256);
    int64_t gy = N, gz = 1;
    while (gy > 65535) { gz *= 2; gy = (N + gz - 1) / gz; }
    dim3 grid((unsigned)((N + 255) / 256), (unsigned)gy, (unsigned)gz);
    build_kernel<<<grid, block, 0, st>>>(nx, ny, nz, mu, U, Delta, H, ldh, ktab);
    BDG_LAUNCH_CHECK(ctx);
    return BDG_OK;
}

}  // namespace bdg
