// Local densities of Eq. (densities2) and the self-consistent update.
//
//   n(r)  = 2 sum_{0<E_n<Ec} ( |v_n(r)|^2 f_T(-E_n) + |u_n(r)|^2 f_T(E_n) ),
//   nu(r) =   sum_{0<E_n<Ec} u_n(r) v_n(r)^* ( f_T(-E_n) - f_T(E_n) ),
//   f_T(E) = 1 / (1 + exp(E/T))   (T = 0: step function, f(0) = 1/2).
// The eigenvalues are sorted, so the window is a contiguous column range; the
// kernel reads only those columns of Z (HBM-bound: 16 B per element of the
// window), accumulating in FP64 per (site, column chunk) and reducing the
// chunks deterministically.
#include <stdarg.h>
#include <stdio.h>

#include <mutex>

#include "internal.h"

namespace bdg {

__device__ __forceinline__ double fermi(double E, double T) {
    if (T == 0.0) return E < 0.0 ? 1.0 : (E > 0.0 ? 0.0 : 0.5);
    return 1.0 / (1.0 + exp(E / T));
}

// window [lo, hi) of sorted w with 0 < w < Ec
__global__ void window_kernel(int64_t n, const double *__restrict__ w, double Ec, int64_t *__restrict__ lohi) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t a = 0, b = n;
    while (a < b) { int64_t m = (a + b) / 2; if (w[m] > 0.0) b = m; else a = m + 1; }
    int64_t lo = a;
    a = lo; b = n;
    while (a < b) { int64_t m = (a + b) / 2; if (w[m] >= Ec) b = m; else a = m + 1; }
    lohi[0] = lo;
    lohi[1] = a;
}

__global__ void __launch_bounds__(256) density_partial_kernel(int64_t V, const double *__restrict__ w,
                                                              const double2 *__restrict__ Z, int64_t ldz,
                                                              const int64_t *__restrict__ lohi, double T,
                                                              int nchunks, double *__restrict__ pn,
                                                              double2 *__restrict__ pnu) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int chunk = blockIdx.y;
    const int64_t lo = lohi[0], hi = lohi[1];
    const int64_t cnt = hi - lo;
    const int64_t cs = (cnt + nchunks - 1) / nchunks;
    const int64_t j0 = lo + chunk * cs, j1 = min(hi, j0 + cs);
    if (s >= V) return;
    double an = 0.0, ax = 0.0, ay = 0.0;
    for (int64_t j = j0; j < j1; ++j) {
        const double E = w[j];
        const double fp = fermi(E, T), fm = fermi(-E, T);
        const double2 u = Z[s + j * ldz], v = Z[V + s + j * ldz];
        an += 2.0 * ((v.x * v.x + v.y * v.y) * fm + (u.x * u.x + u.y * u.y) * fp);
        const double c = fm - fp;
        // u * conj(v)
        ax += c * (u.x * v.x + u.y * v.y);
        ay += c * (u.y * v.x - u.x * v.y);
    }
    pn[(int64_t)chunk * V + s] = an;
    pnu[(int64_t)chunk * V + s] = make_double2(ax, ay);
}

__global__ void density_reduce_kernel(int64_t V, int nchunks, const double *__restrict__ pn,
                                      const double2 *__restrict__ pnu, double *__restrict__ n_out,
                                      double2 *__restrict__ nu_out) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    double a = 0.0;
    double2 b = make_double2(0.0, 0.0);
    for (int c = 0; c < nchunks; ++c) {
        a += pn[(int64_t)c * V + s];
        double2 t = pnu[(int64_t)c * V + s];
        b.x += t.x; b.y += t.y;
    }
    n_out[s] = a;
    nu_out[s] = b;
}

// Densities of the columns [lohi[0], lohi[1]) of Z (device bounds) with the Fermi
// weights of w over those columns; partial sums in pn / pnu (nchunks * V each).
int launch_column_densities(bdg_ctx *ctx, int64_t V, const double *w, const double2 *Z, int64_t ldz,
                            const int64_t *lohi, double T, int nchunks, double *pn, double2 *pnu, double *n_out,
                            double2 *nu_out, cudaStream_t st) {
    dim3 grid((unsigned)((V + 255) / 256), (unsigned)nchunks);
    density_partial_kernel<<<grid, 256, 0, st>>>(V, w, Z, ldz, lohi, T, nchunks, pn, pnu);
    BDG_LAUNCH_CHECK(ctx);
    density_reduce_kernel<<<(unsigned)((V + 255) / 256), 256, 0, st>>>(V, nchunks, pn, pnu, n_out, nu_out);
    BDG_LAUNCH_CHECK(ctx);
    return BDG_OK;
}

int densities_impl(bdg_ctx *ctx, const bdg_grid *g, int64_t n, const double *w, const double2 *Z, int64_t ldz,
                   double T, double Ec, double *n_out, double2 *nu_out, cudaStream_t st) {
    const int64_t V = n / 2;
    const int nchunks = (int)std::max<int64_t>(1, std::min<int64_t>(64, (ctx->num_sms * 8 * 256) / std::max<int64_t>(V, 1)));
    size_t need = align_up(16) + align_up((size_t)nchunks * V * 8) + align_up((size_t)nchunks * V * 16);
    if (ctx->ws_top + need > ctx->ws_bytes) {
        if (ctx->ws_top != 0) return bdg_fail(ctx, BDG_ENOMEM, "densities: workspace arena too small");
        int rc = ws_reserve(ctx, need + 4096);
        if (rc) return rc;
    }
    int64_t *lohi = (int64_t *)ws_take(ctx, 16);
    double *pn = (double *)ws_take(ctx, (size_t)nchunks * V * 8);
    double2 *pnu = (double2 *)ws_take(ctx, (size_t)nchunks * V * 16);
    window_kernel<<<1, 32, 0, st>>>(n, w, Ec, lohi);
    BDG_LAUNCH_CHECK(ctx);
    dim3 grid((unsigned)((V + 255) / 256), (unsigned)nchunks);
    density_partial_kernel<<<grid, 256, 0, st>>>(V, w, Z, ldz, lohi, T, nchunks, pn, pnu);
    BDG_LAUNCH_CHECK(ctx);
    density_reduce_kernel<<<(unsigned)((V + 255) / 256), 256, 0, st>>>(V, nchunks, pn, pnu, n_out, nu_out);
    BDG_LAUNCH_CHECK(ctx);
    (void)g;
    return BDG_OK;
}

// ---- kinetic density tau(r) and current j(r) of Eq. (densities2) ----------------
//   tau = 2 sum_{0<E<Ec} ( |grad v|^2 f_T(-E) + |grad u|^2 f_T(E) ),
//   j   = 2 sum_{0<E<Ec} Im( v grad v^* f_T(-E) - u grad u^* f_T(E) ),
// with the spectral gradient (d_a f)(x) = sum_x' D(x - x') f(x') along each axis,
// D(d) = (1/n) sum_m i k_m e^{i k_m d}, k_m = 2 pi m / n, m = -n/2 .. n/2-1:
//   Dj(d) = -(2/n) sum_{m=1}^{n/2-1} k_m sin(k_m d)   (the Nyquist mode gets derivative 0,
//            so a real state carries no current),
//   Dt(d) = Dj(d) - i pi (-1)^d / n                    (k = -pi kept, so sum_r tau is twice
//            the kinetic energy of the build's kinetic operator).
// A dimension of one point has D = 0.  Tables for x, y, z at offsets 0, nx, nx + ny.
__global__ void deriv_tables_kernel(int nx, int ny, int nz, double *__restrict__ Dj, double2 *__restrict__ Dt) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nx + ny + nz) return;
    const int n = t < nx ? nx : (t < nx + ny ? ny : nz);
    const int d = t < nx ? t : (t < nx + ny ? t - nx : t - nx - ny);
    const double pi = 3.14159265358979323846;
    double sj = 0.0;
    for (int m = 1; m < n / 2; ++m) {
        const int r = (int)(((long long)m * d) % n);       // sin(k_m d) = sin(2 pi r / n), exact argument
        sj += (2.0 * pi * m / n) * sinpi(2.0 * r / n);
    }
    const double dj = n > 1 ? -2.0 * sj / n : 0.0;
    const double ny_im = n > 1 ? -pi * ((d & 1) ? -1.0 : 1.0) / n : 0.0;
    Dj[t] = dj;
    Dt[t] = make_double2(dj, ny_im);
}

// One thread per site over one chunk of the window's columns; partial sums per chunk
// (reduced deterministically by tau_j_reduce_kernel).  The line of each axis through the
// site is read from Z (L1/L2 resident: neighbouring threads read the same lines).
__global__ void __launch_bounds__(128) tau_j_partial_kernel(int nx, int ny, int nz, const double *__restrict__ w,
                                                            const double2 *__restrict__ Z, int64_t ldz,
                                                            const int64_t *__restrict__ lohi, double T, int nchunks,
                                                            const double *__restrict__ Dj,
                                                            const double2 *__restrict__ Dt,
                                                            double *__restrict__ ptau, double *__restrict__ pj) {
    const int64_t V = (int64_t)nx * ny * nz;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int chunk = blockIdx.y;
    const int64_t lo = lohi[0], hi = lohi[1];
    const int64_t cs = (hi - lo + nchunks - 1) / nchunks;
    const int64_t j0 = lo + chunk * cs, j1 = min(hi, j0 + cs);
    if (s >= V) return;
    const int64_t sx = (int64_t)ny * nz, sy = nz;
    const int ix = (int)(s / sx), iy = (int)((s / sy) % ny), iz = (int)(s % nz);
    const int64_t base[3] = {s - ix * sx, s - iy * sy, s - iz};
    const int64_t stride[3] = {sx, sy, 1};
    const int len[3] = {nx, ny, nz}, pos[3] = {ix, iy, iz}, off[3] = {0, nx, nx + ny};
    double at = 0.0, aj[3] = {0.0, 0.0, 0.0};
    for (int64_t j = j0; j < j1; ++j) {
        const double E = w[j];
        const double fp = fermi(E, T), fm = fermi(-E, T);
        const double2 *zu = Z + j * ldz, *zv = zu + V;
        const double2 u = zu[s], v = zv[s];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double2 tu = make_double2(0, 0), tv = make_double2(0, 0), gu = make_double2(0, 0),
                    gv = make_double2(0, 0);
            for (int q = 0; q < len[a]; ++q) {
                int d = pos[a] - q;
                if (d < 0) d += len[a];
                const double dj = Dj[off[a] + d];
                const double2 dt = Dt[off[a] + d];
                const int64_t sq = base[a] + q * stride[a];
                const double2 fu = zu[sq], fv = zv[sq];
                gu.x += dj * fu.x; gu.y += dj * fu.y;
                gv.x += dj * fv.x; gv.y += dj * fv.y;
                tu.x += dt.x * fu.x - dt.y * fu.y; tu.y += dt.x * fu.y + dt.y * fu.x;
                tv.x += dt.x * fv.x - dt.y * fv.y; tv.y += dt.x * fv.y + dt.y * fv.x;
            }
            at += 2.0 * (fm * (tv.x * tv.x + tv.y * tv.y) + fp * (tu.x * tu.x + tu.y * tu.y));
            // Im(f conj(g)) = f.y g.x - f.x g.y
            aj[a] += 2.0 * (fm * (v.y * gv.x - v.x * gv.y) - fp * (u.y * gu.x - u.x * gu.y));
        }
    }
    ptau[(int64_t)chunk * V + s] = at;
    for (int a = 0; a < 3; ++a) pj[((int64_t)chunk * 3 + a) * V + s] = aj[a];
}

__global__ void tau_j_reduce_kernel(int64_t V, int nchunks, const double *__restrict__ ptau,
                                    const double *__restrict__ pj, double *__restrict__ tau_out,
                                    double *__restrict__ j_out) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    double t = 0.0, x = 0.0, y = 0.0, z = 0.0;
    for (int c = 0; c < nchunks; ++c) {
        t += ptau[(int64_t)c * V + s];
        x += pj[((int64_t)c * 3 + 0) * V + s];
        y += pj[((int64_t)c * 3 + 1) * V + s];
        z += pj[((int64_t)c * 3 + 2) * V + s];
    }
    tau_out[s] = t;
    j_out[s] = x;
    j_out[V + s] = y;
    j_out[2 * V + s] = z;
}

int tau_j_impl(bdg_ctx *ctx, const bdg_grid *g, int64_t n, const double *w, const double2 *Z, int64_t ldz,
               double T, double Ec, double *tau_out, double *j_out, cudaStream_t st) {
    const int64_t V = n / 2;
    const int nt = g->nx + g->ny + g->nz;
    const int nchunks = (int)std::max<int64_t>(1, std::min<int64_t>(64, (ctx->num_sms * 8 * 128) / std::max<int64_t>(V, 1)));
    size_t need = align_up(16) + align_up((size_t)nt * 8) + align_up((size_t)nt * 16) +
                  align_up((size_t)nchunks * V * 8) + align_up((size_t)nchunks * V * 24);
    if (ctx->ws_top + need > ctx->ws_bytes) {
        if (ctx->ws_top != 0) return bdg_fail(ctx, BDG_ENOMEM, "tau/j densities: workspace arena too small");
        int rc = ws_reserve(ctx, need + 4096);
        if (rc) return rc;
    }
    int64_t *lohi = (int64_t *)ws_take(ctx, 16);
    double *Dj = (double *)ws_take(ctx, (size_t)nt * 8);
    double2 *Dt = (double2 *)ws_take(ctx, (size_t)nt * 16);
    double *ptau = (double *)ws_take(ctx, (size_t)nchunks * V * 8);
    double *pj = (double *)ws_take(ctx, (size_t)nchunks * V * 24);
    window_kernel<<<1, 32, 0, st>>>(n, w, Ec, lohi);
    BDG_LAUNCH_CHECK(ctx);
    deriv_tables_kernel<<<(unsigned)((nt + 127) / 128), 128, 0, st>>>(g->nx, g->ny, g->nz, Dj, Dt);
    BDG_LAUNCH_CHECK(ctx);
    dim3 grid((unsigned)((V + 127) / 128), (unsigned)nchunks);
    tau_j_partial_kernel<<<grid, 128, 0, st>>>(g->nx, g->ny, g->nz, w, Z, ldz, lohi, T, nchunks, Dj, Dt, ptau, pj);
    BDG_LAUNCH_CHECK(ctx);
    tau_j_reduce_kernel<<<(unsigned)((V + 255) / 256), 256, 0, st>>>(V, nchunks, ptau, pj, tau_out, j_out);
    BDG_LAUNCH_CHECK(ctx);
    return BDG_OK;
}

// U <- (1-a) U + a (-g n/2);  Delta <- (1-a) Delta + a g nu (or its projection on
// the fixed phase);  dn = max |n - n_prev|;  n_prev <- n.   One CTA of 256 threads.
__global__ void __launch_bounds__(256) scf_update_kernel(int64_t V, double g, double alpha,
                                                          const double2 *__restrict__ phase,
                                                          const double *__restrict__ n,
                                                          const double2 *__restrict__ nu, double *__restrict__ U,
                                                          double2 *__restrict__ Delta, double *__restrict__ n_prev,
                                                          double *__restrict__ dn_out) {
    __shared__ double s[256];
    double m = 0.0;
    for (int64_t i = threadIdx.x; i < V; i += blockDim.x) {
        const double ni = n[i];
        m = fmax(m, fabs(ni - n_prev[i]));
        n_prev[i] = ni;
        U[i] = (1.0 - alpha) * U[i] + alpha * (-0.5 * g * ni);
        double2 d = nu[i];
        double2 target;
        if (phase) {
            double2 p = phase[i];
            double proj = d.x * p.x + d.y * p.y;  // Re(nu conj(p))
            target = make_double2(g * proj * p.x, g * proj * p.y);
        } else {
            target = make_double2(g * d.x, g * d.y);
        }
        double2 o = Delta[i];
        Delta[i] = make_double2((1.0 - alpha) * o.x + alpha * target.x, (1.0 - alpha) * o.y + alpha * target.y);
    }
    s[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] = fmax(s[threadIdx.x], s[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *dn_out = s[0];
}

int scf_update_impl(bdg_ctx *ctx, int64_t V, const bdg_scf_params *p, const double *n, const double2 *nu, double *U,
                    double2 *Delta, double *dn_max_dev, cudaStream_t st) {
    scf_update_kernel<<<1, 256, 0, st>>>(V, p->g, p->alpha, p->phase, n, nu, U, Delta, p->n_prev, dn_max_dev);
    BDG_LAUNCH_CHECK(ctx);
    return BDG_OK;
}

}  // namespace bdg

// ---------------------------------------------------------------------------
// Allocation-free densities (bdg_densities_noalloc; no counterpart in the
// paper).  For callers that must not allocate device memory during the SCF
// loop: a host whose own allocator already holds the device memory it may
// use (a cudaMalloc there would fail or break its accounting), and a loop
// that must not take the implicit device-wide synchronisation of cudaFree.
// The per-chunk partial sums and the window bounds live in one file-scope
// device array of fixed size instead of the context workspace; there is no
// context, no cudaMalloc/cudaFree and no allocating library routine.
//
// Scratch layout (bytes): [0, 256) window bounds lo, hi (int64);
// then nchunks*V doubles of n partials, then nchunks*V double2 of nu
// partials, each 256-byte aligned.  Every scratch word this call reads is
// written earlier by the same call (window_kernel writes lo/hi; every
// (chunk, site) slot is written by density_partial_kernel, also for empty
// chunks), so nothing needs to start at zero and nothing is cleared.
// One copy per device: calls that overlap on one device (two streams, or two
// host threads) share it and race.
namespace bdg {
namespace noalloc {
constexpr size_t kScratchBytes = 4u << 20;   // 4 MiB per device
constexpr int64_t kMaxSites = 174720;        // V bound: 768 + 24 V <= kScratchBytes at one chunk
constexpr int kMaxDevices = 64;
static __device__ __align__(256) unsigned char scratch[kScratchBytes];

static std::mutex mu;
static void *addr[kMaxDevices];

static void set_msg(char *msg, size_t len, const char *fmt, ...) {
    if (!msg || len == 0) return;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, len, fmt, ap);
    va_end(ap);
}

// Device address of `scratch` on the current device, looked up once per
// device (cudaGetSymbolAddress with that device current).
static int scratch_addr(int dev, void **out, char *msg, size_t len) {
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            set_msg(msg, len, "bdg_densities_noalloc: cudaGetSymbolAddress failed on device %d: %s", dev,
                    cudaGetErrorString(e));
            return BDG_ECUDA;
        }
        addr[dev] = p;
    }
    *out = addr[dev];
    return BDG_OK;
}
}  // namespace noalloc
}  // namespace bdg

extern "C" int bdg_densities_noalloc(const bdg_grid *grid, int64_t n, const double *w, const double2 *Z,
                                     int64_t ldz, double T, double Ec, double *n_out, double2 *nu_out,
                                     cudaStream_t stream, char *msg, size_t msg_len) {
    using namespace bdg;
    if (msg && msg_len) msg[0] = 0;
    // the grid rule of every other entry point: nx >= 2, each size even or 1 (nx even), dx = 1
    if (!grid || grid->nx < 2 || grid->ny < 1 || grid->nz < 1 || grid->dx != 1.0 || (grid->nx & 1) ||
        (grid->ny > 1 && (grid->ny & 1)) || (grid->nz > 1 && (grid->nz & 1))) {
        noalloc::set_msg(msg, msg_len, "bdg_densities_noalloc: bad grid (sizes must be even or 1, nx >= 2, dx = 1)");
        return BDG_EINVAL;
    }
    const int64_t V = (int64_t)grid->nx * grid->ny * grid->nz;
    if (V > noalloc::kMaxSites) {
        noalloc::set_msg(msg, msg_len,
                         "bdg_densities_noalloc: %lld lattice sites exceed the fixed scratch limit of %lld "
                         "(4 MiB per device); use bdg_densities",
                         (long long)V, (long long)noalloc::kMaxSites);
        return BDG_EUNSUPPORTED;
    }
    if (n != 2 * V || !w || !Z || ldz < n || !n_out || !nu_out || T < 0) {
        noalloc::set_msg(msg, msg_len, "bdg_densities_noalloc: bad arguments");
        return BDG_EINVAL;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= noalloc::kMaxDevices) {
        cudaGetLastError();
        noalloc::set_msg(msg, msg_len, "bdg_densities_noalloc: no usable current device");
        return BDG_ECUDA;
    }
    void *base = nullptr;
    int rc = noalloc::scratch_addr(dev, &base, msg, msg_len);
    if (rc) return rc;

    const int64_t room = (int64_t)((noalloc::kScratchBytes - 768) / (24 * (size_t)V));
    int nsm = 148;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int64_t want = std::min<int64_t>(64, ((int64_t)nsm * 8 * 256) / V);
    const int nchunks = (int)std::max<int64_t>(1, std::min(want, room));
    unsigned char *p = (unsigned char *)base;
    int64_t *lohi = (int64_t *)p;
    double *pn = (double *)(p + 256);
    double2 *pnu = (double2 *)(p + 256 + align_up((size_t)nchunks * V * 8));

    window_kernel<<<1, 32, 0, stream>>>(n, w, Ec, lohi);
    dim3 g2((unsigned)((V + 255) / 256), (unsigned)nchunks);
    density_partial_kernel<<<g2, 256, 0, stream>>>(V, w, Z, ldz, lohi, T, nchunks, pn, pnu);
    density_reduce_kernel<<<(unsigned)((V + 255) / 256), 256, 0, stream>>>(V, nchunks, pn, pnu, n_out, nu_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        noalloc::set_msg(msg, msg_len, "bdg_densities_noalloc: launch failed: %s", cudaGetErrorString(e));
        return BDG_ECUDA;
    }
    return BDG_OK;
}
