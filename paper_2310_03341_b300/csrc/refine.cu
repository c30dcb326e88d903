// Ogita-Aishima iterative refinement of a full approximate eigendecomposition
// X, lambda of the BdG matrix (the eigenproblem of Eq. (stHpsi)); recovers
// FP64-level eigenpairs from the reduced-precision solve.
//
//   G = X^H X (so R = I - G),  S = X^H (H X),
//   lambda_i = Re S_ii / Re G_ii,
//   E_ii = (1 - G_ii) / 2,
//   E_ij = (S_ij - lambda_j G_ij) / (lambda_j - lambda_i)    |lambda_i - lambda_j| >  omega
//        = -G_ij / 2                                          otherwise,
//   X <- X + X E.
// H X is applied in FP64 through the Kronecker-sum structure of h (each row of
// the kinetic operator couples a site only to the sites on its three grid
// lines), so H is never formed.  G and S are the FP64-accurate products.
//
// Particle-hole reduction.  The BdG matrix satisfies P H P^-1 = -H with the
// antiunitary P x = C conj(x), C = [[0, I], [-I, 0]] (the partner of (u, v)
// at E is (conj v, -conj u) at -E).  With a gap at zero the vectors are kept
// as X = [X-, X+], column h-1-a of X- being P applied to column h+a (h = n/2),
// and the iteration needs only the h x h triangles
//   G++ = X+^H X+,  S++ = X+^H H X+         (Hermitian),
//   K = X+^T C X+  (skew-symmetric),  L = X+^T C H X+  (symmetric),
// from which every block of G and S follows:
//   G[h-1-a, h+b] = -K[a][b],    G[h-1-a, h-1-b] = conj G++[a][b],
//   S[h-1-a, h+b] = -L[a][b],    S[h-1-a, h-1-b] = -conj S++[a][b];
// only the X+ columns are updated (X+ <- X+ + X E[:, +]) and X- is
// regenerated from them, which halves every O(n^3) step.
#include <stdlib.h>

#include <algorithm>
#include <vector>

#include <cuda_bf16.h>

#include "internal.h"

namespace bdg {

int ozaki_slice(bdg_ctx *ctx, cudaStream_t st, int64_t rows, int64_t cols, const double2 *X, int64_t ldx,
                __nv_bfloat16 *planes, int *ex, int stored);
int ozaki_product(bdg_ctx *ctx, cudaStream_t st, int64_t rows, int64_t m, int64_t nc, const __nv_bfloat16 *px,
                  const int *ex, const __nv_bfloat16 *py, const int *ey, double2 *C, int64_t ldc, bool upper,
                  bool trans_a, bool cswap_b, int slices, int stored);
size_t ozaki_plane_bytes(int64_t rows, int64_t cols);
template <typename C>
int split_hilo(bdg_ctx *ctx, cudaStream_t st, int64_t rows, int64_t cols, const C *X, int64_t ldx, bool transpose,
               bool conj_, __nv_bfloat16 *planes);
int zgemm_bf16x3_add64(bdg_ctx *ctx, cudaStream_t st, int64_t M, int64_t N, int64_t K, const __nv_bfloat16 *pa,
                       const __nv_bfloat16 *pb, double2 *C, int64_t ldc, double alpha);


// Y = H X for ncols columns; one CTA per column, 256 threads over sites.
__global__ void __launch_bounds__(256) apply_h_kernel(int nx, int ny, int nz, double mu, const double *__restrict__ U,
                                                      const double2 *__restrict__ Delta,
                                                      const double *__restrict__ ktab, int64_t ncols,
                                                      const double2 *__restrict__ X, int64_t ldx,
                                                      double2 *__restrict__ Y, int64_t ldy) {
    extern __shared__ double sk[];
    const int nk = nx + ny + nz;
    for (int i = threadIdx.x; i < nk; i += blockDim.x) sk[i] = ktab[i];
    __syncthreads();
    const double *tx = sk, *ty = sk + nx, *tz = sk + nx + ny;
    const int64_t V = (int64_t)nx * ny * nz;
    const int64_t nyz = (int64_t)ny * nz;
    for (int64_t c = blockIdx.x; c < ncols; c += gridDim.x) {
        const double2 *u = X + c * ldx, *v = u + V;
        double2 *yu = Y + c * ldy, *yv = yu + V;
        for (int64_t s = threadIdx.x; s < V; s += blockDim.x) {
            const int ix = (int)(s / nyz), iy = (int)((s / nz) % ny), iz = (int)(s % nz);
            double2 tu = make_double2(0, 0), tv = make_double2(0, 0);
            const int64_t bx = s - (int64_t)ix * nyz;
            for (int jx = 0; jx < nx; ++jx) {
                double t = tx[(ix - jx + nx) % nx];
                double2 a = u[bx + (int64_t)jx * nyz], bq = v[bx + (int64_t)jx * nyz];
                tu.x = fma(t, a.x, tu.x); tu.y = fma(t, a.y, tu.y);
                tv.x = fma(t, bq.x, tv.x); tv.y = fma(t, bq.y, tv.y);
            }
            const int64_t by = s - (int64_t)iy * nz;
            for (int jy = 0; jy < ny; ++jy) {
                double t = ty[(iy - jy + ny) % ny];
                double2 a = u[by + (int64_t)jy * nz], bq = v[by + (int64_t)jy * nz];
                tu.x = fma(t, a.x, tu.x); tu.y = fma(t, a.y, tu.y);
                tv.x = fma(t, bq.x, tv.x); tv.y = fma(t, bq.y, tv.y);
            }
            const int64_t bz = s - iz;
            for (int jz = 0; jz < nz; ++jz) {
                double t = tz[(iz - jz + nz) % nz];
                double2 a = u[bz + jz], bq = v[bz + jz];
                tu.x = fma(t, a.x, tu.x); tu.y = fma(t, a.y, tu.y);
                tv.x = fma(t, bq.x, tv.x); tv.y = fma(t, bq.y, tv.y);
            }
            const double hd = U[s] - mu;
            const double2 us = u[s], vs = v[s], dl = Delta[s];
            double2 ou, ov;
            ou.x = tu.x + hd * us.x + (dl.x * vs.x - dl.y * vs.y);
            ou.y = tu.y + hd * us.y + (dl.x * vs.y + dl.y * vs.x);
            // conj(Delta) u - (T v + hd v)
            ov.x = (dl.x * us.x + dl.y * us.y) - (tv.x + hd * vs.x);
            ov.y = (dl.x * us.y - dl.y * us.x) - (tv.y + hd * vs.y);
            yu[s] = ou;
            yv[s] = ov;
        }
    }
}

// Y = H X for ncols columns (H from mu, U, Delta and the kinetic tables)
int launch_apply_h(bdg_ctx *ctx, int nx, int ny, int nz, double mu, const double *U, const double2 *Delta,
                   const double *ktab, int64_t ncols, const double2 *X, int64_t ldx, double2 *Y, int64_t ldy,
                   cudaStream_t st) {
    if (ncols <= 0) return BDG_OK;
    const int grid = (int)std::min<int64_t>(ncols, (int64_t)ctx->num_sms * 8);
    apply_h_kernel<<<grid, 256, (nx + ny + nz) * sizeof(double), st>>>(nx, ny, nz, mu, U, Delta, ktab, ncols, X,
                                                                      ldx, Y, ldy);
    BDG_LAUNCH_CHECK(ctx);
    return BDG_OK;
}

// per-column residual ||Y_i - w_i X_i||, block per column; writes res[i]
__global__ void col_resid_kernel(int64_t n, const double2 *__restrict__ X, int64_t ldx,
                                 const double2 *__restrict__ Y, int64_t ldy, const double *__restrict__ w,
                                 double *__restrict__ res) {
    __shared__ double sred[32];
    const int64_t c = blockIdx.x;
    const double lam = w[c];
    double acc = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
        double2 x = X[r + c * ldx], y = Y[r + c * ldy];
        double ax = y.x - lam * x.x, ay = y.y - lam * x.y;
        acc += ax * ax + ay * ay;
    }
    acc = block_sum(acc, sred);
    if (threadIdx.x == 0) res[c] = sqrt(acc);
}

// max over a vector (one block)
__global__ void max_abs_kernel(int64_t n, const double *__restrict__ v, double *__restrict__ out) {
    __shared__ double s[1024];
    double m = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(v[i]));
    s[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] = fmax(s[threadIdx.x], s[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

// lambda_i = Re S_ii / Re G_ii ; gdev_i = |G_ii - 1|
__global__ void oa_lambda_kernel(int64_t n, const double2 *__restrict__ G, int64_t ldg,
                                 const double2 *__restrict__ S, int64_t lds, double *__restrict__ lam) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    lam[i] = S[i + i * lds].x / G[i + i * ldg].x;
}

// per-column max |G_ij - delta_ij|
__global__ void orth_col_kernel(int64_t n, const double2 *__restrict__ G, int64_t ldg, double *__restrict__ out) {
    __shared__ double s[256];
    const int64_t c = blockIdx.x;
    double m = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
        double2 g = G[r + c * ldg];
        double dx = g.x - (r == c ? 1.0 : 0.0);
        m = fmax(m, sqrt(dx * dx + g.y * g.y));
    }
    s[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] = fmax(s[threadIdx.x], s[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = s[0];
}

// E (overwrites G): E_ij as in the header comment
__global__ void oa_e_kernel(int64_t n, double2 *__restrict__ G, int64_t ldg, const double2 *__restrict__ S,
                            int64_t lds, const double *__restrict__ lam, double omega) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    int64_t i = idx % n, j = idx / n;
    double2 g = G[i + j * ldg];
    double2 e;
    if (i == j) {
        e = make_double2(0.5 * (1.0 - g.x), -0.5 * g.y);
    } else {
        double li = lam[i], lj = lam[j], dl = lj - li;
        if (fabs(dl) > omega) {
            double2 s = S[i + j * lds];
            double inv = 1.0 / dl;
            e = make_double2((s.x - lj * g.x) * inv, (s.y - lj * g.y) * inv);
        } else {
            e = make_double2(-0.5 * g.x, -0.5 * g.y);
        }
    }
    G[i + j * ldg] = e;
}

// M <- (M + M^H)/2 in place (one thread per pair i < j, plus the diagonal)
__global__ void hermitize_kernel(int64_t n, double2 *__restrict__ M, int64_t ldm) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    int64_t i = idx % n, j = idx / n;
    if (i > j) return;
    double2 a = M[i + j * ldm];
    if (i == j) { M[i + j * ldm] = make_double2(a.x, 0.0); return; }
    double2 b = M[j + i * ldm];
    double2 h = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
    M[i + j * ldm] = h;
    M[j + i * ldm] = make_double2(h.x, -h.y);
}

// lower triangle from the upper one: M[i][j] = conj(M[j][i]) for i > j; real diagonal
__global__ void mirror_upper_kernel(int64_t n, double2 *__restrict__ M, int64_t ldm) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    int64_t i = idx % n, j = idx / n;
    if (i < j) return;
    if (i == j) { M[i + j * ldm].y = 0.0; return; }
    double2 u = M[j + i * ldm];
    M[i + j * ldm] = make_double2(u.x, -u.y);
}

__global__ void axpy_cols_kernel(int64_t n, int64_t ncols, double2 *__restrict__ X, int64_t ldx,
                                 const double2 *__restrict__ D, int64_t ldd) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * ncols) return;
    int64_t r = idx % n, c = idx / n;
    double2 a = X[r + c * ldx], b = D[r + c * ldd];
    X[r + c * ldx] = make_double2(a.x + b.x, a.y + b.y);
}

__global__ void rank_sort_kernel(int64_t n, const double *__restrict__ w, double *__restrict__ ws,
                                 int *__restrict__ perm) {
    __shared__ double tile[256];
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double wj = (j < n) ? w[j] : 0.0;
    int64_t rank = 0;
    for (int64_t base = 0; base < n; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        tile[threadIdx.x] = (i < n) ? w[i] : 0.0;
        __syncthreads();
        const int64_t lim = min((int64_t)blockDim.x, n - base);
        if (j < n)
            for (int q = 0; q < lim; ++q) {
                double wi = tile[q];
                int64_t ii = base + q;
                rank += (wi < wj || (wi == wj && ii < j)) ? 1 : 0;
            }
        __syncthreads();
    }
    if (j < n) { ws[rank] = wj; perm[rank] = (int)j; }
}

__global__ void permute_cols_kernel(int64_t n, const int *__restrict__ perm, const double2 *__restrict__ src,
                                    int64_t lds, double2 *__restrict__ dst, int64_t ldd) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    int64_t r = idx % n, c = idx / n;
    dst[r + c * ldd] = src[r + (int64_t)perm[c] * lds];
}

// ---------------------------------------------------------------------------
// cluster-aware step (Rayleigh-Ritz on strongly coupled neighbours)
// ---------------------------------------------------------------------------
// The first-order update E_ij = (S_ij - lambda_j G_ij)/(lambda_j - lambda_i)
// is only valid while |E_ij| << 1.  Neighbouring pairs (|i-j| <= W in the
// sorted order) with |E_ij| > tau are linked; maximal runs of linked indices
// are resolved exactly inside their span by a Rayleigh-Ritz rotation before
// the update:  M = (I - dG/2) S_cc (I - dG/2),  dG = G_cc - I,  M = V L V^H,
// W = (I - dG/2) V,  X_c <- X_c W,  G <- W^H G W,  S <- W^H S W.
constexpr int kLinkWindow = 16;
constexpr int kMaxCluster = 64;

// With the particle-hole reduction (split > 0) no link crosses the boundary
// between the halves: the partners of a pair near zero must stay in their
// halves, and their coupling (gap 2E) is left to the linear update.
__global__ void link_kernel(int64_t n, const double2 *__restrict__ G, int64_t ldg, const double2 *__restrict__ S,
                            int64_t lds, const double *__restrict__ lam, double tau, int64_t split,
                            int *__restrict__ reach) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int r = (int)i;
    const double li = lam[i];
    const int64_t jend = (split > 0 && i < split) ? split - 1 : n - 1;
    for (int64_t j = i + 1; j <= jend && j <= i + kLinkWindow; ++j) {
        double lj = lam[j];
        double2 sv = S[i + j * lds], gv = G[i + j * ldg];
        double ax = sv.x - lj * gv.x, ay = sv.y - lj * gv.y;
        double num = sqrt(ax * ax + ay * ay);
        double den = fabs(lj - li);
        if (num > tau * den) r = (int)j;
    }
    reach[i] = r;
}

// cluster ids from the reaches (one CTA): position p is linked to p+1 if
// some i <= p has reach[i] > p.  cstart[c], csize[c]; ccount[0] = #clusters.
__global__ void __launch_bounds__(1024) cluster_kernel(int64_t n, const int *__restrict__ reach,
                                                       int *__restrict__ cstart, int *__restrict__ csize,
                                                       int *__restrict__ ccount) {
    __shared__ int smax[1024];
    __shared__ int scnt[1024];
    const int T = blockDim.x, t = threadIdx.x;
    const int64_t cs = (n + T - 1) / T;
    const int64_t lo = min(n, (int64_t)t * cs), hi = min(n, lo + cs);
    int m = -1;
    for (int64_t i = lo; i < hi; ++i) m = max(m, reach[i]);
    smax[t] = m;
    __syncthreads();
    for (int off = 1; off < T; off <<= 1) {
        int a = smax[t], b = (t >= off) ? smax[t - off] : -1;
        __syncthreads();
        smax[t] = max(a, b);
        __syncthreads();
    }
    // linked[p] = (prefix max of reach over [0, p]) > p ; a cluster starts at p
    // if linked[p] and not linked[p-1]
    int run = (t == 0) ? -1 : smax[t - 1];
    int cnt = 0;
    int prevlinked = 0;
    if (lo > 0) { int rr = run; prevlinked = (rr > lo - 1) ? 1 : 0; }
    int r2 = run;
    for (int64_t p = lo; p < hi; ++p) {
        r2 = max(r2, reach[p]);
        int linked = r2 > p;
        if (linked && !prevlinked) ++cnt;
        prevlinked = linked;
    }
    scnt[t] = cnt;
    __syncthreads();
    for (int off = 1; off < T; off <<= 1) {
        int a = scnt[t], b = (t >= off) ? scnt[t - off] : 0;
        __syncthreads();
        scnt[t] = a + b;
        __syncthreads();
    }
    int id = (t == 0) ? 0 : scnt[t - 1];
    r2 = run;
    prevlinked = (lo > 0 && run > lo - 1) ? 1 : 0;
    for (int64_t p = lo; p < hi; ++p) {
        r2 = max(r2, reach[p]);
        int linked = r2 > p;
        if (linked && !prevlinked) { cstart[id] = (int)p; csize[id] = 0; ++id; }
        prevlinked = linked;
    }
    __syncthreads();
    if (t == T - 1) ccount[0] = scnt[T - 1];
}

__global__ void cluster_size_kernel(int64_t n, const int *__restrict__ reach, const int *__restrict__ cstart,
                                    const int *__restrict__ ccount, int *__restrict__ csize) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ccount[0]) return;
    int p = cstart[c];
    int r = reach[p];
    int q = p;
    while (q < r) { ++q; r = max(r, reach[q]); }
    csize[c] = q - p + 1;
}

// Cyclic Jacobi eigensolver of the Hermitian k x k matrix A (shared memory,
// column-major, leading dimension ld) run by one warp: for each pair (p, q)
// the phase of A[p][q] is removed (column q times e^{-i phi}, row q times
// e^{i phi}) and a real symmetric rotation zeroes it; lane r updates rows and
// columns r and r + 32.  On return V holds the eigenvectors and ev the
// eigenvalues in ascending order.  Sweeps stop when the off-diagonal mass is
// below 1e-34 of the total (or after 30).
__device__ void warp_herm_jacobi(int k, int ld, double2 *A, double2 *V, double *ev) {
    const int lane = threadIdx.x & 31;
    for (int r = lane; r < k; r += 32)
        for (int b = 0; b < k; ++b) V[r + b * ld] = make_double2(r == b ? 1.0 : 0.0, 0.0);
    __syncwarp();
    for (int sweep = 0; sweep < 30; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int e = lane; e < k * k; e += 32) {
            const int a = e % k, b = e / k;
            const double2 v = A[a + b * ld];
            const double m2 = v.x * v.x + v.y * v.y;
            tot += m2;
            if (a != b) off += m2;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
        }
        if (off <= 1e-34 * tot || off == 0.0) break;
        for (int p = 0; p < k - 1; ++p)
            for (int q = p + 1; q < k; ++q) {
                const double2 apq = A[p + q * ld];
                const double mag = sqrt(apq.x * apq.x + apq.y * apq.y);
                if (mag == 0.0) continue;
                const double cph = apq.x / mag, sph = apq.y / mag;   // e^{i phi}
                // phase: the (q, q) entry is touched by column and row; lane of row q does both in order
                for (int r = lane; r < k; r += 32) {
                    double2 x = A[r + q * ld];
                    A[r + q * ld] = make_double2(x.x * cph + x.y * sph, x.y * cph - x.x * sph);
                    x = V[r + q * ld];
                    V[r + q * ld] = make_double2(x.x * cph + x.y * sph, x.y * cph - x.x * sph);
                }
                __syncwarp();
                for (int r = lane; r < k; r += 32) {
                    const double2 x = A[q + r * ld];
                    A[q + r * ld] = make_double2(x.x * cph - x.y * sph, x.y * cph + x.x * sph);
                }
                __syncwarp();
                const double app = A[p + p * ld].x, aqq = A[q + q * ld].x, apr = A[p + q * ld].x;
                const double th = (aqq - app) / (2.0 * apr);
                const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(1.0 + th * th));
                const double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
                __syncwarp();
                for (int r = lane; r < k; r += 32) {   // A <- A J (columns p, q); V <- V J
                    const double2 ap = A[r + p * ld], aq = A[r + q * ld];
                    A[r + p * ld] = make_double2(c * ap.x - sn * aq.x, c * ap.y - sn * aq.y);
                    A[r + q * ld] = make_double2(sn * ap.x + c * aq.x, sn * ap.y + c * aq.y);
                    const double2 vp = V[r + p * ld], vq = V[r + q * ld];
                    V[r + p * ld] = make_double2(c * vp.x - sn * vq.x, c * vp.y - sn * vq.y);
                    V[r + q * ld] = make_double2(sn * vp.x + c * vq.x, sn * vp.y + c * vq.y);
                }
                __syncwarp();
                for (int r = lane; r < k; r += 32) {   // A <- J^T A (rows p, q)
                    const double2 ap = A[p + r * ld], aq = A[q + r * ld];
                    A[p + r * ld] = make_double2(c * ap.x - sn * aq.x, c * ap.y - sn * aq.y);
                    A[q + r * ld] = make_double2(sn * ap.x + c * aq.x, sn * ap.y + c * aq.y);
                }
                __syncwarp();
                if (lane == 0) {
                    A[p + q * ld] = make_double2(0.0, 0.0);
                    A[q + p * ld] = make_double2(0.0, 0.0);
                }
                __syncwarp();
            }
    }
    if (lane == 0) {
        for (int a = 0; a < k; ++a) ev[a] = A[a + a * ld].x;
        // selection sort ascending with the columns of V
        for (int a = 0; a < k; ++a) {
            int best = a;
            for (int b = a + 1; b < k; ++b) if (ev[b] < ev[best]) best = b;
            if (best != a) {
                const double t = ev[a]; ev[a] = ev[best]; ev[best] = t;
                for (int r = 0; r < k; ++r) {
                    const double2 x = V[r + a * ld]; V[r + a * ld] = V[r + best * ld]; V[r + best * ld] = x;
                }
            }
        }
    }
    __syncwarp();
}

// One CTA per cluster: W = (I - dG/2) V (stored in wbuf at woff[c]), lam
// updated.  The three k x k work matrices live in shared memory (leading
// dimension ld = kmax + 1); the products are spread over the CTA's threads,
// the Jacobi rotations run on warp 0.
constexpr int kRrThreads = 128;
__global__ void __launch_bounds__(kRrThreads) cluster_rr_kernel(const double2 *__restrict__ G, int64_t ldg,
                                                               const double2 *__restrict__ S, int64_t lds,
                                                               const int *__restrict__ cstart,
                                                               const int *__restrict__ csize,
                                                               const int *__restrict__ ccount,
                                                               const int64_t *__restrict__ woff,
                                                               double *__restrict__ lam, double2 *__restrict__ wbuf,
                                                               int ld, int *__restrict__ overflow) {
    extern __shared__ double2 rr_smem[];
    const int c = blockIdx.x;
    if (c >= ccount[0]) return;
    const int p0 = cstart[c], k = csize[c];
    if (k < 2) return;
    if (k > kMaxCluster || k >= ld) {
        if (threadIdx.x == 0) atomicAdd(overflow, 1);
        return;
    }
    double2 *Mm = rr_smem;                  // S_cc, then (I - dG/2) S_cc (I - dG/2)
    double2 *Lh = Mm + (int64_t)ld * ld;    // I - dG/2
    double2 *Tm = Lh + (int64_t)ld * ld;    // S_cc Lh, then the eigenvectors
    double *ev = reinterpret_cast<double *>(Tm + (int64_t)ld * ld);
    double2 *W = wbuf + woff[c];
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < k * k; e += nt) {
        const int a = e % k, b = e / k;
        const double2 gv = G[(p0 + a) + (int64_t)(p0 + b) * ldg];
        Lh[a + b * ld] = make_double2((a == b ? 1.0 : 0.0) - 0.5 * (gv.x - (a == b ? 1.0 : 0.0)), -0.5 * gv.y);
        Mm[a + b * ld] = S[(p0 + a) + (int64_t)(p0 + b) * lds];
    }
    __syncthreads();
    // Tm = S_cc Lh ; Mm = Lh^H Tm  (Lh is Hermitian)
    for (int e = tid; e < k * k; e += nt) {
        const int a = e % k, b = e / k;
        double2 acc = make_double2(0, 0);
        for (int q = 0; q < k; ++q) {
            const double2 sv = Mm[a + q * ld], l = Lh[q + b * ld];
            acc.x += sv.x * l.x - sv.y * l.y;
            acc.y += sv.x * l.y + sv.y * l.x;
        }
        Tm[a + b * ld] = acc;
    }
    __syncthreads();
    for (int e = tid; e < k * k; e += nt) {
        const int a = e % k, b = e / k;
        double2 acc = make_double2(0, 0);
        for (int q = 0; q < k; ++q) {
            const double2 l = Lh[q + a * ld];   // (Lh^H)[a][q] = conj(Lh[q][a])
            const double2 t = Tm[q + b * ld];
            acc.x += l.x * t.x + l.y * t.y;
            acc.y += l.x * t.y - l.y * t.x;
        }
        Mm[a + b * ld] = acc;
    }
    __syncthreads();
    // Hermitian part (each unordered pair by one thread)
    for (int e = tid; e < k * k; e += nt) {
        const int a = e % k, b = e / k;
        if (a < b) continue;
        const double2 x = Mm[a + b * ld], y = Mm[b + a * ld];
        const double2 h = make_double2(0.5 * (x.x + y.x), 0.5 * (x.y - y.y));
        Mm[a + b * ld] = h;
        Mm[b + a * ld] = make_double2(h.x, -h.y);
    }
    __syncthreads();
    if (tid < 32) warp_herm_jacobi(k, ld, Mm, Tm, ev);
    __syncthreads();
    // W = Lh V
    for (int e = tid; e < k * k; e += nt) {
        const int a = e % k, b = e / k;
        double2 acc = make_double2(0, 0);
        for (int q = 0; q < k; ++q) {
            const double2 l = Lh[a + q * ld], v = Tm[q + b * ld];
            acc.x += l.x * v.x - l.y * v.y;
            acc.y += l.x * v.y + l.y * v.x;
        }
        W[a + b * k] = acc;
    }
    for (int a = tid; a < k; a += nt) lam[p0 + a] = ev[a];
}

// M[:, c] <- M[:, c] W_c for every cluster (right multiplication); one thread
// per (row, cluster).
__global__ void cluster_right_kernel(int64_t nrows, double2 *__restrict__ M, int64_t ldm,
                                     const int *__restrict__ cstart, const int *__restrict__ csize,
                                     const int *__restrict__ ccount, const int64_t *__restrict__ woff,
                                     const double2 *__restrict__ wbuf) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int c = blockIdx.y;
    if (r >= nrows || c >= ccount[0]) return;
    const int p0 = cstart[c], k = csize[c];
    if (k < 2 || k > kMaxCluster) return;
    const double2 *W = wbuf + woff[c];
    double2 row[kMaxCluster];
    for (int q = 0; q < k; ++q) row[q] = M[r + (int64_t)(p0 + q) * ldm];
    for (int b = 0; b < k; ++b) {
        double2 acc = make_double2(0, 0);
        for (int q = 0; q < k; ++q) {
            double2 w = W[q + b * k];
            acc.x += row[q].x * w.x - row[q].y * w.y;
            acc.y += row[q].x * w.y + row[q].y * w.x;
        }
        M[r + (int64_t)(p0 + b) * ldm] = acc;
    }
}

// M[c, :] <- W_c^H M[c, :] (left multiplication); one thread per (column, cluster).
__global__ void cluster_left_kernel(int64_t ncols, double2 *__restrict__ M, int64_t ldm,
                                    const int *__restrict__ cstart, const int *__restrict__ csize,
                                    const int *__restrict__ ccount, const int64_t *__restrict__ woff,
                                    const double2 *__restrict__ wbuf) {
    int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int c = blockIdx.y;
    if (col >= ncols || c >= ccount[0]) return;
    const int p0 = cstart[c], k = csize[c];
    if (k < 2 || k > kMaxCluster) return;
    const double2 *W = wbuf + woff[c];
    double2 v[kMaxCluster];
    for (int q = 0; q < k; ++q) v[q] = M[(p0 + q) + col * ldm];
    for (int a = 0; a < k; ++a) {
        double2 acc = make_double2(0, 0);
        for (int q = 0; q < k; ++q) {
            double2 w = W[q + a * k];   // conj(W[q][a])
            acc.x += w.x * v[q].x + w.y * v[q].y;
            acc.y += w.x * v[q].y - w.y * v[q].x;
        }
        M[(p0 + a) + col * ldm] = acc;
    }
}

// Full G (or S) from the ++ triangle stored in M[h:, h:] (entries a <= b
// valid) and the cross triangle Q (h x h, entries a < b valid for the
// skew-symmetric K, a <= b for the symmetric L).  For G: cross = -K, minus
// block = conj(++); for S (is_s): cross = -L, minus block = -conj(++).
__global__ void ph_assemble_kernel(int64_t h, double2 *__restrict__ M, int64_t ldm, const double2 *__restrict__ Q,
                                   int64_t ldq, int is_s) {
    const int64_t n = 2 * h;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    const int64_t r = idx % n, c = idx / n;
    auto pp = [&](int64_t a, int64_t b) -> double2 {   // (++)[a][b] from the upper triangle
        if (a <= b) {
            double2 v = M[(h + a) + (h + b) * ldm];
            if (a == b) v.y = 0.0;
            return v;
        }
        double2 v = M[(h + b) + (h + a) * ldm];
        return make_double2(v.x, -v.y);
    };
    auto cross = [&](int64_t a, int64_t b) -> double2 {   // K[a][b] or L[a][b]
        if (a == b) return is_s ? Q[a + b * ldq] : make_double2(0.0, 0.0);
        if (a < b) return Q[a + b * ldq];
        double2 v = Q[b + a * ldq];
        return is_s ? v : make_double2(-v.x, -v.y);
    };
    double2 out;
    if (r >= h && c >= h) {
        out = pp(r - h, c - h);
    } else if (r < h && c >= h) {
        double2 v = cross(h - 1 - r, c - h);
        out = make_double2(-v.x, -v.y);
    } else if (r >= h && c < h) {
        double2 v = cross(h - 1 - c, r - h);   // conj(M[c][r]) with M[c][r] = -cross(h-1-c, r-h)
        out = make_double2(-v.x, v.y);
    } else {
        double2 v = pp(h - 1 - r, h - 1 - c);
        out = is_s ? make_double2(-v.x, v.y) : make_double2(v.x, -v.y);
    }
    M[r + c * ldm] = out;
}

size_t refine_workspace_bytes(int64_t n) {
    const size_t nn = (size_t)n * n;
    const size_t cl_budget = std::min<size_t>((size_t)n * 4 * 64 * 16 + (16 << 20), (size_t)4 << 30);
    return 3 * align_up(nn * 16) + 2 * align_up(ozaki_plane_bytes(n, n)) + 12 * align_up((size_t)n * 8) +
           align_up(4096) + (2 << 20) + cl_budget;
}

int refine_impl(bdg_ctx *ctx, const bdg_grid *g, double mu, const double *U, const double2 *Delta, int64_t n,
                double *w, double2 *Z, int64_t ldz, int max_iter, double tol, double *resid_out, double *orth_out,
                int *iters_out, cudaStream_t st) {
    const size_t nn = (size_t)n * n;
    const int64_t h = n / 2;
    const char *fp64p = getenv("BDG_REFINE_FP64_GEMM");
    const bool tensor = !(fp64p && atoi(fp64p));
    // particle-hole reduction: needs the tensor-core products and a spectrum
    // split at zero (w[h-1] < 0 < w[h], not degenerate within omega); decided
    // on a host copy of the eigenvalue estimates before the workspace is sized
    bool ph = false;
    {
        std::vector<double> hw((size_t)n);
        BDG_CUDA_TRY(ctx, cudaMemcpyAsync(hw.data(), w, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, st));
        BDG_CUDA_TRY(ctx, cudaStreamSynchronize(st));
        double rho0 = 0.0;
        for (int64_t i = 0; i < n; ++i) rho0 = std::max(rho0, std::fabs(hw[(size_t)i]));
        if (rho0 <= 0.0) rho0 = 1.0;
        const double wm = hw[(size_t)(h - 1)], wp = hw[(size_t)h];
        const char *full = getenv("BDG_REFINE_FULL");
        ph = tensor && n >= 2 && !(full && atoi(full)) && wm < 0.0 && wp > 0.0 && (wp - wm) > 2e-8 * rho0;
    }
    const int64_t c0 = ph ? h : 0, nc = ph ? h : n;   // refined columns
    const size_t plane_bytes = ozaki_plane_bytes(n, nc);
    // cluster scratch budget: up to n/8 clusters (4 k^2 complex entries each, k <= 64), capped at 4 GiB
    size_t need = ctx->ws_top + refine_workspace_bytes(n) - 2 * align_up(ozaki_plane_bytes(n, n)) +
                  2 * align_up(plane_bytes);
    if (need > ctx->ws_bytes) {
        // the caller's buffers are not in the arena, so it may be regrown here
        if (ctx->ws_top != 0) return bdg_fail(ctx, BDG_ENOMEM, "refine: workspace arena too small");
        int rc = ws_reserve(ctx, need);
        if (rc) return rc;
    }
    double2 *Y = (double2 *)ws_take(ctx, nn * 16);
    double2 *G = (double2 *)ws_take(ctx, nn * 16);
    double2 *S = (double2 *)ws_take(ctx, nn * 16);
    double *lam = (double *)ws_take(ctx, (size_t)n * 8);
    double *res = (double *)ws_take(ctx, (size_t)n * 8);
    double *ocol = (double *)ws_take(ctx, (size_t)n * 8);
    double *wsrt = (double *)ws_take(ctx, (size_t)n * 8);
    int *perm = (int *)ws_take(ctx, (size_t)n * 8);
    double *scal = (double *)ws_take(ctx, 64);
    double *ktab = (double *)ws_take(ctx, 4096);
    int *reach = (int *)ws_take(ctx, (size_t)n * 4);
    int *cstart = (int *)ws_take(ctx, (size_t)n * 4);
    int *csize = (int *)ws_take(ctx, (size_t)n * 4);
    int *ccount = (int *)ws_take(ctx, 64);
    __nv_bfloat16 *ozX = (__nv_bfloat16 *)ws_take(ctx, plane_bytes);
    __nv_bfloat16 *ozY = (__nv_bfloat16 *)ws_take(ctx, plane_bytes);
    int *exX = (int *)ws_take(ctx, (size_t)n * 4);
    int *exY = (int *)ws_take(ctx, (size_t)n * 4);
    if (!ozX || !ozY || !exX || !exY) return bdg_fail(ctx, BDG_ENOMEM, "refine: workspace (slices)");
    if (!Y || !G || !S || !ktab || !ccount) return bdg_fail(ctx, BDG_ENOMEM, "refine: workspace");
    const size_t mark = ctx->ws_top;   // per-iteration cluster scratch is taken above this mark
    BDG_CUDA_TRY(ctx, cudaMemsetAsync(ccount, 0, 64, st));
    int rc = launch_kinetic_tables(ctx, g->nx, g->ny, g->nz, ktab, st);
    if (rc) return rc;
    const double2 one = make_double2(1, 0), zero = make_double2(0, 0);
    const int nk = g->nx + g->ny + g->nz;
    ctx->last_refine_ph = ph ? 1 : 0;
    if (ph) {
        rc = launch_ph_fill<double>(ctx, n, Z, ldz, w, st);
        if (rc) return rc;
    }
    double2 *Zc = Z + c0 * ldz;
    double2 *Kq = Y + n * h, *Lq = Kq + h * h;        // PH cross triangles (free half of Y)
    const int apply_grid = (int)std::min<int64_t>(nc, (int64_t)ctx->num_sms * 8);
    // pairs with |E_ij| above link_tau go to the cluster Rayleigh-Ritz step.  After the
    // FP32-accurate solves (BF16X9, FP32) the small threshold 0.005 resolves the close pairs
    // that would otherwise converge slowly; the split-precision modes BF16X3 / BF16X6
    // (truncating tensor-core accumulation) leave starts whose long coupled chains it does
    // not handle, and vectors from elsewhere get the same conservative 0.05
    const char *tau_env = getenv("BDG_REFINE_TAU");
    const int hp = ctx->last_heev_prec;
    const double link_tau = tau_env ? atof(tau_env)
                                    : ((hp == BDG_PREC_BF16X9 || hp == BDG_PREC_FP32) ? 0.005 : 0.05);
    double resid = 0, orth = 0, rho = 1;
    int it = 0;
    bool converged = false;
    auto check_flags = [&]() -> int {
        int fl[2];
        BDG_CUDA_TRY(ctx, cudaMemcpy(fl, ctx->dflags + 4, sizeof(fl), cudaMemcpyDeviceToHost));
        if (fl[0] || fl[1])
            return bdg_fail(ctx, BDG_ETIMEOUT, "refine: a tensor-core pipeline wait gave up (codes %d, %d)", fl[0],
                            fl[1]);
        return BDG_OK;
    };
    for (;; ++it) {
        apply_h_kernel<<<apply_grid, 256, nk * sizeof(double), st>>>(g->nx, g->ny, g->nz, mu, U, Delta, ktab, nc, Zc,
                                                                     ldz, Y, n);
        BDG_LAUNCH_CHECK(ctx);
        stage_mark(ctx, st, "ref_apply_h");
        // residuals of the refined columns (the partners have the same ones)
        col_resid_kernel<<<(unsigned)nc, 256, 0, st>>>(n, Zc, ldz, Y, n, w + c0, res);
        BDG_LAUNCH_CHECK(ctx);
        max_abs_kernel<<<1, 1024, 0, st>>>(nc, res, scal);
        max_abs_kernel<<<1, 1024, 0, st>>>(n, w, scal + 1);
        BDG_LAUNCH_CHECK(ctx);
        BDG_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->hscal, scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        BDG_CUDA_TRY(ctx, cudaStreamSynchronize(st));
        rho = ctx->hscal[1] > 0 ? ctx->hscal[1] : 1.0;
        resid = ctx->hscal[0] / rho;
        stage_mark(ctx, st, "ref_check");
        // the stopping test is the residual alone; the final Gram matrix is
        // formed only when the caller asks for the orthogonality
        const bool stop = resid <= tol || it >= max_iter;
        if (stop && !orth_out) {
            rc = check_flags();
            if (rc) return rc;
            converged = resid <= tol;
            break;
        }
        // Slices of this iteration's products.  The first iteration starts from vectors whose
        // pairwise mixing is ~1e-3 and needs products to ~1e-10 only: 4 slices.  Later ones need
        // products below the target: 5 slices reach a residual of ~2e-11 rho, so 5 for
        // tol >= 5e-11 and 6 (FP64 level) below; the final orthogonality check uses 6.
        int nsl = (it == 0) ? 4 : (tol >= 5e-11 ? 5 : 6);
        if (ctx->refine_nslices > 0) nsl = ctx->refine_slices[std::min(it, ctx->refine_nslices - 1)];
        if (stop) nsl = 6;
        // G = X^H X
        if (tensor) {
            rc = ozaki_slice(ctx, st, n, nc, Zc, ldz, ozX, exX, nsl);
            if (rc) return rc;
            stage_mark(ctx, st, "ref_slice_x");
            rc = ozaki_product(ctx, st, n, nc, nc, ozX, exX, ozX, exX, G + c0 + c0 * n, n, true, false, false, nsl, nsl);
            if (!rc && ph) rc = ozaki_product(ctx, st, n, h, h, ozX, exX, ozX, exX, Kq, h, true, true, true, nsl, nsl);
            if (rc) return rc;
            stage_mark(ctx, st, nsl == 4 ? "ref_oz_gram_s4" : nsl == 5 ? "ref_oz_gram_s5" : "ref_oz_gram_s6");
            if (ph)
                ph_assemble_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(h, G, n, Kq, h, 0);
            else
                mirror_upper_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(n, G, n);
        } else {
            rc = gemm<double>(ctx, st, 'C', 'N', n, n, n, one, Z, ldz, Z, ldz, zero, G, n);
            if (rc) return rc;
        }
        orth_col_kernel<<<(unsigned)n, 256, 0, st>>>(n, G, n, ocol);
        max_abs_kernel<<<1, 1024, 0, st>>>(n, ocol, scal + 2);
        BDG_LAUNCH_CHECK(ctx);
        BDG_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->hscal + 2, scal + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
        BDG_CUDA_TRY(ctx, cudaStreamSynchronize(st));
        rc = check_flags();
        if (rc) return rc;
        orth = ctx->hscal[2];
        stage_mark(ctx, st, "ref_orth");
        if (stop) { converged = resid <= tol; break; }
        // S = X^H (H X)
        if (tensor) {
            rc = ozaki_slice(ctx, st, n, nc, Y, n, ozY, exY, nsl);
            if (rc) return rc;
            stage_mark(ctx, st, "ref_slice_y");
            rc = ozaki_product(ctx, st, n, nc, nc, ozX, exX, ozY, exY, S + c0 + c0 * n, n, true, false, false, nsl, nsl);
            if (!rc && ph) rc = ozaki_product(ctx, st, n, h, h, ozX, exX, ozY, exY, Lq, h, true, true, true, nsl, nsl);
            if (rc) return rc;
            stage_mark(ctx, st, nsl == 4 ? "ref_oz_s_s4" : nsl == 5 ? "ref_oz_s_s5" : "ref_oz_s_s6");
            if (ph)
                ph_assemble_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(h, S, n, Lq, h, 1);
            else
                mirror_upper_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(n, S, n);
        } else {
            rc = gemm<double>(ctx, st, 'C', 'N', n, n, n, one, Z, ldz, Y, n, zero, S, n);
            if (rc) return rc;
            hermitize_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(n, G, n);
            hermitize_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(n, S, n);
        }
        stage_mark(ctx, st, "ref_mirror");
        oa_lambda_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, G, n, S, n, lam);
        // cluster-aware step: Rayleigh-Ritz on strongly coupled neighbours.  The link
        // threshold starts at link_tau and is raised (x5, at most to 0.05) while a coupled
        // chain would exceed kMaxCluster members (a poor start couples long runs)
        int ncl = 0;
        std::vector<int> hsize;
        for (double tau = link_tau;; tau = std::min(0.05, tau * 5.0)) {
            link_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, G, n, S, n, lam, tau, ph ? h : 0, reach);
            cluster_kernel<<<1, 1024, 0, st>>>(n, reach, cstart, csize, ccount);
            cluster_size_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, reach, cstart, ccount, csize);
            BDG_LAUNCH_CHECK(ctx);
            BDG_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->hflags, ccount, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
            BDG_CUDA_TRY(ctx, cudaStreamSynchronize(st));
            ncl = ctx->hflags[0];
            hsize.assign((size_t)std::max(ncl, 0), 0);
            if (ncl > 0)
                BDG_CUDA_TRY(ctx, cudaMemcpy(hsize.data(), csize, (size_t)ncl * 4, cudaMemcpyDeviceToHost));
            const bool fits = std::all_of(hsize.begin(), hsize.end(), [](int k) { return k <= kMaxCluster; });
            if (fits || tau >= 0.05) break;
        }
        if (ncl > 0) {
            // compact per-cluster storage: offsets of k^2 entries
            std::vector<int64_t> hoff(ncl);
            int64_t tot = 0;
            int too_big = 0;
            for (int c = 0; c < ncl; ++c) {
                hoff[c] = tot;
                int k = hsize[c];
                if (k > kMaxCluster) { ++too_big; k = 0; }
                tot += (int64_t)k * k;
            }
            if (too_big)
                return bdg_fail(ctx, BDG_EUNSUPPORTED, "refine: %d coupled clusters larger than %d", too_big,
                                kMaxCluster);
            ctx->ws_top = mark;
            int64_t *woff = (int64_t *)ws_take(ctx, (size_t)ncl * 8);
            double2 *wbuf = (double2 *)ws_take(ctx, (size_t)(tot + 1) * 16);
            if (!woff || !wbuf)
                return bdg_fail(ctx, BDG_ENOMEM, "refine: %d coupled clusters exceed the workspace", ncl);
            BDG_CUDA_TRY(ctx, cudaMemcpyAsync(woff, hoff.data(), (size_t)ncl * 8, cudaMemcpyHostToDevice, st));
            const int kmax = *std::max_element(hsize.begin(), hsize.end());
            const int rld = kmax + 1;
            const size_t rsm = (size_t)3 * rld * rld * sizeof(double2) + (size_t)rld * sizeof(double);
            BDG_CUDA_TRY(ctx, cudaFuncSetAttribute(cluster_rr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)rsm));
            cluster_rr_kernel<<<(unsigned)ncl, kRrThreads, rsm, st>>>(G, n, S, n, cstart, csize, ccount, woff, lam,
                                                                     wbuf, rld, ccount + 1);
            BDG_LAUNCH_CHECK(ctx);
            for (int q0 = 0; q0 < ncl; q0 += 65535) {
                int cc = std::min(65535, ncl - q0);
                dim3 gr((unsigned)((n + 127) / 128), (unsigned)cc);
                cluster_right_kernel<<<gr, 128, 0, st>>>(n, Z, ldz, cstart + q0, csize + q0, ccount, woff + q0, wbuf);
                cluster_right_kernel<<<gr, 128, 0, st>>>(n, G, n, cstart + q0, csize + q0, ccount, woff + q0, wbuf);
                cluster_right_kernel<<<gr, 128, 0, st>>>(n, S, n, cstart + q0, csize + q0, ccount, woff + q0, wbuf);
                cluster_left_kernel<<<gr, 128, 0, st>>>(n, G, n, cstart + q0, csize + q0, ccount, woff + q0, wbuf);
                cluster_left_kernel<<<gr, 128, 0, st>>>(n, S, n, cstart + q0, csize + q0, ccount, woff + q0, wbuf);
                BDG_LAUNCH_CHECK(ctx);
            }
        }
        const double omega = 1e-8 * rho;
        oa_e_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(n, G, n, S, n, lam, omega);
        BDG_LAUNCH_CHECK(ctx);
        stage_mark(ctx, st, "ref_clusters_E");
        // X(:, refined) += X E(:, refined)
        if (tensor) {
            // E is small (|E| ~ the current error), so split (hi+lo) bf16 products suffice
            rc = split_hilo<double2>(ctx, st, n, n, Z, ldz, true, false, ozX);
            if (!rc) rc = split_hilo<double2>(ctx, st, n, nc, G + c0 * n, n, false, false, ozY);
            if (!rc) rc = zgemm_bf16x3_add64(ctx, st, n, nc, n, ozX, ozY, Zc, ldz, 1.0);
            if (rc) return rc;
        } else {
            rc = gemm<double>(ctx, st, 'N', 'N', n, n, n, one, Z, ldz, G, n, zero, Y, n);
            if (rc) return rc;
            axpy_cols_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(n, n, Z, ldz, Y, n);
        }
        stage_mark(ctx, st, "ref_update_xe");
        // eigenvalue estimates in ascending order, vectors permuted with them
        rank_sort_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, lam, wsrt, perm);
        permute_cols_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(n, perm, Z, ldz, S, n);
        BDG_LAUNCH_CHECK(ctx);
        BDG_CUDA_TRY(ctx, cudaMemcpy2DAsync(Z, ldz * 16, S, n * 16, n * 16, n, cudaMemcpyDeviceToDevice, st));
        BDG_CUDA_TRY(ctx, cudaMemcpyAsync(w, wsrt, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        if (ph) {
            // the minus half: partners of the refined plus half
            rc = launch_ph_fill<double>(ctx, n, Z, ldz, w, st);
            if (rc) return rc;
        }
    }
    if (resid_out) *resid_out = resid;
    if (orth_out) *orth_out = orth;
    if (iters_out) *iters_out = it;
    if (!converged)
        return bdg_fail(ctx, BDG_ENOCONV, "refine: residual %.3e above tol %.3e after %d iterations", resid, tol, it);
    return BDG_OK;
}

}  // namespace bdg
