/*
 * Plain FP64 CPU oracle for the static BdG eigenproblem (test infrastructure).
 *
 * This file is test infrastructure, not the product: only the tests, the smoke entry
 * point and the benchmark's CPU-baseline leg may call it.  It shares no code,
 * header or table with the CUDA library.  Every routine is the textbook
 * definition, unblocked and in FP64, so that it can be read against the paper:
 *
 *   - the kinetic operator -1/2 nabla^2 = F^-1 (k^2/2) F on the periodic grid,
 *     k = 2 pi m / n, m = -n/2 .. n/2-1 (paper, "Numerical setup and
 *     implementation", kinetic-term equation), evaluated as the explicit
 *     inverse-DFT sum for every matrix element;
 *   - the quasiparticle Hamiltonian [[h, Delta], [Delta^*, -h^*]] of Eq.
 *     (stHpsi), h = T + U - mu, Delta local;
 *   - unblocked Householder reduction of the complex Hermitian matrix to a
 *     Hermitian tridiagonal (Golub & Van Loan, Algorithm 8.3.1, complex form,
 *     reflectors with real tau), then a diagonal unitary that makes the
 *     off-diagonal real;
 *   - the implicit symmetric QR algorithm with Wilkinson shifts for the real
 *     symmetric tridiagonal (Golub & Van Loan, Algorithm 8.3.3),
 *     optionally accumulating its plane rotations into the eigenvectors;
 *   - the back-transformation by the stored reflectors;
 *   - a matrix-free H*x built from the same matrix elements (Kronecker sum of
 *     the three 1-D kinetic matrices), for residual checks at sizes where the
 *     dense matrix is not formed.
 *
 * Layout: dense matrices are column-major, element (i, j) at a[i + j*ld].
 * Site index s = (ix*ny + iy)*nz + iz; rows 0..V-1 hold u, rows V..2V-1 hold v.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* 1-D kinetic matrix T (n x n, column-major) from the inverse-DFT definition:
 * T[a][b] = (1/n) sum_m (k_m^2 / 2) exp(i k_m (a - b)).  The imaginary parts
 * of the terms +m and -m cancel and the m = -n/2 term is real, so T is real;
 * the imaginary part of the sum is returned in `imag_max` for checking. */
void orc_kinetic_1d(int n, double *T, double *imag_max) {
    double im_max = 0.0;
    for (int a = 0; a < n; ++a) {
        for (int b = 0; b < n; ++b) {
            cplx acc = 0.0;
            /* the lattice k set: m = -floor(n/2) .. n - floor(n/2) - 1 (for even n -n/2 .. n/2-1,
               with the Nyquist mode at m = -n/2; for odd n symmetric; for n = 1 only k = 0) */
            for (int m = -(n / 2); m <= n - n / 2 - 1; ++m) {
                double k = 2.0 * M_PI * (double)m / (double)n;
                acc += 0.5 * k * k * cexp(I * k * (double)(a - b));
            }
            acc /= (double)n;
            T[a + (size_t)b * n] = creal(acc);
            if (fabs(cimag(acc)) > im_max) im_max = fabs(cimag(acc));
        }
    }
    if (imag_max) *imag_max = im_max;
}

/* Dense BdG matrix H (N x N, N = 2V, column-major, leading dimension ldh). */
void orc_build(int nx, int ny, int nz, double mu, const double *U,
               const cplx *Delta, cplx *H, int64_t ldh) {
    const int64_t V = (int64_t)nx * ny * nz, N = 2 * V;
    double *Tx = malloc(sizeof(double) * nx * nx);
    double *Ty = malloc(sizeof(double) * ny * ny);
    double *Tz = malloc(sizeof(double) * nz * nz);
    orc_kinetic_1d(nx, Tx, NULL);
    orc_kinetic_1d(ny, Ty, NULL);
    orc_kinetic_1d(nz, Tz, NULL);
    for (int64_t j = 0; j < N; ++j)
        for (int64_t i = 0; i < N; ++i) H[i + j * ldh] = 0.0;
    for (int64_t s = 0; s < V; ++s) {
        int ix = (int)(s / ((int64_t)ny * nz)), iy = (int)((s / nz) % ny), iz = (int)(s % nz);
        for (int64_t t = 0; t < V; ++t) {
            int jx = (int)(t / ((int64_t)ny * nz)), jy = (int)((t / nz) % ny), jz = (int)(t % nz);
            double h = 0.0;
            if (iy == jy && iz == jz) h += Tx[ix + (size_t)jx * nx];
            if (ix == jx && iz == jz) h += Ty[iy + (size_t)jy * ny];
            if (ix == jx && iy == jy) h += Tz[iz + (size_t)jz * nz];
            if (s == t) h += U[s] - mu;
            if (h == 0.0) continue;
            /* upper-left h, lower-right -conj(h) (h is real here: T and U are real) */
            H[s + t * ldh] = h;
            H[(V + s) + (V + t) * ldh] = -conj((cplx)h);
        }
        H[s + (V + s) * ldh] = Delta[s];          /* upper-right Delta */
        H[(V + s) + s * ldh] = conj(Delta[s]);    /* lower-left Delta^* */
    }
    free(Tx); free(Ty); free(Tz);
}

/* Matrix-free Y = H X for ncols columns (each of length N, leading dims ldx, ldy). */
void orc_apply(int nx, int ny, int nz, double mu, const double *U, const cplx *Delta,
               int64_t ncols, const cplx *X, int64_t ldx, cplx *Y, int64_t ldy, int nthreads) {
    const int64_t V = (int64_t)nx * ny * nz;
    double *Tx = malloc(sizeof(double) * nx * nx);
    double *Ty = malloc(sizeof(double) * ny * ny);
    double *Tz = malloc(sizeof(double) * nz * nz);
    orc_kinetic_1d(nx, Tx, NULL);
    orc_kinetic_1d(ny, Ty, NULL);
    orc_kinetic_1d(nz, Tz, NULL);
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < ncols; ++c) {
        const cplx *u = X + c * ldx, *v = u + V;
        cplx *yu = Y + c * ldy, *yv = yu + V;
        for (int64_t s = 0; s < V; ++s) {
            int ix = (int)(s / ((int64_t)ny * nz)), iy = (int)((s / nz) % ny), iz = (int)(s % nz);
            cplx tu = 0.0, tv = 0.0;
            for (int jx = 0; jx < nx; ++jx) {
                int64_t t = ((int64_t)jx * ny + iy) * nz + iz;
                tu += Tx[ix + (size_t)jx * nx] * u[t];
                tv += Tx[ix + (size_t)jx * nx] * v[t];
            }
            for (int jy = 0; jy < ny; ++jy) {
                int64_t t = ((int64_t)ix * ny + jy) * nz + iz;
                tu += Ty[iy + (size_t)jy * ny] * u[t];
                tv += Ty[iy + (size_t)jy * ny] * v[t];
            }
            for (int jz = 0; jz < nz; ++jz) {
                int64_t t = ((int64_t)ix * ny + iy) * nz + jz;
                tu += Tz[iz + (size_t)jz * nz] * u[t];
                tv += Tz[iz + (size_t)jz * nz] * v[t];
            }
            double hd = U[s] - mu;
            yu[s] = tu + hd * u[s] + Delta[s] * v[s];
            yv[s] = conj(Delta[s]) * u[s] - (tv + hd * v[s]);
        }
    }
    free(Tx); free(Ty); free(Tz);
}

/* Householder reflector with real tau: given x (length m), returns beta and
 * overwrites x with v (v[0] = 1) so that (I - tau v v^H) x = beta e_1 with
 * beta = -exp(i arg x_0) ||x||.  tau = 1 + |x_0| / ||x||; tau = 0 when x = 0. */
static double reflector(int64_t m, cplx *x, cplx *beta) {
    double nrm2 = 0.0;
    for (int64_t i = 0; i < m; ++i) nrm2 += creal(x[i]) * creal(x[i]) + cimag(x[i]) * cimag(x[i]);
    double nrm = sqrt(nrm2);
    if (nrm == 0.0) { *beta = 0.0; for (int64_t i = 1; i < m; ++i) x[i] = 0.0; x[0] = 1.0; return 0.0; }
    double a = cabs(x[0]);
    cplx ph = (a == 0.0) ? 1.0 : x[0] / a;
    *beta = -ph * nrm;
    cplx pivot = x[0] - *beta;           /* = ph * (a + nrm), never cancels */
    for (int64_t i = 1; i < m; ++i) x[i] /= pivot;
    x[0] = 1.0;
    return 1.0 + a / nrm;
}

/* Householder tridiagonalisation of the Hermitian A (n x n, full storage, lda).
 * On exit: d (real diagonal), e (complex sub-diagonal, length n-1), the
 * reflector vectors v_k below the sub-diagonal of column k (v_k[0] = 1 is
 * implicit) and tau[k] (length n-1; tau[n-2] = 0).  A = Q T Q^H with
 * Q = H_0 H_1 ... H_{n-3}, H_k = I - tau_k v_k v_k^H acting on rows k+1..n-1. */
void orc_tridiag(int64_t n, cplx *A, int64_t lda, double *d, cplx *e, double *tau, int nthreads) {
    set_threads(nthreads);
    cplx *v = malloc(sizeof(cplx) * (size_t)n);
    cplx *p = malloc(sizeof(cplx) * (size_t)n);
    cplx *w = malloc(sizeof(cplx) * (size_t)n);
    for (int64_t k = 0; k + 2 < n; ++k) {
        int64_t m = n - k - 1;                 /* length of x = A[k+1:n, k] */
        cplx *x = A + (k + 1) + k * lda;
        for (int64_t i = 0; i < m; ++i) v[i] = x[i];
        cplx beta;
        double t = reflector(m, v, &beta);
        tau[k] = t;
        e[k] = beta;
        x[0] = beta;
        for (int64_t i = 1; i < m; ++i) x[i] = v[i];   /* store v below the sub-diagonal */
        /* keep the matrix Hermitian in full storage: row k mirrors column k */
        A[k + (k + 1) * lda] = conj(beta);
        for (int64_t i = 1; i < m; ++i) A[k + (k + 1 + i) * lda] = 0.0;
        if (t == 0.0) continue;
        cplx *B = A + (k + 1) + (k + 1) * lda;  /* trailing block, m x m */
        /* p = tau * B v */
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < m; ++i) p[i] = 0.0;
#pragma omp parallel
        {
#pragma omp for schedule(static)
            for (int64_t i = 0; i < m; ++i) {
                cplx acc = 0.0;
                for (int64_t j = 0; j < m; ++j) acc += conj(B[j + i * lda]) * v[j]; /* B[i][j] = conj(B[j][i]) */
                p[i] = t * acc;
            }
        }
        /* K = (tau/2) v^H p (real), w = p - K v */
        cplx vp = 0.0;
        for (int64_t i = 0; i < m; ++i) vp += conj(v[i]) * p[i];
        double K = 0.5 * t * creal(vp);
        for (int64_t i = 0; i < m; ++i) w[i] = p[i] - K * v[i];
        /* B <- B - v w^H - w v^H */
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < m; ++j) {
            cplx wj = conj(w[j]), vj = conj(v[j]);
            cplx *col = B + j * lda;
            for (int64_t i = 0; i < m; ++i) col[i] -= v[i] * wj + w[i] * vj;
        }
    }
    if (n >= 2) { e[n - 2] = A[(n - 1) + (n - 2) * lda]; tau[n - 2] = 0.0; }
    for (int64_t k = 0; k < n; ++k) d[k] = creal(A[k + k * lda]);
    free(v); free(p); free(w);
}

/* Diagonal unitary making the sub-diagonal real: D_0 = 1, D_{k+1} = D_k e_k/|e_k|.
 * Writes |e_k| into er and the phases into D (length n). */
void orc_phase(int64_t n, const cplx *e, double *er, cplx *D) {
    D[0] = 1.0;
    for (int64_t k = 0; k + 1 < n; ++k) {
        double a = cabs(e[k]);
        er[k] = a;
        D[k + 1] = (a == 0.0) ? D[k] : D[k] * (e[k] / a);
    }
}

/* Symmetric tridiagonal QR algorithm (Golub & Van Loan, Algorithms 8.3.2 and
 * 8.3.3): implicit QR steps with the Wilkinson shift taken from the trailing
 * 2x2 of the active block, each step a chase of one bulge by plane rotations
 * from the top of the block to its bottom; negligible off-diagonals split the
 * matrix.  (d, e): e[i] couples i and i+1 (length n-1).  On exit d holds the
 * eigenvalues (unsorted).  If Q != NULL (n x n, ldq, initialised by the
 * caller, normally to I) every rotation R is accumulated as Q <- Q R^T, so that
 * the columns of Q are the eigenvectors.  Returns 0, or -1 if a block needed
 * more than 30*n steps. */
int orc_tqr(int64_t n, double *d, const double *e_in, double *Q, int64_t ldq, int nthreads) {
    set_threads(nthreads);
    double *e = malloc(sizeof(double) * (size_t)(n > 1 ? n : 1));
    for (int64_t i = 0; i + 1 < n; ++i) e[i] = e_in[i];
    const double eps = 0x1p-53;
    int64_t steps = 0, max_steps = 30 * n + 30;
    int64_t h = n - 1;
    while (h > 0) {
        if (fabs(e[h - 1]) <= eps * (fabs(d[h - 1]) + fabs(d[h]))) { e[h - 1] = 0.0; --h; continue; }
        int64_t l = h - 1;
        while (l > 0 && fabs(e[l - 1]) > eps * (fabs(d[l - 1]) + fabs(d[l]))) --l;
        if (l > 0) e[l - 1] = 0.0;
        if (++steps > max_steps) { free(e); return -1; }
        /* Wilkinson shift: eigenvalue of the trailing 2x2 closer to d[h] */
        double delta = 0.5 * (d[h - 1] - d[h]);
        double eh = e[h - 1];
        double sg = (delta >= 0.0) ? 1.0 : -1.0;
        double shift = d[h] - eh * eh / (delta + sg * hypot(delta, eh));
        double x = d[l] - shift, z = e[l], bulge = 0.0;
        for (int64_t k = l; k < h; ++k) {
            if (k > l) { x = e[k - 1]; z = bulge; }
            double r = hypot(x, z);
            double c = (r == 0.0) ? 1.0 : x / r, s = (r == 0.0) ? 0.0 : z / r;
            if (k > l) e[k - 1] = r;
            /* T <- R T R^T on rows/columns k, k+1, R = [[c, s], [-s, c]] */
            double a = d[k], b = e[k], cc = d[k + 1];
            d[k] = c * c * a + 2.0 * c * s * b + s * s * cc;
            d[k + 1] = s * s * a - 2.0 * c * s * b + c * c * cc;
            e[k] = c * s * (cc - a) + (c * c - s * s) * b;
            if (k + 1 < h) { bulge = s * e[k + 1]; e[k + 1] = c * e[k + 1]; }
            if (Q) {
                double *qk = Q + k * ldq, *qk1 = Q + (k + 1) * ldq;
#pragma omp parallel for schedule(static) if (n > 2048)
                for (int64_t i = 0; i < n; ++i) {
                    double u = qk[i], v = qk1[i];
                    qk[i] = c * u + s * v;
                    qk1[i] = -s * u + c * v;
                }
            }
        }
    }
    free(e);
    return 0;
}

/* Back-transformation Z <- Q Z for the reflectors stored by orc_tridiag
 * (columns of A below the sub-diagonal), Q = H_0 ... H_{n-3}. */
void orc_backtransform(int64_t n, const cplx *A, int64_t lda, const double *tau,
                       int64_t ncols, cplx *Z, int64_t ldz, int nthreads) {
    set_threads(nthreads);
    for (int64_t k = n - 3; k >= 0; --k) {
        double t = tau[k];
        if (t == 0.0) continue;
        int64_t m = n - k - 1;
        const cplx *vs = A + (k + 1) + k * lda;   /* vs[0] is beta; v[0] = 1 implicit */
#pragma omp parallel for schedule(static)
        for (int64_t c = 0; c < ncols; ++c) {
            cplx *z = Z + (k + 1) + c * ldz;
            cplx acc = z[0];
            for (int64_t i = 1; i < m; ++i) acc += conj(vs[i]) * z[i];
            acc *= t;
            z[0] -= acc;
            for (int64_t i = 1; i < m; ++i) z[i] -= vs[i] * acc;
        }
    }
}

/* Full Hermitian eigensolver: eigenvalues ascending in w; if Z != NULL, the
 * eigenvectors in its columns (n x n, ldz).  A is destroyed.  Returns 0 or -1. */
int orc_heev(int64_t n, cplx *A, int64_t lda, double *w, cplx *Z, int64_t ldz, int nthreads) {
    set_threads(nthreads);
    double *d = malloc(sizeof(double) * (size_t)n);
    double *er = malloc(sizeof(double) * (size_t)(n > 1 ? n - 1 : 1));
    cplx *e = malloc(sizeof(cplx) * (size_t)(n > 1 ? n - 1 : 1));
    double *tau = malloc(sizeof(double) * (size_t)(n > 1 ? n - 1 : 1));
    cplx *D = malloc(sizeof(cplx) * (size_t)n);
    int status = 0;
    if (n == 1) {
        w[0] = creal(A[0]);
        if (Z) Z[0] = 1.0;
        goto done;
    }
    orc_tridiag(n, A, lda, d, e, tau, nthreads);
    orc_phase(n, e, er, D);
    double *Y = NULL;
    if (Z) {
        Y = malloc(sizeof(double) * (size_t)n * (size_t)n);
        for (int64_t j = 0; j < n; ++j)
            for (int64_t i = 0; i < n; ++i) Y[i + j * n] = (i == j) ? 1.0 : 0.0;
    }
    status = orc_tqr(n, d, er, Y, n, nthreads);
    /* sort ascending (selection sort on indices keeps it plain) */
    int64_t *idx = malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) idx[i] = i;
    for (int64_t i = 0; i < n; ++i) {
        int64_t best = i;
        for (int64_t j = i + 1; j < n; ++j) if (d[idx[j]] < d[idx[best]]) best = j;
        int64_t tmp = idx[i]; idx[i] = idx[best]; idx[best] = tmp;
    }
    for (int64_t i = 0; i < n; ++i) w[i] = d[idx[i]];
    if (Z) {
        /* Z = D Y (phase rows), columns permuted into ascending order */
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < n; ++j) {
            const double *y = Y + idx[j] * n;
            cplx *z = Z + j * ldz;
            for (int64_t i = 0; i < n; ++i) z[i] = D[i] * y[i];
        }
        orc_backtransform(n, A, lda, tau, n, Z, ldz, nthreads);
        free(Y);
    }
    free(idx);
done:
    free(d); free(er); free(e); free(tau); free(D);
    return status;
}

/* Sturm count of the real symmetric tridiagonal (d, e): number of eigenvalues
 * strictly below sigma (the LDL^T inertia recurrence). */
int64_t orc_sturm_count(int64_t n, const double *d, const double *e, double sigma) {
    int64_t cnt = 0;
    double q = d[0] - sigma;
    const double tiny = 1e-300;
    if (q < 0.0) cnt++;
    for (int64_t i = 1; i < n; ++i) {
        if (fabs(q) < tiny) q = -tiny;
        q = (d[i] - sigma) - e[i - 1] * e[i - 1] / q;
        if (q < 0.0) cnt++;
    }
    return cnt;
}
