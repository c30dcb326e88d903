// FP64 eigensolver for the Hermitian tridiagonal produced by stage 2
// (paper, section "Performance of the Matrix Diagonalization Algorithm":
// step ii of the solver, "diagonalizing this tridiagonal form").
//
//  1. prepare (one CTA): d_i = Re t_ii, e_i = |t_{i+1,i}|, the diagonal
//     unitary D (D_0 = 1, D_{i+1} = D_i t_{i+1,i}/|t_{i+1,i}|) that makes the
//     off-diagonal real (T_complex = D T_real D^H), and the split of T_real
//     into unreduced blocks where |e_i| <= eps (|d_i| + |d_{i+1}|);
//  2. bisection with Sturm counts, one thread per eigenvalue, inside its block;
//  3. inverse iteration by the twisted factorization of T - lambda I
//     (forward pivots D+_i, backward pivots D-_i, twist index
//     r = argmin |D+_r + D-_r - (d_r - lambda)|), one thread per cluster of
//     close eigenvalues; cluster members after the first are re-iterated
//     with modified Gram-Schmidt against the earlier members;
//  4. global ascending order (rank by counting) and assembly of
//     E = D Y(:, perm) in the working precision, column-major.
// Eigenvalue index j of the global list equals the row index of the block it
// belongs to: block [bs, be) owns eigenvalues bs .. be-1.
#include <stdlib.h>

#include "internal.h"

namespace bdg {

constexpr double kEps = 1.1102230246251565e-16;

template <typename R>
__global__ void __launch_bounds__(1024) tri_prepare_kernel(int64_t n, const cplx<R> *__restrict__ band, int ldband,
                                                            double *__restrict__ d, double *__restrict__ e,
                                                            double *__restrict__ e2, double2 *__restrict__ Dph,
                                                            int *__restrict__ bstart, int *__restrict__ bend,
                                                            double *__restrict__ tnorm_out) {
    __shared__ double2 s_pre[1024];
    __shared__ int s_i[1024];
    __shared__ double s_m[1024];
    const int T = blockDim.x, t = threadIdx.x;
    const int64_t cs = (n + T - 1) / T;
    const int64_t lo = min(n, (int64_t)t * cs), hi = min(n, lo + cs);
    // d, e, split, local phase product, local max norm
    double2 prod = make_double2(1.0, 0.0);
    double mx = 0.0;
    for (int64_t i = lo; i < hi; ++i) {
        cplx<R> dd = band[(int64_t)i * ldband];
        d[i] = (double)dd.x;
        mx = fmax(mx, fabs((double)dd.x));
        if (i + 1 < n) {
            cplx<R> ee = band[1 + (int64_t)i * ldband];
            double ex = ee.x, ey = ee.y, a = sqrt(ex * ex + ey * ey);
            double di = fabs((double)dd.x), dn = fabs((double)band[(int64_t)(i + 1) * ldband].x);
            mx = fmax(mx, a);
            if (a <= kEps * (di + dn)) a = 0.0;   // split
            e[i] = a;
            e2[i] = a * a;
            if (a > 0.0) {
                double ux = ex / sqrt(ex * ex + ey * ey), uy = ey / sqrt(ex * ex + ey * ey);
                double px = prod.x * ux - prod.y * uy, py = prod.x * uy + prod.y * ux;
                prod = make_double2(px, py);
            }
        }
    }
    s_pre[t] = prod;
    s_m[t] = mx;
    __syncthreads();
    // inclusive scan of the chunk products (Hillis-Steele), renormalised
    for (int off = 1; off < T; off <<= 1) {
        double2 a = s_pre[t];
        double2 bq = (t >= off) ? s_pre[t - off] : make_double2(1.0, 0.0);
        __syncthreads();
        double px = bq.x * a.x - bq.y * a.y, py = bq.x * a.y + bq.y * a.x;
        double nr = rsqrt(px * px + py * py);
        s_pre[t] = make_double2(px * nr, py * nr);
        __syncthreads();
    }
    for (int off = T / 2; off > 0; off >>= 1) {
        if (t < off) s_m[t] = fmax(s_m[t], s_m[t + off]);
        __syncthreads();
    }
    if (t == 0) *tnorm_out = s_m[0];
    // exclusive prefix for this chunk
    double2 cur = (t == 0) ? make_double2(1.0, 0.0) : s_pre[t - 1];
    for (int64_t i = lo; i < hi; ++i) {
        Dph[i] = cur;
        if (i + 1 < n && e[i] > 0.0) {
            cplx<R> ee = band[1 + (int64_t)i * ldband];
            double ex = ee.x, ey = ee.y, a = sqrt(ex * ex + ey * ey);
            double ux = ex / a, uy = ey / a;
            double px = cur.x * ux - cur.y * uy, py = cur.x * uy + cur.y * ux;
            double nr = rsqrt(px * px + py * py);
            cur = make_double2(px * nr, py * nr);
        }
    }
    __syncthreads();
    // block starts: prefix max of "start index" (i starts a block if i == 0 or e[i-1] == 0)
    int last = -1;
    for (int64_t i = lo; i < hi; ++i)
        if (i == 0 || e[i - 1] == 0.0) last = (int)i;
    s_i[t] = last;
    __syncthreads();
    for (int off = 1; off < T; off <<= 1) {
        int a = s_i[t];
        int bq = (t >= off) ? s_i[t - off] : -1;
        __syncthreads();
        s_i[t] = max(a, bq);
        __syncthreads();
    }
    int run = (t == 0) ? 0 : s_i[t - 1];
    for (int64_t i = lo; i < hi; ++i) {
        if (i == 0 || e[i - 1] == 0.0) run = (int)i;
        bstart[i] = run;
    }
    __syncthreads();
    // block ends: suffix min of "end index" (i ends a block if i == n-1 or e[i] == 0)
    int first = (int)n;
    for (int64_t i = hi - 1; i >= lo; --i)
        if (i == n - 1 || e[i] == 0.0) first = (int)(i + 1);
    s_i[t] = first;
    __syncthreads();
    for (int off = 1; off < T; off <<= 1) {
        int a = s_i[t];
        int bq = (t + off < T) ? s_i[t + off] : (int)n;
        __syncthreads();
        s_i[t] = min(a, bq);
        __syncthreads();
    }
    int runE = (t == T - 1) ? (int)n : s_i[t + 1];
    for (int64_t i = hi - 1; i >= lo; --i) {
        if (i == n - 1 || e[i] == 0.0) runE = (int)(i + 1);
        bend[i] = runE;
    }
}

// Number of eigenvalues of block [bs, be) below sigma: the negative pivots q_i of
// the LDL^T factorisation of T - sigma I.  The sequence is carried in product form,
// p_i = (d_i - sigma) p_{i-1} - e_{i-1}^2 p_{i-2}, as the pair (a, b) = (p_{i-1}, p_i)
// up to a common power of two: q_i = b / a, so a negative pivot is a sign change and
// no division is needed (an FP64 divide costs many FP64 instructions).  As in the
// quotient form, a pivot below pivmin in magnitude is replaced by -pivmin; the pair
// is rescaled exactly when its larger member leaves [2^-200, 2^200].
__device__ __forceinline__ int sturm_count(const double *__restrict__ d, const double *__restrict__ e2, int bs,
                                           int be, double sigma, double pivmin) {
    int cnt = 0;
    double a = 1.0, b = d[bs] - sigma;
    if (b < 0.0) ++cnt;
    if (fabs(b) < pivmin) b = -pivmin;
    // B300's FP64 pipe is the bound here, so the tests that need no rounding run on the integer
    // pipes: nb != 0 from its bits; |nb| < pivmin |a| as an unsigned compare of the bit patterns
    // (their order is the numeric order for non-negative doubles, NaN included: never smaller);
    // and the guarded pivot reuses the guard's product (-pivmin a = -copysign(pivmin |a|, a), bit
    // for bit)
    for (int i = bs + 1; i < be; ++i) {
        const double nb = fma(d[i] - sigma, b, -e2[i - 1] * a);
        const int nh = __double2hiint(nb);
        const unsigned long long nabs = (unsigned long long)__double_as_longlong(nb) & 0x7fffffffffffffffull;
        cnt += (nabs != 0ull && ((nh ^ __double2hiint(b)) < 0)) ? 1 : 0;
        a = b;
        const double pm = pivmin * fabs(a);
        b = (nabs < (unsigned long long)__double_as_longlong(pm)) ? -copysign(pm, a) : nb;   // signed zero keeps the sign if this underflows
        const int ea = (__double2hiint(a) >> 20) & 0x7ff, eb = (__double2hiint(b) >> 20) & 0x7ff;
        const int em = max(ea, eb);
        if ((em > 1023 + 200 && em < 2047) || em < 1023 - 200) {
            const double sc = __hiloint2double((2046 - em) << 20, 0);   // 2^(1023 - em), exact
            a *= sc;
            b *= sc;
        }
    }
    return cnt;
}

// With pos_only, eigenvalues below zero are not computed (set to -inf): the
// particle-hole mode needs only the upper half of the spectrum.
__global__ void bisect_kernel(int64_t n, const double *__restrict__ d, const double *__restrict__ e,
                              const double *__restrict__ e2, const int *__restrict__ bstart,
                              const int *__restrict__ bend, double *__restrict__ w, int pos_only) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int bs = bstart[j], be = bend[j];
    const int l = (int)(j - bs);
    if (be - bs == 1) { w[j] = (pos_only && d[bs] < 0.0) ? -INFINITY : d[bs]; return; }
    double lo = 1e300, hi = -1e300, emax2 = 0.0;
    for (int i = bs; i < be; ++i) {
        double r = (i > bs ? e[i - 1] : 0.0) + (i + 1 < be ? e[i] : 0.0);
        lo = fmin(lo, d[i] - r);
        hi = fmax(hi, d[i] + r);
        if (i + 1 < be) emax2 = fmax(emax2, e2[i]);
    }
    const double tn = fmax(fabs(lo), fabs(hi));
    const double pivmin = fmax(2.2250738585072014e-308 * fmax(emax2, 1.0), 1e-300);
    if (pos_only && l < sturm_count(d, e2, bs, be, 0.0, pivmin)) { w[j] = -INFINITY; return; }
    lo -= 2.0 * kEps * tn + 2.0 * pivmin;
    hi += 2.0 * kEps * tn + 2.0 * pivmin;
    // invariant: count(lo) <= l < count(hi)
    for (int it = 0; it < 120; ++it) {
        double mid = 0.5 * (lo + hi);
        if (hi - lo <= 2.0 * kEps * fmax(fabs(lo), fabs(hi)) + 4.0 * pivmin || mid <= lo || mid >= hi) break;
        int c = sturm_count(d, e2, bs, be, mid, pivmin);
        if (c > l) hi = mid;
        else lo = mid;
    }
    w[j] = 0.5 * (lo + hi);
}

// Number of eigenvalues below -delta and below +delta (two threads).
__global__ void pm_count_kernel(int64_t n, const double *__restrict__ d, const double *__restrict__ e2, double delta,
                                int *__restrict__ out) {
    const int t = threadIdx.x;
    if (t > 1) return;
    double emax2 = 0.0;
    for (int64_t i = 0; i + 1 < n; ++i) emax2 = fmax(emax2, e2[i]);
    const double pivmin = fmax(2.2250738585072014e-308 * fmax(emax2, 1.0), 1e-300);
    out[t] = sturm_count(d, e2, 0, (int)n, t == 0 ? -delta : delta, pivmin);
}

// Twisted factorisation of T - lambda I on block [bs, be): stores D+ and D-
// (column `col` of the row-major scratch arrays, leading dimension ldw) and
// returns the twist index r and gamma_r.
__device__ void twisted_factor(const double *__restrict__ d, const double *__restrict__ e,
                               const double *__restrict__ e2, int bs, int be, double lam, double *Dp,
                               double *Dm, int64_t ldw, int64_t col, double pivmin, int *r_out,
                               double *gam_out) {
    double q = d[bs] - lam;
    Dp[(int64_t)bs * ldw + col] = q;
    for (int i = bs + 1; i < be; ++i) {
        if (fabs(q) < pivmin) q = (q < 0.0 ? -pivmin : pivmin);
        q = (d[i] - lam) - e2[i - 1] / q;
        Dp[(int64_t)i * ldw + col] = q;
    }
    double p = d[be - 1] - lam;
    Dm[(int64_t)(be - 1) * ldw + col] = p;
    double best = fabs(q);  // gamma at be-1 = D+_{be-1}
    int r = be - 1;
    double gbest = q;
    for (int i = be - 2; i >= bs; --i) {
        if (fabs(p) < pivmin) p = (p < 0.0 ? -pivmin : pivmin);
        double pm = (d[i] - lam) - e2[i] / p;
        Dm[(int64_t)i * ldw + col] = pm;
        double dp = Dp[(int64_t)i * ldw + col];
        double gam = dp + pm - (d[i] - lam);
        if (fabs(gam) < best) { best = fabs(gam); r = i; gbest = gam; }
        p = pm;
    }
    *r_out = r;
    *gam_out = gbest;
}

// Solve (T - lambda I) x = rhs with the twisted factors; x overwrites rhs
// (row-major column `xcol` of X, leading dimension ldx).
__device__ void twisted_solve(const double *__restrict__ e, int bs, int be, const double *Dp,
                              const double *Dm, int64_t ldw, int64_t col, int r, double gam, double *X,
                              int64_t ldx, int64_t xcol, double pivmin) {
    auto XA = [&](int i) -> double & { return X[(int64_t)i * ldx + xcol]; };
    auto P = [&](int i) { double v = Dp[(int64_t)i * ldw + col]; return fabs(v) < pivmin ? (v < 0 ? -pivmin : pivmin) : v; };
    auto M = [&](int i) { double v = Dm[(int64_t)i * ldw + col]; return fabs(v) < pivmin ? (v < 0 ? -pivmin : pivmin) : v; };
    // forward elimination above the twist, backward below it
    for (int i = bs + 1; i < r; ++i) XA(i) -= (e[i - 1] / P(i - 1)) * XA(i - 1);
    for (int i = be - 2; i > r; --i) XA(i) -= (e[i] / M(i + 1)) * XA(i + 1);
    double br = XA(r);
    if (r > bs) br -= (e[r - 1] / P(r - 1)) * XA(r - 1);
    if (r < be - 1) br -= (e[r] / M(r + 1)) * XA(r + 1);
    double g = gam;
    if (fabs(g) < pivmin) g = (g < 0 ? -pivmin : pivmin);
    XA(r) = br / g;
    for (int i = r - 1; i >= bs; --i) XA(i) = (XA(i) - e[i] * XA(i + 1)) / P(i);
    for (int i = r + 1; i < be; ++i) XA(i) = (XA(i) - e[i - 1] * XA(i - 1)) / M(i);
}

// Counter-based uniform variate in [-1, 1): the SplitMix64 finaliser applied to
// (a, b) (Steele, Lea & Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014).
__device__ __forceinline__ double hash_uniform(uint64_t a, uint64_t b) {
    uint64_t z = a * 0x9E3779B97F4A7C15ull + b + 0x632BE59BD9B4E019ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * 0x1.0p-52 - 1.0;
}

__device__ void normalize_col(double *X, int64_t ldx, int64_t xcol, int bs, int be) {
    double s = 0.0, mx = 0.0;
    for (int i = bs; i < be; ++i) mx = fmax(mx, fabs(X[(int64_t)i * ldx + xcol]));
    if (mx == 0.0) { X[(int64_t)bs * ldx + xcol] = 1.0; return; }
    double inv = 1.0 / mx;
    for (int i = bs; i < be; ++i) { double v = X[(int64_t)i * ldx + xcol] * inv; s += v * v; }
    double sc = inv / sqrt(s);
    for (int i = bs; i < be; ++i) X[(int64_t)i * ldx + xcol] *= sc;
}

// Gaussian elimination with partial (row) pivoting of the tridiagonal
// T - lambda I on block [bs, be): U has diagonal u0, first and second
// super-diagonals u1, u2 (u2 != 0 only after an interchange), L holds the
// multipliers lm; the interchange at the last step is recorded in u2[be-1].
// Four scratch columns, all row-major with leading dimension ldw.
struct LuCols {
    double *u0, *u1, *u2, *lm;
    int64_t ldw, col0, col1, col2, col3;
};

__device__ __forceinline__ void lu_factor(const double *__restrict__ d, const double *__restrict__ e, int bs, int be, double lam,
                          const LuCols &L, double tiny) {
    auto U0 = [&](int i) -> double & { return L.u0[(int64_t)i * L.ldw + L.col0]; };
    auto U1 = [&](int i) -> double & { return L.u1[(int64_t)i * L.ldw + L.col1]; };
    auto U2 = [&](int i) -> double & { return L.u2[(int64_t)i * L.ldw + L.col2]; };
    auto LM = [&](int i) -> double & { return L.lm[(int64_t)i * L.ldw + L.col3]; };
    double a = d[bs] - lam;                      // current pivot-row diagonal
    double bsup = (bs + 1 < be) ? e[bs] : 0.0;   // current pivot-row super-diagonal
    for (int i = bs; i < be - 1; ++i) {
        const double c = e[i];                   // sub-diagonal below the pivot
        const double anext = d[i + 1] - lam;
        const double bnext = (i + 2 < be) ? e[i + 1] : 0.0;
        if (fabs(a) >= fabs(c)) {
            double aa = (a == 0.0) ? tiny : a;
            double l = c / aa;
            U0(i) = aa; U1(i) = bsup; U2(i) = 0.0; LM(i) = l;
            a = anext - l * bsup;
            bsup = bnext;
            if (i == be - 2) U2(be - 1) = 0.0;
        } else {
            double l = a / c;
            U0(i) = c; U1(i) = anext; U2(i) = bnext; LM(i) = l;
            a = bsup - l * anext;
            bsup = -l * bnext;
            if (i == be - 2) U2(be - 1) = 1.0;   // interchange at the last step
        }
    }
    U0(be - 1) = (a == 0.0) ? tiny : a;
    if (be - bs == 1) U2(be - 1) = 0.0;
}

__device__ __forceinline__ void lu_solve(int bs, int be, const LuCols &L, double tiny, double *X, int64_t ldx, int64_t xcol) {
    auto U0 = [&](int i) { double v = L.u0[(int64_t)i * L.ldw + L.col0]; return fabs(v) < tiny ? (v < 0 ? -tiny : tiny) : v; };
    auto U1 = [&](int i) { return L.u1[(int64_t)i * L.ldw + L.col1]; };
    auto U2 = [&](int i) { return L.u2[(int64_t)i * L.ldw + L.col2]; };
    auto LM = [&](int i) { return L.lm[(int64_t)i * L.ldw + L.col3]; };
    auto XA = [&](int i) -> double & { return X[(int64_t)i * ldx + xcol]; };
    // apply P and L^-1
    for (int i = bs; i < be - 1; ++i) {
        const bool swapped = (i < be - 2) ? (U2(i) != 0.0) : (U2(be - 1) != 0.0);
        double xi = XA(i), xn = XA(i + 1);
        if (swapped) { double t = xi; xi = xn; xn = t; }
        XA(i) = xi;
        XA(i + 1) = xn - LM(i) * xi;
    }
    // U x = y
    for (int i = be - 1; i >= bs; --i) {
        double v = XA(i);
        if (i + 1 < be) v -= U1(i) * XA(i + 1);
        if (i + 2 < be) v -= U2(i) * XA(i + 2);
        XA(i) = v / U0(i);
    }
}

// Clusters of at least this many members go to invit_cluster_kernel (one CTA
// each); smaller ones stay with the thread that found them.
constexpr int kCtaCluster = 8;

// One thread per cluster of eigenvalues whose consecutive gaps are <= ctol.
// Singletons: one twisted-factorisation solve from e_r.  Clusters: every
// member by inverse iteration with the pivoted LU (three solves from a
// pseudo-random start), each followed by Gram-Schmidt against the earlier
// members; the LU uses the scratch columns of the first two members.
// Clusters of kCtaCluster or more members are only recorded in clist
// (count in *ccount) for invit_cluster_kernel.
__global__ void invit_kernel(int64_t n, const double *__restrict__ d, const double *__restrict__ e,
                             const double *__restrict__ e2, const int *__restrict__ bstart,
                             const int *__restrict__ bend, const double *__restrict__ w, double *Y, double *Dp,
                             double *Dm, double ctol, int2 *clist, int *ccount) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    if (w[j] == -INFINITY) return;                    // not computed (particle-hole mode)
    const int bs = bstart[j], be = bend[j];
    if (j > bs && w[j] - w[j - 1] <= ctol) return;   // not a cluster start
    int64_t jend = j + 1;
    while (jend < be && w[jend] - w[jend - 1] <= ctol) ++jend;
    if (jend - j >= kCtaCluster) {
        clist[atomicAdd(ccount, 1)] = make_int2((int)j, (int)jend);
        return;
    }
    if (be - bs == 1) { Y[(int64_t)bs * n + j] = 1.0; return; }
    double emax2 = 0.0, tn = 0.0;
    for (int i = bs; i < be; ++i) {
        tn = fmax(tn, fabs(d[i]) + (i > bs ? e[i - 1] : 0.0) + (i + 1 < be ? e[i] : 0.0));
        if (i + 1 < be) emax2 = fmax(emax2, e2[i]);
    }
    const double pivmin = fmax(2.2250738585072014e-308 * fmax(emax2, 1.0), 1e-300);
    if (jend == j + 1) {
        const double lam = w[j];
        int r;
        double gam;
        twisted_factor(d, e, e2, bs, be, lam, Dp, Dm, n, j, pivmin, &r, &gam);
        for (int i = bs; i < be; ++i) Y[(int64_t)i * n + j] = (i == r) ? 1.0 : 0.0;
        twisted_solve(e, bs, be, Dp, Dm, n, j, r, gam, Y, n, j, pivmin);
        normalize_col(Y, n, j, bs, be);
        return;
    }
    LuCols L;
    L.u0 = Dp; L.u1 = Dm; L.u2 = Dp; L.lm = Dm; L.ldw = n;
    L.col0 = j; L.col1 = j; L.col2 = j + 1; L.col3 = j + 1;
    const double tiny = kEps * fmax(tn, 1e-300);
    const double pert = 10.0 * kEps * fmax(tn, 1e-300);
    double lam_prev = -1e300;
    for (int64_t m = j; m < jend; ++m) {
        double lam = w[m];
        if (lam - lam_prev < pert) lam = lam_prev + pert;   // separate equal shifts slightly
        lam_prev = lam;
        lu_factor(d, e, bs, be, lam, L, tiny);
        for (int i = bs; i < be; ++i) Y[(int64_t)i * n + m] = hash_uniform((uint64_t)m, (uint64_t)i);
        for (int it = 0; it < 3; ++it) {
            lu_solve(bs, be, L, tiny, Y, n, m);
            normalize_col(Y, n, m, bs, be);
            for (int rep = 0; rep < 2; ++rep) {
                for (int64_t p = j; p < m; ++p) {
                    double dot = 0.0;
                    for (int i = bs; i < be; ++i) dot += Y[(int64_t)i * n + p] * Y[(int64_t)i * n + m];
                    for (int i = bs; i < be; ++i) Y[(int64_t)i * n + m] -= dot * Y[(int64_t)i * n + p];
                }
                normalize_col(Y, n, m, bs, be);
            }
        }
    }
}

__device__ double block_max(double v, double *scratch) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < nw; ++i) t = fmax(t, scratch[i]);
    return t;
}

// normalize_col with the block's threads over the rows
__device__ void block_normalize(double *X, int64_t ldx, int64_t xcol, int bs, int be, double *scratch) {
    double mx = 0.0;
    for (int i = bs + threadIdx.x; i < be; i += blockDim.x) mx = fmax(mx, fabs(X[(int64_t)i * ldx + xcol]));
    mx = block_max(mx, scratch);
    if (mx == 0.0) {
        if (threadIdx.x == 0) X[(int64_t)bs * ldx + xcol] = 1.0;
        __syncthreads();
        return;
    }
    const double inv = 1.0 / mx;
    double s = 0.0;
    for (int i = bs + threadIdx.x; i < be; i += blockDim.x) {
        const double v = X[(int64_t)i * ldx + xcol] * inv;
        s += v * v;
    }
    s = block_sum(s, scratch);
    const double sc = inv / sqrt(s);
    for (int i = bs + threadIdx.x; i < be; i += blockDim.x) X[(int64_t)i * ldx + xcol] *= sc;
    __syncthreads();
}

// The large clusters recorded by invit_kernel, one CTA each (CTAs stride over
// the list).  Same iteration as the thread version -- pivoted LU, three solves
// from the same pseudo-random start, each followed by two Gram-Schmidt passes
// against the earlier members -- with the recurrences of the LU on one thread
// and the normalisations and Gram-Schmidt passes on all of them.  A pass takes
// the earlier members in chunks of kDotChunk: all dot products of a chunk
// first, then one update (classical Gram-Schmidt within a chunk, repeated
// twice, which keeps the columns orthogonal to working precision).
constexpr int kDotChunk = 256;
__global__ void __launch_bounds__(256, 1) invit_cluster_kernel(int64_t n, const double *__restrict__ d,
                                                            const double *__restrict__ e,
                                                            const double *__restrict__ e2,
                                                            const int *__restrict__ bstart,
                                                            const int *__restrict__ bend,
                                                            const double *__restrict__ w, double *Y, double *Dp,
                                                            double *Dm, const int2 *__restrict__ clist,
                                                            const int *__restrict__ ccount) {
    __shared__ double s_red[32];
    __shared__ double s_dot[kDotChunk];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int ncl = *ccount;
    for (int c = blockIdx.x; c < ncl; c += gridDim.x) {
        const int2 cl = clist[c];
        const int64_t j = cl.x, jend = cl.y;
        const int bs = bstart[j], be = bend[j];
        double tl = 0.0;
        for (int i = bs + threadIdx.x; i < be; i += blockDim.x)
            tl = fmax(tl, fabs(d[i]) + (i > bs ? e[i - 1] : 0.0) + (i + 1 < be ? e[i] : 0.0));
        const double tn = block_max(tl, s_red);
        LuCols L;
        L.u0 = Dp; L.u1 = Dm; L.u2 = Dp; L.lm = Dm; L.ldw = n;
        L.col0 = j; L.col1 = j; L.col2 = j + 1; L.col3 = j + 1;
        const double tiny = kEps * fmax(tn, 1e-300);
        const double pert = 10.0 * kEps * fmax(tn, 1e-300);
        double lam_prev = -1e300;
        for (int64_t m = j; m < jend; ++m) {
            double lam = w[m];
            if (lam - lam_prev < pert) lam = lam_prev + pert;   // separate equal shifts slightly
            lam_prev = lam;
            if (threadIdx.x == 0) lu_factor(d, e, bs, be, lam, L, tiny);
            for (int i = bs + threadIdx.x; i < be; i += blockDim.x)
                Y[(int64_t)i * n + m] = hash_uniform((uint64_t)m, (uint64_t)i);
            __syncthreads();
            for (int it = 0; it < 3; ++it) {
                if (threadIdx.x == 0) lu_solve(bs, be, L, tiny, Y, n, m);
                __syncthreads();
                block_normalize(Y, n, m, bs, be, s_red);
                for (int rep = 0; rep < 2; ++rep) {
                    for (int64_t p0 = j; p0 < m; p0 += kDotChunk) {
                        const int np = (int)min((int64_t)kDotChunk, m - p0);
                        for (int q = wid; q < np; q += nw) {
                            double sdot = 0.0;
                            for (int i = bs + lane; i < be; i += 32)
                                sdot += Y[(int64_t)i * n + p0 + q] * Y[(int64_t)i * n + m];
                            sdot = warp_sum(sdot);
                            if (lane == 0) s_dot[q] = sdot;
                        }
                        __syncthreads();
                        for (int i = bs + threadIdx.x; i < be; i += blockDim.x) {
                            double y = Y[(int64_t)i * n + m];
                            for (int q = 0; q < np; ++q) y -= s_dot[q] * Y[(int64_t)i * n + p0 + q];
                            Y[(int64_t)i * n + m] = y;
                        }
                        __syncthreads();
                    }
                    block_normalize(Y, n, m, bs, be, s_red);
                }
            }
        }
    }
}

__global__ void rank_kernel(int64_t n, const double *__restrict__ w, double *__restrict__ ws,
                            int *__restrict__ perm) {
    __shared__ double tile[1024];
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

// E[r + c*lde] = D_r * Y[r*n + perm[coff + c]], c < ncols  (working
// precision, column-major)
template <typename R>
__global__ void assemble_kernel(int64_t n, int64_t coff, int64_t ncols, const double *__restrict__ Y,
                                const int *__restrict__ perm, const double2 *__restrict__ Dph, cplx<R> *__restrict__ E,
                                int64_t lde) {
    __shared__ double tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int k = 0; k < 32; k += 8) {
        int64_t r = r0 + ty + k, c = c0 + tx;
        tile[ty + k][tx] = (r < n && c < ncols) ? Y[r * n + perm[coff + c]] : 0.0;
    }
    __syncthreads();
    for (int k = 0; k < 32; k += 8) {
        int64_t r = r0 + tx, c = c0 + ty + k;
        if (r < n && c < ncols) {
            double y = tile[tx][ty + k];
            double2 p = Dph[r];
            E[r + c * lde] = mk<R>((R)(p.x * y), (R)(p.y * y));
        }
    }
}

// With want_ph (a particle-hole symmetric spectrum), the upper half only:
// if no eigenvalue lies within the cluster tolerance of zero and exactly n/2
// lie below it, eigenvalues w_sorted[n/2 ..] and their vectors
// are produced into E[:, n/2 ..] (*used_ph = 1) and w_sorted[0 .. n/2) is
// left at -inf;
// otherwise the full solve runs (*used_ph = 0).
template <typename R>
int tridiag_solve(bdg_ctx *ctx, cudaStream_t st, int64_t n, const cplx<R> *band, int ldband, const TriWork &tw,
                  double *w_sorted, cplx<R> *E, int64_t lde, double ctol_rel, bool want_ph, int *used_ph) {
    tri_prepare_kernel<R><<<1, 1024, 0, st>>>(n, band, ldband, tw.d, tw.e, tw.e2, tw.Dph, tw.bstart, tw.bend,
                                              tw.tnorm);
    BDG_LAUNCH_CHECK(ctx);
    // cluster tolerance relative to the largest |d|,|e| (read back once; tiny copy)
    double tn = 0.0;
    BDG_CUDA_TRY(ctx, cudaMemcpyAsync(&tn, tw.tnorm, sizeof(double), cudaMemcpyDeviceToHost, st));
    BDG_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    const char *cr = getenv("BDG_CLUSTER_REL");
    if (cr) ctol_rel = atof(cr);
    const double ctol = ctol_rel * (tn > 0 ? 3.0 * tn : 1.0);
    int ph = 0;
    if (want_ph && (n % 2) == 0 && n >= 4) {
        pm_count_kernel<<<1, 32, 0, st>>>(n, tw.d, tw.e2, ctol, tw.pmcount);
        BDG_LAUNCH_CHECK(ctx);
        int cnt[2] = {0, 0};
        BDG_CUDA_TRY(ctx, cudaMemcpyAsync(cnt, tw.pmcount, sizeof(cnt), cudaMemcpyDeviceToHost, st));
        BDG_CUDA_TRY(ctx, cudaStreamSynchronize(st));
        ph = (cnt[0] == n / 2 && cnt[1] == n / 2) ? 1 : 0;
    }
    *used_ph = ph;
    bisect_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(n, tw.d, tw.e, tw.e2, tw.bstart, tw.bend,
                                                              tw.w_unsorted, ph);
    BDG_LAUNCH_CHECK(ctx);
    BDG_CUDA_TRY(ctx, cudaMemsetAsync(tw.Y, 0, (size_t)n * n * sizeof(double), st));
    stage_mark(ctx, st, "tri_bisection");
    BDG_CUDA_TRY(ctx, cudaMemsetAsync(tw.pmcount + 2, 0, sizeof(int), st));
    invit_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(n, tw.d, tw.e, tw.e2, tw.bstart, tw.bend,
                                                             tw.w_unsorted, tw.Y, tw.Dp, tw.Dm, ctol, tw.clist,
                                                             tw.pmcount + 2);
    BDG_LAUNCH_CHECK(ctx);
    // the large clusters: a fixed grid (at most one CTA per 64 rows), the count stays on the device
    const int ncta = (int)std::max<int64_t>(1, std::min<int64_t>(2 * ctx->num_sms, n / 64));
    invit_cluster_kernel<<<(unsigned)ncta, 256, 0, st>>>(
        n, tw.d, tw.e, tw.e2, tw.bstart, tw.bend, tw.w_unsorted, tw.Y, tw.Dp, tw.Dm, tw.clist, tw.pmcount + 2);
    BDG_LAUNCH_CHECK(ctx);
    stage_mark(ctx, st, "tri_invit");
    rank_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, tw.w_unsorted, w_sorted, tw.perm);
    BDG_LAUNCH_CHECK(ctx);
    const int64_t coff = ph ? n / 2 : 0, ncols = n - coff;
    dim3 grid((unsigned)((ncols + 31) / 32), (unsigned)((n + 31) / 32));
    assemble_kernel<R><<<grid, dim3(32, 8), 0, st>>>(n, coff, ncols, tw.Y, tw.perm, tw.Dph, E + coff * lde, lde);
    BDG_LAUNCH_CHECK(ctx);
    return BDG_OK;
}

template int tridiag_solve<float>(bdg_ctx *, cudaStream_t, int64_t, const float2 *, int, const TriWork &,
                                  double *, float2 *, int64_t, double, bool, int *);
template int tridiag_solve<double>(bdg_ctx *, cudaStream_t, int64_t, const double2 *, int, const TriWork &,
                                   double *, double2 *, int64_t, double, bool, int *);

}  // namespace bdg
