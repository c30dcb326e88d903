// Stage 2 of the two-stage reduction: Hermitian band (width b) -> Hermitian
// tridiagonal by bulge chasing, and the matching back-transformation
// (paper, section "Performance of the Matrix Diagonalization Algorithm": the
// 2-stage solver transforms the banded matrix into tridiagonal form and the
// back-transformation also takes two stages).
//
// Sweep s (s = 0 .. n-3) removes column s below its first sub-diagonal entry
// with one reflector of length <= b, then chases the bulge that reflector
// creates down the band, one b x b block per step.  Step k of sweep s:
//   column c = s (k = 0) or s+1+(k-1)b (k >= 1), rows r0 = s+1+kb .. r0+L-1,
//   L = min(b, n-r0);
//   generate H = I - tau v v^H from column c of that row block (H x = beta e1);
//   apply H from the left to the rest of that block (k >= 1),
//   H D H to the diagonal block D = A[r0:r0+L, r0:r0+L],
//   and H from the right to the block below D (which fills a new bulge).
// Step k of sweep s touches rows s+1+kb .. s+(k+2)b and columns
// s+1+(k-1)b .. s+(k+1)b.  Of sweep s-1 that overlaps all of step k+1 and, of
// step k+2, a single entry (row s+(k+2)b, column s+(k+1)b) of the row block
// that step's left application stores; the diagonal block of step k+2 starts
// at column s+(k+2)b and the block below it at row s+(k+3)b, both out of
// reach.  So sweep s may run step k once sweep s-1 has finished step k+1 and
// stored the row block of step k+2.  Progress is published per half step
// (2j+1: row block of step j stored, 2j+2: step j complete), so a sweep trails
// the previous one by two and a half steps rather than three.  One CTA runs
// one sweep at a time; sweeps are handed out in order by an atomic ticket, and
// the inter-sweep dependency is a bounded spin on a per-sweep progress counter.
// The band lives in a (2b+1) x n lower band array (row d of column j =
// A[j+d][j]); all band accesses bypass L1 so that concurrent sweeps see each
// other's writes.
#include <stdlib.h>

#include <type_traits>

#include "internal.h"

namespace bdg {

__host__ __device__ inline int64_t sweep_steps(int64_t n, int b, int64_t s) {
    // number of steps k >= 0 with min(b, n - (s+1+k b)) >= 2
    if (s > n - 3) return 0;
    return (n - s - 3) / b + 1;
}

struct Stage2Args {
    int64_t n;
    int b;
    int ldband;
    int g;                      // sweeps per stored group
    void *band;                 // cplx<R>*
    void *refl;                 // cplx<R>*: reflector vectors (b entries each)
    void *tau;                  // R*
    const int64_t *grp_off;     // per group: offset (in vectors) of its first (k=0, i=0) slot
    unsigned int *ticket;
    int *progress;              // per sweep: half steps done
    int *err;
    long long wait;             // cap of the inter-sweep wait, SM clock cycles
    int half;                   // publish the mid-step point (wide bands), else whole steps only
};

template <typename R>
__device__ __forceinline__ cplx<R> bget(const cplx<R> *band, int ldband, int64_t r, int64_t c) {
    return ldcg(band + (r - c) + c * (int64_t)ldband);
}
template <typename R>
__device__ __forceinline__ void bset(cplx<R> *band, int ldband, int64_t r, int64_t c, cplx<R> v) {
    stcg(band + (r - c) + c * (int64_t)ldband, v);
}

template <typename R>
__global__ void __launch_bounds__(256) bulge_chase_kernel(Stage2Args a) {
    using Cx = cplx<R>;
    const int64_t n = a.n;
    const int b = a.b, ldb = a.ldband, g = a.g;
    Cx *band = reinterpret_cast<Cx *>(a.band);
    Cx *refl = reinterpret_cast<Cx *>(a.refl);
    R *taus = reinterpret_cast<R *>(a.tau);
    extern __shared__ unsigned char smem_raw[];
    // the three tiles are column-major with leading dimension b + 1 (an odd number of
    // complex entries): the mirrored stores D[j][i] and the 4-threads-per-row/column
    // products then spread over the banks instead of hitting one
    const int ls = b + 1;
    Cx *Rc = reinterpret_cast<Cx *>(smem_raw);   // current row block L x b   (ld ls)
    Cx *D = Rc + b * ls;                          // diagonal block L x L     (ld ls)
    Cx *Rn = D + b * ls;                          // next block below  L2 x L (ld ls)
    __shared__ Cx s_v[64];
    __shared__ Cx s_p[64];
    __shared__ Cx s_w[64];
    __shared__ R s_red[32];
    __shared__ R s_tau;
    __shared__ Cx s_beta;
    __shared__ int64_t s_sweep;
    __shared__ int s_abort;
    const int tid = threadIdx.x;
    const int64_t nsweeps = n >= 3 ? n - 2 : 0;

    for (;;) {
        if (tid == 0) {
            s_sweep = (int64_t)atomicAdd(a.ticket, 1u);
            s_abort = *((volatile int *)a.err);
        }
        __syncthreads();
        const int64_t s = s_sweep;
        if (s >= nsweeps || s_abort) return;
        const int64_t nst = sweep_steps(n, b, s);
        const int64_t prev_nst = s > 0 ? sweep_steps(n, b, s - 1) : 0;
        const int64_t grp = s / g, gi = s % g;
        for (int64_t k = 0; k < nst; ++k) {
            // wait for sweep s-1 (half steps, see the head of this file): step k+1 complete and
            // the row block of step k+2 stored, 2(k+2)+1, or the whole sweep when it is shorter.
            // Without the mid-step point (narrow bands, where its fence costs more than the half
            // step it saves), step k+2 complete: 2(k+3)
            if (tid == 0 && s > 0) {
                const int64_t need = min(a.half ? 2 * k + 5 : 2 * k + 6, 2 * prev_nst);
                volatile int *pp = a.progress + (s - 1);
                volatile int *ve = a.err;
                const long long t0 = clock64();
                while ((int64_t)(*pp) < need) {
                    if (*ve) { s_abort = 1; break; }
                    if (clock64() - t0 > a.wait) { atomicCAS(a.err, 0, 2); s_abort = 1; break; }
                    __nanosleep(64);
                }
                __threadfence();
            }
            __syncthreads();
            if (s_abort) return;

            const int64_t r0 = s + 1 + k * b;
            const int L = (int)min((int64_t)b, n - r0);
            const int64_t c = (k == 0) ? s : s + 1 + (k - 1) * b;
            // ---- 1. the column to annihilate
            if (tid < L) s_v[tid] = (k == 0) ? bget<R>(band, ldb, r0 + tid, c) : Rc[tid];
            __syncthreads();
            // ---- 2. reflector (one warp)
            if (tid < 32) {
                R acc = 0;
                for (int i = 1 + tid; i < L; i += 32) acc += cabs2(s_v[i]);
                acc = warp_sum(acc);
                if (tid == 0) {
                    Cx al = s_v[0];
                    double ax = al.x, ay = al.y;
                    double aa = sqrt(ax * ax + ay * ay);
                    double nrm = sqrt((double)acc + aa * aa);
                    double tau = 0.0, bx = 0.0, by = 0.0, px = 0.0, py = 0.0;
                    if (nrm > 0.0) {
                        double phx = aa == 0.0 ? 1.0 : ax / aa, phy = aa == 0.0 ? 0.0 : ay / aa;
                        bx = -phx * nrm; by = -phy * nrm;
                        double sc = 1.0 / (aa + nrm);
                        px = phx * sc; py = -phy * sc;   // 1 / (alpha - beta)
                        tau = 1.0 + aa / nrm;
                    }
                    s_tau = (R)tau;
                    s_beta = mk<R>((R)bx, (R)by);
                    s_p[0] = mk<R>((R)px, (R)py);
                }
            }
            __syncthreads();
            const R tau = s_tau;
            if (tid < L) {
                Cx v = (tid == 0) ? mk<R>(1, 0) : cmul(s_v[tid], s_p[0]);
                if (tau == 0) v = (tid == 0) ? mk<R>(1, 0) : czero<Cx>();
                s_v[tid] = v;
            }
            __syncthreads();
            // store the reflector for the back-transformation
            {
                Cx *dst = refl + (a.grp_off[grp] + k * g + gi) * (int64_t)b;
                if (tid < b) dst[tid] = (tid < L) ? s_v[tid] : czero<Cx>();
                if (tid == 0) taus[a.grp_off[grp] + k * g + gi] = tau;
            }
            // ---- 3. the annihilated column
            if (k == 0) {
                if (tid < L) bset<R>(band, ldb, r0 + tid, c, tid == 0 ? s_beta : czero<Cx>());
            } else {
                if (tid < L) Rc[tid] = (tid == 0) ? s_beta : czero<Cx>();
            }
            // ---- 4. left application to the rest of the current block, then store it
            if (k > 0) {
                // w_cc = v^H Rc[:, cc], cc = 1..b-1 ; 4 threads per column
                for (int base = 0; base < b; base += 64) {
                    int cc = base + (tid >> 2), q = tid & 3;
                    Cx acc = czero<Cx>();
                    if (cc >= 1 && cc < b)
                        for (int i = q; i < L; i += 4) cfmac(acc, s_v[i], Rc[i + cc * ls]);
                    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
                    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
                    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
                    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
                    if (q == 0 && cc < b) s_w[cc] = cscale(acc, tau);
                }
                __syncthreads();
                for (int e = tid; e < L * b; e += blockDim.x) {
                    int i = e % L, cc = e / L;
                    if (cc == 0) continue;
                    Rc[i + cc * ls] = csub(Rc[i + cc * ls], cmul(s_v[i], s_w[cc]));
                }
                __syncthreads();
                for (int e = tid; e < L * b; e += blockDim.x) {
                    int i = e % L, cc = e / L;
                    bset<R>(band, ldb, r0 + i, c + cc, Rc[i + cc * ls]);
                }
            }
            // the row block (or, at step 0, the annihilated column) is stored: half-step progress
            if (a.half) {
                __threadfence();
                __syncthreads();
                if (tid == 0) atomicExch(a.progress + s, (int)(2 * k + 1));
            }
            // ---- 5. two-sided application to the diagonal block
            {
                // all loads of this thread first (independent, in flight together)
                constexpr int PER = 16;   // (64 * 64) / 256
                Cx vals[PER];
#pragma unroll
                for (int q = 0; q < PER; ++q) {
                    int e = tid + q * 256;
                    int i = e % L, j = e / L;
                    vals[q] = (e < L * L && i >= j) ? bget<R>(band, ldb, r0 + i, r0 + j) : czero<Cx>();
                }
#pragma unroll
                for (int q = 0; q < PER; ++q) {
                    int e = tid + q * 256;
                    int i = e % L, j = e / L;
                    if (e < L * L && i >= j) {
                        Cx v = vals[q];
                        if (i == j) v.y = 0;
                        D[i + j * ls] = v;
                        if (i != j) D[j + i * ls] = cconj(v);
                    }
                }
            }
            __syncthreads();
            // p = tau D v  (4 threads per row)
            {
                int i = tid >> 2, q = tid & 3;
                Cx acc = czero<Cx>();
                if (i < L)
                    for (int j = q; j < L; j += 4) cfma(acc, D[i + j * ls], s_v[j]);
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
                if (q == 0 && i < L) s_p[i] = cscale(acc, tau);
            }
            __syncthreads();
            // K = tau/2 Re(v^H p) ; w = p - K v
            if (tid < 32) {
                R acc = 0;
                for (int i = tid; i < L; i += 32) { Cx t = s_v[i], p = s_p[i]; acc += t.x * p.x + t.y * p.y; }
                acc = warp_sum(acc);
                if (tid == 0) s_red[0] = (R)0.5 * tau * acc;
            }
            __syncthreads();
            if (tid < L) s_w[tid] = csub(s_p[tid], cscale(s_v[tid], s_red[0]));
            __syncthreads();
            // D -= v w^H + w v^H ; store the lower triangle
            for (int e = tid; e < L * L; e += blockDim.x) {
                int i = e % L, j = e / L;
                if (i < j) continue;
                Cx t = D[i + j * ls];
                Cx vi = s_v[i], wi = s_w[i], vj = s_v[j], wj = s_w[j];
                // v_i conj(w_j) + w_i conj(v_j)
                Cx u1 = mk<R>(vi.x * wj.x + vi.y * wj.y, vi.y * wj.x - vi.x * wj.y);
                Cx u2 = mk<R>(wi.x * vj.x + wi.y * vj.y, wi.y * vj.x - wi.x * vj.y);
                t = csub(t, cadd(u1, u2));
                if (i == j) t.y = 0;
                bset<R>(band, ldb, r0 + i, r0 + j, t);
            }
            // ---- 6. right application to the block below (creates the next bulge)
            const int64_t rn0 = r0 + L;
            const int L2 = (int)min((int64_t)b, n - rn0);
            if (L2 > 0) {
                {
                    constexpr int PER = 16;
                    Cx vals[PER];
#pragma unroll
                    for (int q = 0; q < PER; ++q) {
                        int e = tid + q * 256;
                        int i = e % L2, j = e / L2;
                        vals[q] = (e < L2 * L) ? bget<R>(band, ldb, rn0 + i, r0 + j) : czero<Cx>();
                    }
#pragma unroll
                    for (int q = 0; q < PER; ++q) {
                        int e = tid + q * 256;
                        int i = e % L2, j = e / L2;
                        if (e < L2 * L) Rn[i + j * ls] = vals[q];
                    }
                }
                __syncthreads();
                // y_i = sum_j Rn[i][j] v_j ; Rn[i][j] -= tau y_i conj(v_j)
                {
                    int i = tid >> 2, q = tid & 3;
                    Cx acc = czero<Cx>();
                    if (i < L2)
                        for (int j = q; j < L; j += 4) cfma(acc, Rn[i + j * ls], s_v[j]);
                    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
                    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
                    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
                    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
                    if (q == 0 && i < L2) s_p[i] = cscale(acc, tau);
                }
                __syncthreads();
                const bool keep = (k + 1 < nst);
                for (int e = tid; e < L2 * L; e += blockDim.x) {
                    int i = e % L2, j = e / L2;
                    Cx vj = s_v[j], y = s_p[i];
                    // y * conj(v_j)
                    Cx u = mk<R>(y.x * vj.x + y.y * vj.y, y.y * vj.x - y.x * vj.y);
                    Cx t = csub(Rn[i + j * ls], u);
                    if (keep) Rc[i + j * ls] = t;          // becomes the next step's row block
                    else bset<R>(band, ldb, rn0 + i, r0 + j, t);
                }
            }
            // publish progress: every thread fences its band writes first
            __threadfence();
            __syncthreads();
            if (tid == 0) atomicExch(a.progress + s, (int)(2 * k + 2));
        }
        __syncthreads();
    }
}

// T factors of the grouped block reflectors used by the back-transformation:
// block (J, k) = H(j0,k) H(j0+1,k) ... H(j0+g-1,k) = I - V T V^H, where the
// member i's vector sits at rows i .. i+b-1 of the (g+b-1)-row block.
template <typename R>
__global__ void bt2_tfactor_kernel(int64_t n, int b, int g, const cplx<R> *__restrict__ refl,
                                   const R *__restrict__ taus, const int64_t *__restrict__ grp_off,
                                   const int64_t *__restrict__ blk_list, cplx<R> *__restrict__ VTst,
                                   int64_t blk0) {
    using Cx = cplx<R>;
    // blk_list[2*q] = group J, blk_list[2*q+1] = k
    const int64_t J = blk_list[2 * blockIdx.x], k = blk_list[2 * blockIdx.x + 1];
    const int64_t slot0 = grp_off[J] + k * g;
    const Cx *V = refl + slot0 * (int64_t)b;   // member i at V + i*b (b entries, row offset i)
    const R *tau = taus + slot0;
    const int MR = g + b - 1;
    Cx *VT = VTst + (blk0 + blockIdx.x) * (int64_t)MR * g;   // MR x g, ld MR
    extern __shared__ unsigned char smem_raw[];
    Cx *Gm = reinterpret_cast<Cx *>(smem_raw);  // g x g Gram, ld g
    Cx *Tm = Gm + g * g;                        // g x g T factor
    // Gram(i, j) = v_i^H v_j for i < j (rows overlap where j - i < b)
    for (int e = threadIdx.x; e < g * g; e += blockDim.x) {
        int i = e % g, j = e / g;
        Cx acc = czero<Cx>();
        if (i < j && j - i < b) {
            // v_i row r (0..b-1) is block row i + r; v_j row r' is block row j + r'
            for (int r = j - i; r < b; ++r) cfmac(acc, V[(int64_t)i * b + r], V[(int64_t)j * b + (r - (j - i))]);
        }
        Gm[e] = acc;
    }
    __syncthreads();
    for (int j = 0; j < g; ++j) {
        const R tj = tau[j];
        int i = threadIdx.x;
        Cx zi = czero<Cx>();
        if (i < j)
            for (int q = i; q < j; ++q) {
                Cx tiq = (q == i) ? mk<R>(tau[i], 0) : Gm[i + q * g];
                cfma(zi, tiq, Gm[q + j * g]);
            }
        __syncthreads();
        if (i < j) Gm[i + j * g] = cscale(zi, -tj);
        __syncthreads();
    }
    for (int e = threadIdx.x; e < g * g; e += blockDim.x) {
        int i = e % g, j = e / g;
        Cx t = czero<Cx>();
        if (i < j) t = Gm[e];
        else if (i == j) t = mk<R>(tau[i], 0);
        Tm[e] = t;
    }
    __syncthreads();
    // VT(r, j) = sum_{q <= j} V(r, q) T(q, j), V(r, q) = refl[q][r - q] for 0 <= r - q < b
    for (int e = threadIdx.x; e < MR * g; e += blockDim.x) {
        int r = e % MR, j = e / MR;
        Cx acc = czero<Cx>();
        int qlo = max(0, r - b + 1), qhi = min(j, r);
        for (int q = qlo; q <= qhi; ++q) cfma(acc, V[(int64_t)q * b + (r - q)], Tm[q + j * g]);
        VT[e] = acc;
    }
}

// E <- Q2 E for a slab of 64 columns per CTA.  For groups J from last to
// first and k ascending (the order in which overlapping block reflectors
// must be applied), with the window Ew = E[rs : rs+MR, slab]:
//   W  = V^H Ew      (g x 64; V is a staircase: member i has rows i .. i+b-1)
//   Ew = Ew - VT W   (VT = V T precomputed per block; VT(r, i) = 0 for i <= r-b)
// Both products are register-tiled (4x4 and 8x4 complex per thread).
template <typename R>
__global__ void __launch_bounds__(256, 1) bt2_apply_kernel(int64_t n, int b, int g, int64_t ngroups,
                                                           const cplx<R> *__restrict__ refl,
                                                           const int64_t *__restrict__ grp_off,
                                                           const int64_t *__restrict__ blk_off,
                                                           const cplx<R> *__restrict__ VTst, cplx<R> *__restrict__ E,
                                                           int64_t lde, int64_t ncols) {
    using Cx = cplx<R>;
    constexpr int NC = 64;
    extern __shared__ unsigned char smem_raw[];
    const int MR = g + b - 1;
    const int MRP = ((MR + 7) / 8) * 8;          // padded window rows
    Cx *Ew = reinterpret_cast<Cx *>(smem_raw);   // MRP x NC, [r][c]
    Cx *Vs = Ew + (int64_t)MRP * NC;             // g x b, [i][t]
    Cx *VTs = Vs + (int64_t)g * b;               // MRP x g, [r][i]
    Cx *Ws = VTs + (int64_t)MRP * g;             // g x NC, [i][c]
    const int tid = threadIdx.x;
    const int tc = tid & 15, ti = tid >> 4;      // 16 column groups x 16 row groups
    const int64_t c0 = (int64_t)blockIdx.x * NC;
    const int ncl = (int)min((int64_t)NC, ncols - c0);
    for (int64_t J = ngroups - 1; J >= 0; --J) {
        const int64_t j0 = J * g;
        const int64_t nst = sweep_steps(n, b, j0);
        for (int64_t k = 0; k < nst; ++k) {
            const int64_t rs = j0 + 1 + k * b;
            const int rows = (int)min((int64_t)MR, n - rs);
            const int64_t slot0 = grp_off[J] + k * g;
            const Cx *VTg = VTst + (blk_off[J] + k) * (int64_t)MR * g;
            // ---- load window, reflectors, VT
            for (int e = tid; e < MRP * NC; e += 256) {
                int r = e % MRP, c = e / MRP;
                Ew[r * NC + c] = (r < rows && c < ncl) ? E[(rs + r) + (c0 + c) * lde] : czero<Cx>();
            }
            for (int e = tid; e < g * b; e += 256) Vs[e] = refl[slot0 * (int64_t)b + e];
            for (int e = tid; e < MRP * g; e += 256) {
                int r = e % MRP, i = e / MRP;
                VTs[r * g + i] = (r < MR) ? VTg[r + (int64_t)i * MR] : czero<Cx>();
            }
            __syncthreads();
            // ---- W = V^H Ew : thread owns rows i = 4 ti .. 4 ti + 3 (g = 64) and columns tc + 16 q
            {
                Cx acc[4][4];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[a][q] = czero<Cx>();
                const int i0 = 4 * ti;
                if (i0 < g) {
                    const int rlo = i0, rhi = min(i0 + 3 + b - 1, MR - 1);
                    for (int r = rlo; r <= rhi; ++r) {
                        Cx e4[4], v4[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) e4[q] = Ew[r * NC + tc + 16 * q];
#pragma unroll
                        for (int a = 0; a < 4; ++a) {
                            const int t = r - (i0 + a);
                            v4[a] = (t >= 0 && t < b && i0 + a < g) ? Vs[(i0 + a) * b + t] : czero<Cx>();
                        }
#pragma unroll
                        for (int a = 0; a < 4; ++a)
#pragma unroll
                            for (int q = 0; q < 4; ++q) cfmac(acc[a][q], v4[a], e4[q]);
                    }
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (i0 + a < g) Ws[(i0 + a) * NC + tc + 16 * q] = acc[a][q];
                }
            }
            __syncthreads();
            // ---- Ew -= VT W : thread owns rows r = 8 ti .. 8 ti + 7 and columns tc + 16 q
            for (int rb = 8 * ti; rb < MRP; rb += 128) {
                Cx acc[8][4];
#pragma unroll
                for (int a = 0; a < 8; ++a)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[a][q] = czero<Cx>();
                const int ilo = max(0, rb - b + 1);
                for (int i = ilo; i < g; ++i) {
                    Cx w4[4], v8[8];
#pragma unroll
                    for (int q = 0; q < 4; ++q) w4[q] = Ws[i * NC + tc + 16 * q];
#pragma unroll
                    for (int a = 0; a < 8; ++a) v8[a] = VTs[(rb + a) * g + i];
#pragma unroll
                    for (int a = 0; a < 8; ++a)
#pragma unroll
                        for (int q = 0; q < 4; ++q) cfma(acc[a][q], v8[a], w4[q]);
                }
#pragma unroll
                for (int a = 0; a < 8; ++a) {
                    const int r = rb + a;
                    if (r < rows) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int c = tc + 16 * q;
                            if (c < ncl) E[(rs + r) + (c0 + c) * lde] = csub(Ew[r * NC + c], acc[a][q]);
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Asynchronous global -> shared copy of one complex element (8 or 16 bytes).
template <typename C>
__device__ __forceinline__ void cp_async_elem(C *dst, const C *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(C) == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Same operation as bt2_apply_kernel, arranged for the sequence of windows
// of one group: the window E[rs : rs+MR, slab] of step k+1 shares MR-b rows
// with that of step k, so the window lives in a circular buffer of BUF rows
// (row r of the matrix at position r mod BUF) and each step loads only its b
// new rows and writes back only the b rows no later step of the group
// touches.  V is kept as a dense G x BUF staircase (zeros outside rows
// i .. i+b-1 of member i) so the inner loops have no bounds tests; all
// shared tiles are column-major with an odd leading dimension for Ew
// (conflict-free column accesses).  V and VT arrive by cp.async.
// THREADS = 16 column groups x TI row groups (256 or 512); one CTA per SM (the
// shared tiles take ~226 KB), so 512 threads give twice the warps to hide the
// shared-memory latency of the inner loops.
template <typename R, int NC, int BUF, int G, int THREADS>
__global__ void __launch_bounds__(THREADS, 1) bt2_apply_circ_kernel(int64_t n, int b, int64_t ngroups,
                                                                const cplx<R> *__restrict__ refl,
                                                                const int64_t *__restrict__ grp_off,
                                                                const int64_t *__restrict__ blk_off,
                                                                const cplx<R> *__restrict__ VTst,
                                                                cplx<R> *__restrict__ E, int64_t lde, int64_t ncols) {
    using Cx = cplx<R>;
    // FP32: the inner products run on packed two-lane FMAs (one instruction per two FMAs)
    constexpr bool kPacked = std::is_same<R, float>::value;
    constexpr int LDR = BUF + 1;
    constexpr int TI = THREADS / 16;   // row groups
    constexpr int QC = NC / 16;        // columns per thread
    constexpr int A1 = G / TI;         // reflectors per thread in W = V^H Ew
    constexpr int A2 = BUF / TI;       // window rows per thread in Ew -= VT W
    static_assert(BUF == 2 * G && A2 % 2 == 0 && TI * (A2 / 2) == G && A1 * TI == G,
                  "bt2_apply_circ_kernel: the balanced row split assumes BUF = 2 G and b = G");
    const int MR = G + b - 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx *Ew = reinterpret_cast<Cx *>(smem_raw);   // [NC][LDR]
    Cx *Vf = Ew + NC * LDR;                      // [G][BUF]
    Cx *VT = Vf + G * BUF;                       // [G][BUF]
    Cx *Ws = VT + G * BUF;                       // [G][NC]
    const int tid = threadIdx.x, tc = tid & 15, ti = tid >> 4;
    const int64_t c0 = (int64_t)blockIdx.x * NC;
    const int ncl = (int)min((int64_t)NC, ncols - c0);
    for (int e = tid; e < 2 * G * BUF; e += THREADS) Vf[e] = czero<Cx>();   // Vf and VT: zeros off the staircase
    __syncthreads();
    for (int64_t J = ngroups - 1; J >= 0; --J) {
        const int64_t j0 = J * G;
        const int64_t nst = sweep_steps(n, b, j0);
        for (int64_t k = 0; k < nst; ++k) {
            const int64_t rs = j0 + 1 + k * b;
            const int rows = (int)min((int64_t)MR, n - rs);
            const Cx *Vg = refl + (grp_off[J] + k * G) * (int64_t)b;
            const Cx *VTg = VTst + (blk_off[J] + k) * (int64_t)MR * G;
            for (int e = tid; e < G * b; e += THREADS) {
                const int i = e / b, t = e - i * b;
                cp_async_elem(&Vf[i * BUF + i + t], Vg + e);
            }
            for (int e = tid; e < G * MR; e += THREADS) {
                const int i = e / MR, r = e - i * MR;
                cp_async_elem(&VT[i * BUF + r], VTg + e);
            }
            // window rows: all of them at the first step, else the b new ones
            const int lr0 = (k == 0) ? 0 : MR - b;
            const int nl = MR - lr0;
#pragma unroll 4
            for (int e = tid; e < nl * NC; e += THREADS) {
                const int c = e / nl, r = lr0 + (e - c * nl);
                const int64_t gr = rs + r;
                Ew[c * LDR + (int)(gr & (BUF - 1))] =
                    (gr < n && c < ncl) ? ldcg(&E[gr + (c0 + c) * lde]) : czero<Cx>();
            }
            cp_async_wait_all();
            __syncthreads();
            // ---- W = V^H Ew
            if constexpr (kPacked) {
                // two packed sums per entry: P = sum Re v (Re e, Im e), Q = sum Im v (Re e, Im e);
                // conj(v) e = (P.x + Q.y, P.y - Q.x)
                float2 accP[A1][QC], accQ[A1][QC];
#pragma unroll
                for (int a = 0; a < A1; ++a)
#pragma unroll
                    for (int q = 0; q < QC; ++q) { accP[a][q] = make_float2(0.f, 0.f); accQ[a][q] = accP[a][q]; }
                const int i0 = ti * A1;
                const int rend = i0 + A1 - 1 + b;   // <= MR
                for (int r = i0; r < rend; ++r) {
                    const int pos = (int)((rs + r) & (BUF - 1));
                    float2 ev[QC];
#pragma unroll
                    for (int q = 0; q < QC; ++q) ev[q] = Ew[(tc + 16 * q) * LDR + pos];
#pragma unroll
                    for (int a = 0; a < A1; ++a) {
                        const float2 v = Vf[(i0 + a) * BUF + r];
                        const float2 vr = make_float2(v.x, v.x), vi = make_float2(v.y, v.y);
#pragma unroll
                        for (int q = 0; q < QC; ++q) {
                            accP[a][q] = __ffma2_rn(vr, ev[q], accP[a][q]);
                            accQ[a][q] = __ffma2_rn(vi, ev[q], accQ[a][q]);
                        }
                    }
                }
#pragma unroll
                for (int a = 0; a < A1; ++a)
#pragma unroll
                    for (int q = 0; q < QC; ++q)
                        Ws[(i0 + a) * NC + tc + 16 * q] =
                            make_float2(accP[a][q].x + accQ[a][q].y, accP[a][q].y - accQ[a][q].x);
            } else {
                Cx acc[A1][QC];
#pragma unroll
                for (int a = 0; a < A1; ++a)
#pragma unroll
                    for (int q = 0; q < QC; ++q) acc[a][q] = czero<Cx>();
                const int i0 = ti * A1;
                const int rend = i0 + A1 - 1 + b;   // <= MR
                for (int r = i0; r < rend; ++r) {
                    const int pos = (int)((rs + r) & (BUF - 1));
                    Cx ev[QC], vv[A1];
#pragma unroll
                    for (int q = 0; q < QC; ++q) ev[q] = Ew[(tc + 16 * q) * LDR + pos];
#pragma unroll
                    for (int a = 0; a < A1; ++a) vv[a] = Vf[(i0 + a) * BUF + r];
#pragma unroll
                    for (int a = 0; a < A1; ++a)
#pragma unroll
                        for (int q = 0; q < QC; ++q) cfmac(acc[a][q], vv[a], ev[q]);
                }
#pragma unroll
                for (int a = 0; a < A1; ++a)
#pragma unroll
                    for (int q = 0; q < QC; ++q) Ws[(i0 + a) * NC + tc + 16 * q] = acc[a][q];
            }
            __syncthreads();
            // ---- Ew -= VT W.  Window row r has VT(r, i) = 0 for i < r - b + 1 (b = G here), so
            // the rows r >= G need only the tail i >= r - G + 1 of the reflector range.  Each
            // thread group ti takes HT top rows (r = HT ti + a, the full range) and HT rows
            // r = G + ti + TI c, whose ranges start at i = 1 + ti + TI c: the groups then do
            // nearly equal work.  The i loop runs in HT + 1 segments; in segment c the bottom
            // rows 0 .. c are active.
            {
                constexpr int HT = A2 / 2;
                // FP32: two packed sums per entry, P = sum Re v (Re w, Im w) and Q = sum Im v
                // (Re w, Im w), so v w = (P.x - Q.y, P.y + Q.x); FP64: complex FMAs
                Cx acc[A2][QC];   // [0, HT): top rows; [HT, A2): bottom rows (P when packed)
                Cx accQ[kPacked ? A2 : 1][kPacked ? QC : 1];
#pragma unroll
                for (int a = 0; a < A2; ++a)
#pragma unroll
                    for (int q = 0; q < QC; ++q) acc[a][q] = czero<Cx>();
                if constexpr (kPacked) {
#pragma unroll
                    for (int a = 0; a < A2; ++a)
#pragma unroll
                        for (int q = 0; q < QC; ++q) accQ[a][q] = czero<Cx>();
                }
                auto fma_row = [&](int a, Cx vv, const Cx *wv) {
                    if constexpr (kPacked) {
                        const float2 vr = make_float2(vv.x, vv.x), vi = make_float2(vv.y, vv.y);
#pragma unroll
                        for (int q = 0; q < QC; ++q) {
                            acc[a][q] = __ffma2_rn(vr, wv[q], acc[a][q]);
                            accQ[a][q] = __ffma2_rn(vi, wv[q], accQ[a][q]);
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < QC; ++q) cfma(acc[a][q], vv, wv[q]);
                    }
                };
#pragma unroll
                for (int c = -1; c < HT; ++c) {
                    const int ilo = (c < 0) ? 0 : 1 + ti + TI * c;
                    const int ihi = min(G, (c + 1 < HT) ? 1 + ti + TI * (c + 1) : G);
                    for (int i = ilo; i < ihi; ++i) {
                        Cx wv[QC];
#pragma unroll
                        for (int q = 0; q < QC; ++q) wv[q] = Ws[i * NC + tc + 16 * q];
#pragma unroll
                        for (int a = 0; a < HT; ++a) fma_row(a, VT[i * BUF + ti * HT + a], wv);
#pragma unroll
                        for (int cc = 0; cc < HT; ++cc) {
                            if (cc <= c) fma_row(HT + cc, VT[i * BUF + G + ti + TI * cc], wv);
                        }
                    }
                }
#pragma unroll
                for (int a = 0; a < A2; ++a) {
                    const int r = (a < HT) ? ti * HT + a : G + ti + TI * (a - HT);
                    if (r < rows) {
                        const int pos = (int)((rs + r) & (BUF - 1));
#pragma unroll
                        for (int q = 0; q < QC; ++q) {
                            Cx &x = Ew[(tc + 16 * q) * LDR + pos];
                            if constexpr (kPacked) {
                                const Cx t = acc[a][q], u = accQ[kPacked ? a : 0][kPacked ? q : 0];
                                x = csub(x, mk<R>(t.x - u.y, t.y + u.x));
                            } else {
                                x = csub(x, acc[a][q]);
                            }
                        }
                    }
                }
            }
            __syncthreads();
            // ---- rows no later step of this group touches go back to E
            const int nw = (k == nst - 1) ? rows : min(b, rows);
#pragma unroll 4
            for (int e = tid; e < nw * NC; e += THREADS) {
                const int c = e / nw, r = e - c * nw;
                if (c < ncl) E[(rs + r) + (c0 + c) * lde] = Ew[c * LDR + (int)((rs + r) & (BUF - 1))];
            }
            __syncthreads();
        }
    }
}

template <typename R>
int stage2_reduce(bdg_ctx *ctx, cudaStream_t st, int64_t n, int b, int g, cplx<R> *band, int ldband,
                  cplx<R> *refl, R *taus, const int64_t *grp_off_dev, unsigned int *ticket, int *progress,
                  int64_t nrefl_slots) {
    using Cx = cplx<R>;
    if (n < 3) return BDG_OK;
    BDG_CUDA_TRY(ctx, cudaMemsetAsync(refl, 0, (size_t)nrefl_slots * b * sizeof(Cx), st));
    BDG_CUDA_TRY(ctx, cudaMemsetAsync(taus, 0, (size_t)nrefl_slots * sizeof(R), st));
    BDG_CUDA_TRY(ctx, cudaMemsetAsync(ticket, 0, sizeof(unsigned int), st));
    BDG_CUDA_TRY(ctx, cudaMemsetAsync(progress, 0, (size_t)n * sizeof(int), st));
    BDG_CUDA_TRY(ctx, cudaMemsetAsync(ctx->dflags, 0, 4 * sizeof(int), st));
    size_t smem = (size_t)3 * b * (b + 1) * sizeof(Cx);
    BDG_CUDA_TRY(ctx, cudaFuncSetAttribute(bulge_chase_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem));
    int per_sm = 0;
    BDG_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bulge_chase_kernel<R>, 256, smem));
    if (per_sm < 1) return bdg_fail(ctx, BDG_EUNSUPPORTED, "bulge-chasing kernel cannot be resident (b=%d)", b);
    int64_t grid = (int64_t)per_sm * ctx->num_sms;
    grid = std::min<int64_t>(grid, n - 2);
    Stage2Args a;
    a.n = n; a.b = b; a.ldband = ldband; a.g = g; a.band = band; a.refl = refl; a.tau = taus;
    a.grp_off = grp_off_dev; a.ticket = ticket; a.progress = progress; a.err = ctx->dflags;
    a.wait = ctx->wait_cycles;
    // the mid-step point pays where a step is long (about 21 us at b = 64): it lets the next sweep
    // start half a step earlier for one more fence and barrier per step
    a.half = b >= 48 ? 1 : 0;
    bulge_chase_kernel<R><<<(unsigned)grid, 256, smem, st>>>(a);
    BDG_LAUNCH_CHECK(ctx);
    return BDG_OK;
}

template <typename R>
int stage2_backtransform(bdg_ctx *ctx, cudaStream_t st, int64_t n, int b, int g, const cplx<R> *refl,
                         const R *taus, const int64_t *grp_off_dev, const int64_t *blk_list_dev, int64_t nblk,
                         const int64_t *blk_off_dev, cplx<R> *Tst, cplx<R> *E, int64_t lde, int64_t ncols) {
    using Cx = cplx<R>;
    if (n < 3 || nblk == 0) return BDG_OK;
    size_t smt = (size_t)2 * g * g * sizeof(Cx);
    if (smt > 48 * 1024)
        BDG_CUDA_TRY(ctx, cudaFuncSetAttribute(bt2_tfactor_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smt));
    int64_t done = 0;
    while (done < nblk) {
        int64_t cnt = std::min<int64_t>(nblk - done, 1 << 30);
        bt2_tfactor_kernel<R><<<(unsigned)cnt, 64, smt, st>>>(n, b, g, refl, taus, grp_off_dev,
                                                              blk_list_dev + 2 * done, Tst, done);
        BDG_LAUNCH_CHECK(ctx);
        done += cnt;
    }
    int64_t ngroups = (n - 2 + g - 1) / g;
    // circular-window kernel for the standard (b, g) of each precision
    if constexpr (sizeof(R) == 4) {
        if (b == 64 && g == 64) {
            constexpr int NCc = 64, BUF = 128, G = 64, TH = 512;
            const size_t smc = ((size_t)NCc * (BUF + 1) + 2 * (size_t)G * BUF + (size_t)G * NCc) * sizeof(Cx);
            if (smc <= (size_t)ctx->smem_optin) {
                BDG_CUDA_TRY(ctx, cudaFuncSetAttribute(bt2_apply_circ_kernel<R, NCc, BUF, G, TH>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc));
                unsigned gx = (unsigned)((ncols + NCc - 1) / NCc);
                bt2_apply_circ_kernel<R, NCc, BUF, G, TH><<<gx, TH, smc, st>>>(n, b, ngroups, refl, grp_off_dev,
                                                                               blk_off_dev, Tst, E, lde, ncols);
                BDG_LAUNCH_CHECK(ctx);
                return BDG_OK;
            }
        }
    } else {
        if (b == 32 && g == 32) {
            constexpr int NCc = 32, BUF = 64, G = 32, TH = 256;
            const size_t smc = ((size_t)NCc * (BUF + 1) + 2 * (size_t)G * BUF + (size_t)G * NCc) * sizeof(Cx);
            if (smc <= (size_t)ctx->smem_optin) {
                BDG_CUDA_TRY(ctx, cudaFuncSetAttribute(bt2_apply_circ_kernel<R, NCc, BUF, G, TH>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc));
                unsigned gx = (unsigned)((ncols + NCc - 1) / NCc);
                bt2_apply_circ_kernel<R, NCc, BUF, G, TH><<<gx, TH, smc, st>>>(n, b, ngroups, refl, grp_off_dev,
                                                                               blk_off_dev, Tst, E, lde, ncols);
                BDG_LAUNCH_CHECK(ctx);
                return BDG_OK;
            }
        }
    }
    constexpr int NC = 64;
    const int MR = g + b - 1, MRP = ((MR + 7) / 8) * 8;
    size_t sm = ((size_t)MRP * NC + (size_t)g * b + (size_t)MRP * g + (size_t)g * NC) * sizeof(Cx);
    if (sm > (size_t)ctx->smem_optin)
        return bdg_fail(ctx, BDG_EUNSUPPORTED, "stage-2 back-transformation: %zu bytes of shared memory", sm);
    BDG_CUDA_TRY(ctx, cudaFuncSetAttribute(bt2_apply_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    unsigned gridx = (unsigned)((ncols + NC - 1) / NC);
    bt2_apply_kernel<R><<<gridx, 256, sm, st>>>(n, b, g, ngroups, refl, grp_off_dev, blk_off_dev, Tst, E, lde, ncols);
    BDG_LAUNCH_CHECK(ctx);
    return BDG_OK;
}

template int stage2_reduce<float>(bdg_ctx *, cudaStream_t, int64_t, int, int, float2 *, int, float2 *, float *,
                                  const int64_t *, unsigned int *, int *, int64_t);
template int stage2_reduce<double>(bdg_ctx *, cudaStream_t, int64_t, int, int, double2 *, int, double2 *,
                                   double *, const int64_t *, unsigned int *, int *, int64_t);
template int stage2_backtransform<float>(bdg_ctx *, cudaStream_t, int64_t, int, int, const float2 *,
                                         const float *, const int64_t *, const int64_t *, int64_t, const int64_t *,
                                         float2 *, float2 *, int64_t, int64_t);
template int stage2_backtransform<double>(bdg_ctx *, cudaStream_t, int64_t, int, int, const double2 *,
                                          const double *, const int64_t *, const int64_t *, int64_t, const int64_t *,
                                          double2 *, double2 *, int64_t, int64_t);

}  // namespace bdg
