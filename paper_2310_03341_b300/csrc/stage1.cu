// Stage 1 of the two-stage reduction: dense Hermitian -> band of width b
// (paper, section "Performance of the Matrix Diagonalization Algorithm":
// the 2-stage solver first transforms the dense matrix into a banded one).
//
// For panel p (columns c0 = p*b .. c0+b-1, rows r0 = c0+b .. n-1, m = n-r0):
//   1. Householder QR of the m x b panel:  Q_p = H_1 ... H_b = I - V T V^H,
//      H_j = I - tau_j v_j v_j^H with real tau_j and v_j(0) = 1, chosen so
//      that H_j x = beta_j e_1, beta_j = -exp(i arg x_0) ||x||.
//   2. Two-sided trailing update A22 <- Q_p^H A22 Q_p written as the rank-2b
//      update  A22 -= V W^H + W V^H  with
//          X = A22 V T,  M = V^H X,  W = X - 1/2 V (T^H M).
// The panel QR runs as one cooperative kernel: every CTA keeps its slice of
// panel rows in shared memory and the column reductions (norms, v^H P) go
// through a bounded software grid barrier -- two barriers per column.
// The trailing update is three GEMMs plus a split-K reduction.
#include <cuda_bf16.h>

#include <algorithm>

#include <stdlib.h>

#include "internal.h"

namespace bdg {

template <typename C>
int split_planes(bdg_ctx *ctx, cudaStream_t st, int64_t rows, int64_t cols, const C *X, int64_t ldx, bool transpose,
                 bool conj_, int S, __nv_bfloat16 *planes);
int cgemm_bf16(bdg_ctx *ctx, cudaStream_t st, int S, int64_t M, int64_t N, int64_t K, const __nv_bfloat16 *pa,
               const __nv_bfloat16 *pb, float2 *C, int64_t ldc, float alpha, float beta, float2 *part, int splits);
// K-split factor for a narrow product with `mtiles` output tiles
static inline int narrow_splits(int64_t mtiles, int num_sms) {
    int64_t z = (2 * (int64_t)num_sms + mtiles - 1) / std::max<int64_t>(mtiles, 1);
    return (int)std::max<int64_t>(1, std::min<int64_t>(8, z));
}

// Panel QR.  Writes:
//   A[r0.., c0..]  : R (upper triangle) and v_j below it (LAPACK-like);
//   Vout (m x b, ld ldv) : explicit V (unit diagonal, zeros above);
//   Tout (b x b, ld b)   : the upper-triangular T factor;
//   red (workspace)      : gridDim.x * (2 + 2b + b*b) + b*b + 2b + 2 complex partials.
// Every sum over the CTAs' partials is a warp reduction (lanes stride over
// the CTAs, then a shuffle tree): fixed order, and a few dependent L2 loads
// per lane instead of one per CTA.
template <typename R>
__global__ void __launch_bounds__(256) panel_qr_kernel(int64_t m, int b, int nb, cplx<R> *__restrict__ P,
                                                       int64_t lda, cplx<R> *__restrict__ Vout, int64_t ldv,
                                                       cplx<R> *__restrict__ Vout2, int64_t ldv2,
                                                       cplx<R> *__restrict__ Tout, cplx<R> *__restrict__ red,
                                                       R *__restrict__ tau_out, GridBarrier *gb, int64_t chunk) {
    using Cx = cplx<R>;
    extern __shared__ unsigned char smem_raw[];
    Cx *S = reinterpret_cast<Cx *>(smem_raw);      // [b][chunk] panel slice, column-major
    __shared__ R s_red[32];
    __shared__ Cx s_w[64];
    __shared__ Cx s_scal[4];                        // alpha, pivot^-1, beta, (tau, 0)
    const int G = gridDim.x, g = blockIdx.x;
    const int64_t rlo = (int64_t)g * chunk, rhi = min(m, rlo + chunk);
    const int64_t nloc = max((int64_t)0, rhi - rlo);
    // partials of column j live in buffer j & 1: a CTA writes those of column j+1 only after the
    // barrier of column j, which every CTA reaches after reading those of column j-1
    Cx *red_norm = red;                          // [2][G]: ||x_tail||^2 partials (in .x)
    Cx *red_alpha = red_norm + 2 * G;            // [2]: the owner's alpha = P(j, j)
    Cx *red_row = red_alpha + 2;                 // [2][b]: the owner's row j, P(j, c) for c > j
    Cx *red_x = red_row + 2 * b;                 // [2][G][b]: sum over local rows r > j of conj(x_r) P(r, c)
    Cx *red_vv = red_x + 2 * (int64_t)G * b;     // [G][b][b]
    Cx *red_gram = red_vv + (int64_t)G * b * b;  // [b][b] sum of red_vv over the CTAs
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;

    // load the slice
    for (int64_t e = threadIdx.x; e < nloc * b; e += blockDim.x) {
        int64_t r = e % nloc, c = e / nloc;
        S[r + c * chunk] = P[(rlo + r) + c * lda];
    }
    __syncthreads();

    // Everything the reflector of column j needs, from column j and the panel as the reflectors
    // 0 .. j-1 left them, in one pass: the partial squared norm below row j, alpha and row j
    // (from the CTA that holds row j), and the partial products sum_r conj(x_r) P(r, c) over
    // the rows r > j.  With v = x / pivot below row j and v_j = 1, w_c = sum conj(v) P(:, c) is
    // then P(j, c) + conj(1 / pivot) sum_r conj(x_r) P(r, c): one grid barrier per column.
    auto column_partials = [&](int j) {
        const int buf = j & 1;
        R acc = 0;
        for (int64_t r = threadIdx.x; r < nloc; r += blockDim.x) {
            const int64_t gr = rlo + r;
            if (gr > j) {
                acc += cabs2(S[r + (int64_t)j * chunk]);
            } else if (gr == j) {
                red_alpha[buf] = S[r + (int64_t)j * chunk];
                for (int c = j + 1; c < b; ++c) red_row[buf * b + c] = S[r + (int64_t)c * chunk];
            }
        }
        acc = block_sum(acc, s_red);
        if (threadIdx.x == 0) red_norm[buf * G + g] = mk<R>(acc, 0);
        for (int c = j + 1 + wid; c < b; c += nw) {
            Cx x = czero<Cx>();
            for (int64_t r = lane; r < nloc; r += 32)
                if (rlo + r > j) cfmac(x, S[r + (int64_t)j * chunk], S[r + (int64_t)c * chunk]);
            x.x = warp_sum(x.x);
            x.y = warp_sum(x.y);
            if (lane == 0) red_x[((int64_t)buf * G + g) * b + c] = x;
        }
    };

    column_partials(0);
    for (int j = 0; j < nb; ++j) {
        if (!grid_sync(gb)) return;
        const int buf = j & 1;
        // reflector scalars (every CTA computes them redundantly, in FP64 for FP32 data)
        if (threadIdx.x < 32) {
            double nrm2 = 0.0;
            for (int q = lane; q < G; q += 32) nrm2 += (double)ldcg(&red_norm[buf * G + q]).x;
            nrm2 = warp_sum(nrm2);
        if (threadIdx.x == 0) {
            Cx al = ldcg(&red_alpha[buf]);
            double ax = (double)al.x, ay = (double)al.y;
            double a = sqrt(ax * ax + ay * ay);
            double nrm = sqrt(nrm2 + a * a);
            double tau, bx, by, pinvx, pinvy;
            if (nrm == 0.0) {
                tau = 0.0; bx = 0.0; by = 0.0; pinvx = 0.0; pinvy = 0.0;
            } else {
                double phx = (a == 0.0) ? 1.0 : ax / a, phy = (a == 0.0) ? 0.0 : ay / a;
                bx = -phx * nrm; by = -phy * nrm;
                // pivot = alpha - beta = ph * (a + nrm); 1/pivot = conj(ph) / (a + nrm)
                double s = 1.0 / (a + nrm);
                pinvx = phx * s; pinvy = -phy * s;
                tau = 1.0 + a / nrm;
            }
            s_scal[0] = mk<R>((R)pinvx, (R)pinvy);
            s_scal[1] = mk<R>((R)bx, (R)by);
            s_scal[2] = mk<R>((R)tau, 0);
        }
        }
        __syncthreads();
        const Cx pinv = s_scal[0];
        const R tau = s_scal[2].x;
        // w_c = P(j, c) + conj(pinv) sum over the CTAs of their partial products (one warp per column)
        for (int c = j + 1 + wid; c < b; c += nw) {
            Cx x = czero<Cx>();
            for (int q = lane; q < G; q += 32) x = cadd(x, ldcg(&red_x[((int64_t)buf * G + q) * b + c]));
            x.x = warp_sum(x.x);
            x.y = warp_sum(x.y);
            if (lane == 0) s_w[c] = cscale(cadd(ldcg(&red_row[buf * b + c]), cmulc(pinv, x)), tau);
        }
        // v = x / pivot below row j; v(j) = 1
        for (int64_t r = threadIdx.x; r < nloc; r += blockDim.x) {
            int64_t gr = rlo + r;
            if (gr > j) S[r + (int64_t)j * chunk] = cmul(S[r + (int64_t)j * chunk], pinv);
        }
        __syncthreads();
        // update the panel: P(:, c) -= tau v w_c
        for (int64_t e = threadIdx.x; e < nloc * (b - j - 1); e += blockDim.x) {
            int64_t r = e % nloc;
            int c = j + 1 + (int)(e / nloc);
            int64_t gr = rlo + r;
            if (gr < j) continue;
            Cx v = (gr == j) ? mk<R>(1, 0) : S[r + (int64_t)j * chunk];
            Cx &pc = S[r + (int64_t)c * chunk];
            pc = csub(pc, cmul(v, s_w[c]));
        }
        // row j of column j becomes beta
        for (int64_t r = threadIdx.x; r < nloc; r += blockDim.x)
            if (rlo + r == j) S[r + (int64_t)j * chunk] = s_scal[1];
        if (g == 0 && threadIdx.x == 0) tau_out[j] = tau;
        __syncthreads();
        if (j + 1 < nb) column_partials(j + 1);
    }
    // columns nb..b-1 (only when m < b): nothing to annihilate, tau = 0
    if (g == 0)
        for (int j = nb + threadIdx.x; j < b; j += blockDim.x) tau_out[j] = 0;

    // write back R / v into A and the explicit V
    for (int64_t e = threadIdx.x; e < nloc * b; e += blockDim.x) {
        int64_t r = e % nloc, c = e / nloc;
        int64_t gr = rlo + r;
        Cx val = S[r + c * chunk];
        P[gr + c * lda] = val;
        Cx v;
        if (c >= nb) v = czero<Cx>();
        else if (gr < c) v = czero<Cx>();
        else if (gr == c) v = mk<R>(1, 0);
        else v = val;
        Vout[gr + c * ldv] = v;
        if (Vout2) Vout2[gr + c * ldv2] = v;
        S[r + c * chunk] = v;  // keep V for the Gram partial
    }
    __syncthreads();
    // partial Gram matrix V^H V over this slice
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
        int i = e % b, k = e / b;
        Cx acc = czero<Cx>();
        if (i < k) {
            for (int64_t r = 0; r < nloc; ++r) cfmac(acc, S[r + (int64_t)i * chunk], S[r + (int64_t)k * chunk]);
        }
        red_vv[(int64_t)g * b * b + e] = acc;
    }
    if (!grid_sync(gb)) return;
    // the Gram matrix: its entries spread over every warp of the grid
    for (int e = g * nw + wid; e < b * b; e += G * nw) {
        const int i = e % b, k = e / b;
        Cx s = czero<Cx>();
        if (i < k) {
            for (int q = lane; q < G; q += 32) s = cadd(s, ldcg(&red_vv[(int64_t)q * b * b + e]));
            s.x = warp_sum(s.x);
            s.y = warp_sum(s.y);
        }
        if (lane == 0) red_gram[e] = s;
    }
    if (!grid_sync(gb)) return;
    if (g != 0) return;
    // T factor (forward, columnwise): T(j,j) = tau_j, T(0:j, j) = -tau_j T(0:j,0:j) (V^H v_j)(0:j)
    Cx *T = Tout;
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) T[e] = ldcg(&red_gram[e]);   // (V^H V)(i, k), i < k
    __syncthreads();
    for (int j = 0; j < b; ++j) {
        // z = T(0:j, 0:j) * g(0:j) where g = (V^H V)(0:j, j); thread i computes row i
        const R tj = tau_out[j];
        Cx zi = czero<Cx>();
        int i = threadIdx.x;
        if (i < j) {
            for (int k = i; k < j; ++k) {
                Cx tik = (k == i) ? mk<R>(tau_out[i], 0) : T[i + k * b];
                cfma(zi, tik, T[k + j * b]);
            }
        }
        __syncthreads();
        if (i < j) T[i + j * b] = cscale(zi, -tj);
        if (i == j) T[j + j * b] = mk<R>(tj, 0);
        __syncthreads();
    }
    // zero strictly-lower part
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
        int i = e % b, k = e / b;
        if (i > k) T[e] = czero<Cx>();
    }
}

template <typename R>
__global__ void extract_band_kernel(int64_t n, int b, const cplx<R> *__restrict__ A, int64_t lda,
                                    cplx<R> *__restrict__ Bnd, int ldb_band) {
    // Bnd[d + j*ldb_band] = A[j+d, j] for 0 <= d <= b, zero for b < d < ldb_band
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * ldb_band) return;
    int d = (int)(idx % ldb_band);
    int64_t j = idx / ldb_band;
    cplx<R> v = czero<cplx<R>>();
    if (d <= b && j + d < n) v = A[(j + d) + j * lda];
    if (d == 0) v.y = 0;
    Bnd[idx] = v;
}

// Upper triangle of the n x n Hermitian block A from its lower triangle:
// A[i][j] = conj(A[j][i]) for i < j (32 x 32 tiles through shared memory).
template <typename R>
__global__ void mirror_lower_kernel(int64_t n, cplx<R> *__restrict__ A, int64_t lda) {
    __shared__ cplx<R> tile[32][33];
    const int64_t bi = blockIdx.y, bj = blockIdx.x;   // destination tile (rows bi, columns bj), bi <= bj
    if (bi > bj) return;
    const int tx = threadIdx.x, ty = threadIdx.y;     // 32 x 8
    // source: rows of tile bj, columns of tile bi (lower part)
    for (int k = 0; k < 32; k += 8) {
        const int64_t r = bj * 32 + tx, c = bi * 32 + ty + k;
        if (r < n && c < n) tile[ty + k][tx] = A[r + c * lda];
    }
    __syncthreads();
    for (int k = 0; k < 32; k += 8) {
        const int64_t r = bi * 32 + tx, c = bj * 32 + ty + k;   // destination A[r][c], r < c
        if (r < n && c < n && r < c) {
            const cplx<R> v = tile[tx][ty + k];                 // A[c][r]
            A[r + c * lda] = mk<R>(v.x, -v.y);
        }
    }
}

template <typename R>
__global__ void copy_cols_kernel(int64_t rows, int cols, const cplx<R> *__restrict__ src, int64_t lds,
                                 cplx<R> *__restrict__ dst, int64_t ldd) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    int64_t r = idx % rows, c = idx / rows;
    dst[r + c * ldd] = src[r + c * lds];
}

template <typename R>
int panel_qr(bdg_ctx *ctx, cudaStream_t st, int64_t m, int b, cplx<R> *P, int64_t lda, cplx<R> *V,
             int64_t ldv, cplx<R> *V2, int64_t ldv2, cplx<R> *T, R *tau, cplx<R> *red, int G, int64_t chunk) {
    int nb = (int)std::min<int64_t>(b, m);
    size_t smem = (size_t)chunk * b * sizeof(cplx<R>);
    BDG_CUDA_TRY(ctx, cudaMemsetAsync(ctx->barrier, 0, sizeof(GridBarrier), st));
    void *args[] = {&m, &b, &nb, &P, &lda, &V, &ldv, &V2, &ldv2, &T, &red, &tau, &ctx->barrier, &chunk};
    BDG_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((void *)panel_qr_kernel<R>, dim3(G), dim3(256), args, smem, st));
    return BDG_OK;
}

// Stage-1 driver.  A (n x n, lda) is reduced in place; on return:
//   Bnd  (ldband x n)  lower band (diagonal row 0), bandwidth b, extra rows zero;
//   Vst  panels' V stacked (panel p at Vst + voff[p], m_p x b, ld m_p);
//   Tst  panels' T (b x b each, panel p at Tst + p*b*b).
template <typename R>
int stage1_reduce(bdg_ctx *ctx, cudaStream_t st, int64_t n, int b, cplx<R> *A, int64_t lda,
                  cplx<R> *Bnd, int ldband, cplx<R> *Vst, const int64_t *voff, cplx<R> *Tst, R *taust,
                  cplx<R> *VWV, cplx<R> *Ytmp, cplx<R> *Msmall, cplx<R> *Psmall, cplx<R> *red,
                  cplx<R> *splitws, int npanels, const TcPlanes *tcp) {
    using Cx = cplx<R>;
    const Cx one = mk<R>(1, 0), zero = mk<R>(0, 0), mone = mk<R>(-1, 0), mhalf = mk<R>(-0.5, 0);
    // cooperative grid size for the panel kernel
    int maxG = 0;
    for (int p = 0; p < npanels; ++p) {
        int64_t c0 = (int64_t)p * b, r0 = c0 + b, m = n - r0;
        if (m <= 0) break;
        // choose the number of CTAs: at least ~64 rows each, at most one per SM
        int G = (int)std::min<int64_t>(ctx->num_sms, (m + 63) / 64);
        if (G < 1) G = 1;
        int64_t chunk = (m + G - 1) / G;
        size_t smem = (size_t)chunk * b * sizeof(Cx);
        if (smem > (size_t)ctx->smem_optin)
            return bdg_fail(ctx, BDG_EUNSUPPORTED, "panel slice %lld x %d does not fit shared memory",
                            (long long)chunk, b);
        if (smem > 48 * 1024)
            BDG_CUDA_TRY(ctx, cudaFuncSetAttribute(panel_qr_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem));
        int nbpm = 0;
        BDG_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nbpm, panel_qr_kernel<R>, 256, smem));
        if (nbpm < 1) return bdg_fail(ctx, BDG_EUNSUPPORTED, "panel kernel cannot be resident");
        maxG = std::max(maxG, G);
        cplx<R> *Vp = Vst + voff[p];
        cplx<R> *Tp = Tst + (int64_t)p * b * b;
        cplx<R> *P = A + r0 + c0 * lda;
        // V also goes to columns [0,b) and [2b,3b) of VWV (ld = m)
        int rc = panel_qr<R>(ctx, st, m, b, P, lda, Vp, m, VWV, m, Tp, taust + (int64_t)p * b, red, G, chunk);
        if (rc) return rc;
        // copy V into the third block of VWV
        {
            int64_t tot = m * b;
            copy_cols_kernel<R><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(m, b, VWV, m, VWV + 2 * b * m, m);
            BDG_LAUNCH_CHECK(ctx);
        }
        if (m <= 1) continue;
        cplx<R> *A22 = A + r0 + r0 * lda;
        cplx<R> *V = VWV;                 // m x b
        cplx<R> *W = VWV + (int64_t)b * m;  // m x b (X, then W)
        int rc2;
        // Y = A22 V
        if constexpr (sizeof(R) == 4) {
            if (tcp && tcp->S == kExactSlices) {
                // Y = A22^H V (= A22 V: both triangles of A22 are current); X = A22 as stored
                rc2 = xs_slice(ctx, st, m, m, A22, 1, lda, false, false, tcp->big, tcp->ebig);
                if (!rc2) rc2 = xs_slice(ctx, st, m, b, V, 1, m, false, true, tcp->skB, tcp->eB);
                if (!rc2)
                    rc2 = xs_product(ctx, st, m, m, b, tcp->big, tcp->ebig, tcp->skB, tcp->eB, Ytmp, m, 1.f, 0.f,
                                     false);
                if (rc2) return rc2;
            } else if (tcp) {
                // A operand: row i, k = j -> A22[i][j] = conj(column-major storage read along j)
                rc2 = split_planes<float2>(ctx, st, m, m, A22, lda, false, true, tcp->S, tcp->big);
                if (!rc2) rc2 = split_planes<float2>(ctx, st, m, b, V, m, false, false, tcp->S, tcp->skB);
                if (!rc2)
                    rc2 = cgemm_bf16(ctx, st, tcp->S, m, b, m, tcp->big, tcp->skB, Ytmp, m, 1.f, 0.f, tcp->part,
                                     narrow_splits((m + 127) / 128, tcp->num_sms));
                if (rc2) return rc2;
            } else {
                rc2 = gemm<R>(ctx, st, 'N', 'N', m, b, m, one, A22, lda, V, m, zero, Ytmp, m); if (rc2) return rc2;
            }
        } else {
            rc2 = gemm<R>(ctx, st, 'N', 'N', m, b, m, one, A22, lda, V, m, zero, Ytmp, m); if (rc2) return rc2;
        }
        // X = Y T   -> W
        rc2 = gemm<R>(ctx, st, 'N', 'N', m, b, b, one, Ytmp, m, Tp, b, zero, W, m); if (rc2) return rc2;
        // M = V^H X  (split-K over m)
        int splits = (int)std::max<int64_t>(1, std::min<int64_t>(64, m / 256));
        rc2 = gemm_splitk<R>(ctx, st, 'C', 'N', b, b, m, one, V, m, W, m, zero, Msmall, b, splits, splitws);
        if (rc2) return rc2;
        // P = T^H M
        rc2 = gemm<R>(ctx, st, 'C', 'N', b, b, b, one, Tp, b, Msmall, b, zero, Psmall, b); if (rc2) return rc2;
        // W = X - 1/2 V P
        rc2 = gemm<R>(ctx, st, 'N', 'N', m, b, b, mhalf, V, m, Psmall, b, one, W, m); if (rc2) return rc2;
        // A22 -= [V W] [W V]^H
        if constexpr (sizeof(R) == 4) {
            if (tcp && tcp->S == kExactSlices) {
                // exact-slice rank-2b update on the lower triangle: X = [V W]^H,
                // Y = [W V]^H (element (k, c) = conj of row c, column k), then the
                // upper triangle of the next trailing block for its A22 V product
                rc2 = xs_slice(ctx, st, 2 * b, m, VWV, m, 1, true, false, tcp->skA, tcp->eA);
                if (!rc2) rc2 = xs_slice(ctx, st, 2 * b, m, VWV + (int64_t)b * m, m, 1, true, true, tcp->skB, tcp->eB);
                if (!rc2)
                    rc2 = xs_product(ctx, st, 2 * b, m, m, tcp->skA, tcp->eA, tcp->skB, tcp->eB, A22, lda, -1.f, 1.f,
                                     true);
                if (rc2) return rc2;
                if (m > b) {
                    const int64_t mm = m - b;
                    dim3 gr((unsigned)((mm + 31) / 32), (unsigned)((mm + 31) / 32));
                    mirror_lower_kernel<R><<<gr, dim3(32, 8), 0, st>>>(mm, A22 + b + (int64_t)b * lda, lda);
                    BDG_LAUNCH_CHECK(ctx);
                }
            } else if (tcp) {
                rc2 = split_planes<float2>(ctx, st, m, 2 * b, VWV, m, true, false, tcp->S, tcp->skA);
                if (!rc2)
                    rc2 = split_planes<float2>(ctx, st, m, 2 * b, VWV + (int64_t)b * m, m, true, true, tcp->S, tcp->skB);
                if (!rc2) rc2 = cgemm_bf16(ctx, st, tcp->S, m, m, 2 * b, tcp->skA, tcp->skB, A22, lda, -1.f, 1.f, nullptr, 1);
                if (rc2) return rc2;
            } else {
                rc2 = gemm<R>(ctx, st, 'N', 'C', m, m, 2 * b, mone, VWV, m, VWV + (int64_t)b * m, m, one, A22, lda);
                if (rc2) return rc2;
            }
        } else {
            rc2 = gemm<R>(ctx, st, 'N', 'C', m, m, 2 * b, mone, VWV, m, VWV + (int64_t)b * m, m, one, A22, lda);
            if (rc2) return rc2;
        }
    }
    (void)maxG;
    int64_t tot = n * (int64_t)ldband;
    extract_band_kernel<R><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, b, A, lda, Bnd, ldband);
    BDG_LAUNCH_CHECK(ctx);
    return BDG_OK;
}

// Exact-slice back-transformation, two panels per pass.  For panels p-1, p
// (rows r1 = p b .., m1 = n - r1; panel p starts b rows lower)
//   Q_{p-1} Q_p = I - Vg Tg Vg^H,  Vg = [V_{p-1} | (0_b; V_p)],
//   Tg = [[T_{p-1}, -T_{p-1} (V_{p-1}(b:, :)^H V_p) T_p], [0, T_p]]
// (the compact-WY merge), applied as W1^H = Es^H Vg, W2^H = W1^H Tg^H,
// Es -= Vg W2 with K = 2b: half the passes over the E slab of one panel at a
// time (its slicing and its read-modify-write).  An odd first panel goes alone.
static int bt1_exact(bdg_ctx *ctx, cudaStream_t st, int64_t n, int b, int npanels, const float2 *Vst,
                     const int64_t *voff, const float2 *Tst, float2 *E, int64_t lde, int64_t ncols, float2 *W1,
                     float2 *W2, float2 *splitws, const TcPlanes *tcp) {
    const float2 one = mk<float>(1, 0), zero = mk<float>(0, 0), mone = mk<float>(-1, 0);
    const int64_t b2 = 2 * (int64_t)b;
    float2 *Tg = tcp->tagg, *Yb = Tg + 4 * (int64_t)b * b, *Tm = Yb + (int64_t)b * b;
    int p = npanels - 1;
    while (p >= 0) {
        const int64_t r0 = (int64_t)p * b + b, m = n - r0;
        if (m <= 0) { --p; continue; }
        const float2 *V;
        const float2 *T;
        int64_t K, mm, r, ldv;
        int rc;
        if (p >= 1) {
            const int p1 = p - 1;
            const int64_t r1 = (int64_t)p1 * b + b, m1 = n - r1, m2 = m;
            const float2 *V1 = Vst + voff[p1], *V2 = Vst + voff[p];
            const float2 *T1 = Tst + (int64_t)p1 * b * b, *T2 = Tst + (int64_t)p * b * b;
            float2 *Vg = tcp->vagg;
            // Vg = [V1 | (0; V2)], ld m1
            copy_cols_kernel<float><<<(unsigned)((m1 * b + 255) / 256), 256, 0, st>>>(m1, b, V1, m1, Vg, m1);
            BDG_LAUNCH_CHECK(ctx);
            BDG_CUDA_TRY(ctx, cudaMemset2DAsync(Vg + (int64_t)b * m1, (size_t)m1 * 8, 0, (size_t)b * 8, (size_t)b, st));
            copy_cols_kernel<float><<<(unsigned)((m2 * b + 255) / 256), 256, 0, st>>>(m2, b, V2, m2,
                                                                                    Vg + (int64_t)b * m1 + b, m1);
            BDG_LAUNCH_CHECK(ctx);
            // Tg = [[T1, -T1 Y T2], [0, T2]], Y = V1(b:, :)^H V2; ld 2b.  Y is b x b with a
            // contraction of length m2: split over up to 64 CTA layers (one 64 x 64 tile otherwise)
            const int ysplit = (int)std::max<int64_t>(1, std::min<int64_t>(64, m2 / 256));
            rc = gemm_splitk<float>(ctx, st, 'C', 'N', b, b, m2, one, V1 + b, m1, V2, m2, zero, Yb, b, ysplit,
                                    splitws);
            if (!rc) rc = gemm<float>(ctx, st, 'N', 'N', b, b, b, one, T1, b, Yb, b, zero, Tm, b);
            if (!rc) rc = gemm<float>(ctx, st, 'N', 'N', b, b, b, mone, Tm, b, T2, b, zero, Tg + b * b2, b2);
            if (rc) return rc;
            copy_cols_kernel<float><<<(unsigned)(((int64_t)b * b + 255) / 256), 256, 0, st>>>(b, b, T1, b, Tg, b2);
            copy_cols_kernel<float><<<(unsigned)(((int64_t)b * b + 255) / 256), 256, 0, st>>>(b, b, T2, b,
                                                                                            Tg + b + b * b2, b2);
            BDG_LAUNCH_CHECK(ctx);
            BDG_CUDA_TRY(ctx, cudaMemset2DAsync(Tg + b, (size_t)b2 * 8, 0, (size_t)b * 8, (size_t)b, st));
            V = Vg; T = Tg; K = b2; mm = m1; r = r1; ldv = m1;
            p -= 2;
        } else {
            V = Vst + voff[p]; T = Tst + (int64_t)p * b * b; K = b; mm = m; r = r0; ldv = m;
            p -= 1;
        }
        float2 *Es = E + r;
        rc = xs_slice(ctx, st, mm, ncols, Es, 1, lde, false, false, tcp->big, tcp->ebig);
        if (!rc) rc = xs_slice(ctx, st, mm, K, V, 1, ldv, false, true, tcp->skB, tcp->eB);
        if (!rc)
            rc = xs_product(ctx, st, mm, ncols, K, tcp->big, tcp->ebig, tcp->skB, tcp->eB, W1, ncols, 1.f, 0.f,
                            false);
        if (!rc) rc = gemm<float>(ctx, st, 'N', 'C', ncols, K, K, one, W1, ncols, T, K, zero, W2, ncols);
        if (!rc) rc = xs_slice(ctx, st, K, mm, V, ldv, 1, true, false, tcp->skA, tcp->eA);
        if (!rc) rc = xs_slice(ctx, st, K, ncols, W2, ncols, 1, true, true, tcp->skB, tcp->eB);
        if (!rc)
            rc = xs_product(ctx, st, K, mm, ncols, tcp->skA, tcp->eA, tcp->skB, tcp->eB, Es, lde, -1.f, 1.f, false);
        if (rc) return rc;
    }
    return BDG_OK;
}

// Back-transformation by the stage-1 panels: E <- Q_0 Q_1 ... Q_{P-1} E,
// Q_p = I - V_p T_p V_p^H acting on rows r0_p .. n-1 (applied last panel first).
template <typename R>
int stage1_backtransform(bdg_ctx *ctx, cudaStream_t st, int64_t n, int b, int npanels, const cplx<R> *Vst,
                         const int64_t *voff, const cplx<R> *Tst, cplx<R> *E, int64_t lde, int64_t ncols,
                         cplx<R> *W1, cplx<R> *W2, cplx<R> *splitws, const TcPlanes *tcp) {
    using Cx = cplx<R>;
    const Cx one = mk<R>(1, 0), zero = mk<R>(0, 0), mone = mk<R>(-1, 0);
    if constexpr (sizeof(R) == 4) {
        if (tcp && tcp->S == kExactSlices)
            return bt1_exact(ctx, st, n, b, npanels, Vst, voff, Tst, E, lde, ncols, W1, W2, splitws, tcp);
    }
    for (int p = npanels - 1; p >= 0; --p) {
        int64_t r0 = (int64_t)p * b + b, m = n - r0;
        if (m <= 0) continue;
        const Cx *V = Vst + voff[p];
        const Cx *T = Tst + (int64_t)p * b * b;
        Cx *Es = E + r0;
        int rc;
        if constexpr (sizeof(R) == 4) {
            if (tcp && tcp->S == kExactSlices) {
                // W1^H (ncols x b) = Es^H V;  W2^H = W1^H T^H;  Es -= V W2 with
                // X = V^H and Y = W2 (element (k, c) = conj W2^H[c][k])
                rc = xs_slice(ctx, st, m, ncols, Es, 1, lde, false, false, tcp->big, tcp->ebig);
                if (!rc) rc = xs_slice(ctx, st, m, b, V, 1, m, false, true, tcp->skB, tcp->eB);
                if (!rc)
                    rc = xs_product(ctx, st, m, ncols, b, tcp->big, tcp->ebig, tcp->skB, tcp->eB, W1, ncols, 1.f, 0.f,
                                    false);
                if (!rc) rc = gemm<R>(ctx, st, 'N', 'C', ncols, b, b, one, W1, ncols, T, b, zero, W2, ncols);
                if (!rc) rc = xs_slice(ctx, st, b, m, V, m, 1, true, false, tcp->skA, tcp->eA);
                if (!rc) rc = xs_slice(ctx, st, b, ncols, W2, ncols, 1, true, true, tcp->skB, tcp->eB);
                if (!rc)
                    rc = xs_product(ctx, st, b, m, ncols, tcp->skA, tcp->eA, tcp->skB, tcp->eB, Es, lde, -1.f, 1.f,
                                    false);
                if (rc) return rc;
                continue;
            }
            if (tcp) {
                // W1^T (ncols x b) = Es^T conj(V);  W2^T = W1^T T^T;  Es -= V W2
                rc = split_planes<float2>(ctx, st, m, ncols, Es, lde, false, false, tcp->S, tcp->big);
                if (!rc) rc = split_planes<float2>(ctx, st, m, b, V, m, false, true, tcp->S, tcp->skB);
                if (!rc)
                    rc = cgemm_bf16(ctx, st, tcp->S, ncols, b, m, tcp->big, tcp->skB, W1, ncols, 1.f, 0.f, tcp->part,
                                    narrow_splits((ncols + 127) / 128, tcp->num_sms));
                if (rc) return rc;
                rc = gemm<R>(ctx, st, 'N', 'T', ncols, b, b, one, W1, ncols, T, b, zero, W2, ncols);
                if (rc) return rc;
                rc = split_planes<float2>(ctx, st, m, b, V, m, true, false, tcp->S, tcp->skA);
                if (!rc) rc = split_planes<float2>(ctx, st, ncols, b, W2, ncols, true, false, tcp->S, tcp->skB);
                if (!rc) rc = cgemm_bf16(ctx, st, tcp->S, m, ncols, b, tcp->skA, tcp->skB, Es, lde, -1.f, 1.f, nullptr, 1);
                if (rc) return rc;
                continue;
            }
        }
        rc = gemm<R>(ctx, st, 'C', 'N', b, ncols, m, one, V, m, Es, lde, zero, W1, b); if (rc) return rc;
        rc = gemm<R>(ctx, st, 'N', 'N', b, ncols, b, one, T, b, W1, b, zero, W2, b); if (rc) return rc;
        rc = gemm<R>(ctx, st, 'N', 'N', m, ncols, b, mone, V, m, W2, b, one, Es, lde); if (rc) return rc;
    }
    return BDG_OK;
}

template int stage1_reduce<float>(bdg_ctx *, cudaStream_t, int64_t, int, float2 *, int64_t, float2 *, int,
                                  float2 *, const int64_t *, float2 *, float *, float2 *, float2 *, float2 *,
                                  float2 *, float2 *, float2 *, int, const TcPlanes *);
template int stage1_reduce<double>(bdg_ctx *, cudaStream_t, int64_t, int, double2 *, int64_t, double2 *, int,
                                   double2 *, const int64_t *, double2 *, double *, double2 *, double2 *,
                                   double2 *, double2 *, double2 *, double2 *, int, const TcPlanes *);
template int stage1_backtransform<float>(bdg_ctx *, cudaStream_t, int64_t, int, int, const float2 *,
                                         const int64_t *, const float2 *, float2 *, int64_t, int64_t, float2 *,
                                         float2 *, float2 *, const TcPlanes *);
template int stage1_backtransform<double>(bdg_ctx *, cudaStream_t, int64_t, int, int, const double2 *,
                                          const int64_t *, const double2 *, double2 *, int64_t, int64_t,
                                          double2 *, double2 *, double2 *, const TcPlanes *);

}  // namespace bdg
