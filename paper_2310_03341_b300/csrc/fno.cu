// Fourier neural operator for the SCF initial guess: forward, backward, loss
// and Adam kernels.
//
// The network maps per-site input channels (mu, Delta0, |ansatz|, cos theta,
// sin theta) on a periodic g^3 grid (site x = (ix g + iy) g + iz, the site
// order of the BdG builder) to (U, Re Delta, Im Delta):
//   h_0   = P in + p                                      (lift, cin -> W)
//   z_l   = W_l h_l + b_l + Re IDFT( R_l . DFT(h_l) )     (l = 0 .. L-1)
//   h_l+1 = GELU(z_l) for l < L-1,  h_L = z_{L-1}
//   out   = Q h_L + q                                     (projection, W -> cout)
// DFT(h)[k] = sum_x h[x] e^{-2 pi i k.x / g} is kept only on the modes
// k in [-(m-1), m-1]^3; R_l[k] is a complex W x W matrix per kept mode;
// IDFT(G)[x] = (1/g^3) sum_k G[k] e^{+2 pi i k.x / g}.  The transforms are
// direct sums over the kept modes (exact twiddles from a table of the g-th
// roots of unity), so nothing depends on an FFT library.
//
// Weights are FP32 in memory; with bf16_weights the forward and backward use
// their bf16-rounded values (BF16 weights, FP32 accumulation).
//
// Parameter layout (floats): P[cin][W], p[W]; per layer W_l[W][W], b_l[W],
// R_l[M][W][W] complex (re, im); Q[W][cout], q[cout].  M = (2m-1)^3.
// Activation cache per layer l (floats, batch B, X = g^3): h_l [B][X][W],
// z_l [B][X][W], F_l [B][M][W] complex; then h_L [B][X][W].
#include <math.h>

#include <cuda_bf16.h>

#include <algorithm>

#include "internal.h"

namespace bdg {
namespace fno {

struct Dims {
    int g, W, m, L, cin, cout, bf16;
    int64_t X, M;
};

static Dims dims_of(const bdg_fno_config *c) {
    Dims d;
    d.g = c->g; d.W = c->width; d.m = c->modes; d.L = c->layers; d.cin = c->cin; d.cout = c->cout;
    d.bf16 = c->bf16_weights;
    d.X = (int64_t)d.g * d.g * d.g;
    const int64_t km = 2 * d.m - 1;
    d.M = km * km * km;
    return d;
}

// offsets into the parameter vector
struct POff {
    int64_t P, p, Q, q, total;
    int64_t Wl(int l) const { return layer0 + l * per_layer; }
    int64_t bl(int l) const { return Wl(l) + ww; }
    int64_t Rl(int l) const { return bl(l) + w; }
    int64_t layer0, per_layer, ww, w;
};

static POff poff(const Dims &d) {
    POff o;
    o.P = 0;
    o.p = o.P + (int64_t)d.cin * d.W;
    o.layer0 = o.p + d.W;
    o.ww = (int64_t)d.W * d.W;
    o.w = d.W;
    o.per_layer = o.ww + o.w + d.M * o.ww * 2;
    o.Q = o.layer0 + d.L * o.per_layer;
    o.q = o.Q + (int64_t)d.W * d.cout;
    o.total = o.q + d.cout;
    return o;
}

// cache offsets (floats)
struct COff {
    int64_t h(int l) const { return l * per_layer; }
    int64_t z(int l) const { return h(l) + act; }
    int64_t F(int l) const { return z(l) + act; }
    int64_t hL() const { return L * per_layer; }
    int64_t act, spec, per_layer, total;
    int L;
};

static COff coff(const Dims &d, int B) {
    COff o;
    o.L = d.L;
    o.act = (int64_t)B * d.X * d.W;
    o.spec = (int64_t)B * d.M * d.W * 2;
    o.per_layer = 2 * o.act + o.spec;
    o.total = d.L * o.per_layer + o.act;
    return o;
}

__device__ __forceinline__ float wval(const float *p, int64_t i, int bf16) {
    const float v = p[i];
    return bf16 ? __bfloat162float(__float2bfloat16_rn(v)) : v;
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
    const float cdf = 0.5f * (1.f + erff(x * 0.70710678118654752f));
    const float pdf = 0.39894228040143268f * expf(-0.5f * x * x);
    return cdf + x * pdf;
}

// mode index -> (kx, ky, kz) in [-(m-1), m-1]; site index -> (ix, iy, iz)
__device__ __forceinline__ void mode_of(int64_t k, int m, int &kx, int &ky, int &kz) {
    const int km = 2 * m - 1;
    kz = (int)(k % km) - (m - 1);
    ky = (int)((k / km) % km) - (m - 1);
    kx = (int)(k / ((int64_t)km * km)) - (m - 1);
}
// e^{-2 pi i p / g} for the phase index p = k.x mod g, from the table (cos, sin) of 2 pi p / g
__device__ __forceinline__ int phase_index(int kx, int ky, int kz, int64_t x, int g) {
    const int iz = (int)(x % g), iy = (int)((x / g) % g), ix = (int)(x / ((int64_t)g * g));
    int p = (kx * ix + ky * iy + kz * iz) % g;
    return p < 0 ? p + g : p;
}

__global__ void twiddle_kernel(int g, float2 *tw) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g) return;
    double s, c;
    sincospi(2.0 * (double)p / (double)g, &s, &c);
    tw[p] = make_float2((float)c, (float)s);
}

// out[b][x][o] = sum_c in[b][x][c] Wt[c][o] + bias[o]   (pointwise linear)
__global__ void pointwise_kernel(int64_t BX, int cin, int cout, const float *__restrict__ in,
                                 const float *__restrict__ prm, int64_t wo, int64_t bo, int bf16,
                                 float *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= BX * cout) return;
    const int64_t bx = i / cout;
    const int o = (int)(i % cout);
    float acc = wval(prm, bo + o, bf16);
    for (int c = 0; c < cin; ++c) acc = fmaf(in[bx * cin + c], wval(prm, wo + (int64_t)c * cout + o, bf16), acc);
    out[i] = acc;
}

// F[b][k][c] = sum_x h[b][x][c] e^{-i theta(k, x)}
__global__ void dft_fwd_kernel(int B, int g, int m, int64_t X, int64_t M, int W, const float *__restrict__ h,
                               const float2 *__restrict__ tw, float2 *__restrict__ F) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)B * M * W) return;
    const int c = (int)(i % W);
    const int64_t k = (i / W) % M;
    const int b = (int)(i / ((int64_t)W * M));
    int kx, ky, kz;
    mode_of(k, m, kx, ky, kz);
    float re = 0.f, im = 0.f;
    const float *hb = h + (int64_t)b * X * W + c;
    for (int64_t x = 0; x < X; ++x) {
        const float2 t = tw[phase_index(kx, ky, kz, x, g)];
        const float v = hb[x * W];
        re = fmaf(v, t.x, re);
        im = fmaf(-v, t.y, im);
    }
    F[i] = make_float2(re, im);
}

// G[b][k][o] = sum_c R[k][c][o] F[b][k][c]
__global__ void mode_mix_kernel(int B, int64_t M, int W, const float2 *__restrict__ F, const float *__restrict__ prm,
                                int64_t ro, int bf16, float2 *__restrict__ G) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)B * M * W) return;
    const int o = (int)(i % W);
    const int64_t k = (i / W) % M;
    const int b = (int)(i / ((int64_t)W * M));
    const float2 *Fb = F + ((int64_t)b * M + k) * W;
    float re = 0.f, im = 0.f;
    for (int c = 0; c < W; ++c) {
        const int64_t r = ro + ((k * W + c) * W + o) * 2;
        const float rr = wval(prm, r, bf16), ri = wval(prm, r + 1, bf16);
        const float2 f = Fb[c];
        re += rr * f.x - ri * f.y;
        im += rr * f.y + ri * f.x;
    }
    G[i] = make_float2(re, im);
}

// z[b][x][o] = (1/X) Re sum_k G[b][k][o] e^{+i theta} + sum_c W[c][o] h[b][x][c] + bias[o];
// hn = GELU(z) (or z for the last layer)
__global__ void layer_out_kernel(int B, int g, int m, int64_t X, int64_t M, int W, const float2 *__restrict__ G,
                                 const float *__restrict__ h, const float *__restrict__ prm, int64_t wo, int64_t bo,
                                 int bf16, const float2 *__restrict__ tw, int act, float *__restrict__ z,
                                 float *__restrict__ hn) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)B * X * W) return;
    const int o = (int)(i % W);
    const int64_t x = (i / W) % X;
    const int b = (int)(i / ((int64_t)W * X));
    float s = 0.f;
    const float2 *Gb = G + (int64_t)b * M * W + o;
    for (int64_t k = 0; k < M; ++k) {
        int kx, ky, kz;
        mode_of(k, m, kx, ky, kz);
        const float2 t = tw[phase_index(kx, ky, kz, x, g)];
        const float2 gk = Gb[k * W];
        s += gk.x * t.x - gk.y * t.y;   // Re(G e^{+i theta})
    }
    float acc = s / (float)X + wval(prm, bo + o, bf16);
    const float *hx = h + ((int64_t)b * X + x) * W;
    for (int c = 0; c < W; ++c) acc = fmaf(hx[c], wval(prm, wo + (int64_t)c * W + o, bf16), acc);
    z[i] = acc;
    hn[i] = act ? gelu(acc) : acc;
}

// ---------------------------------------------------------------- backward
// dW[c][o] += sum_{b,x} in[b][x][c] d[b][x][o];  dbias[o] += sum d[b][x][o]
__global__ void wgrad_kernel(int64_t BX, int cin, int cout, const float *__restrict__ in, const float *__restrict__ d,
                             float *__restrict__ grad, int64_t wo, int64_t bo) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)(cin + 1) * cout) return;
    const int c = (int)(i / cout), o = (int)(i % cout);
    float acc = 0.f;
    if (c < cin) {
        for (int64_t bx = 0; bx < BX; ++bx) acc = fmaf(in[bx * cin + c], d[bx * cout + o], acc);
        grad[wo + (int64_t)c * cout + o] += acc;
    } else {
        for (int64_t bx = 0; bx < BX; ++bx) acc += d[bx * cout + o];
        grad[bo + o] += acc;
    }
}

// din[b][x][c] = sum_o W[c][o] d[b][x][o]   (accumulate if add)
__global__ void dinput_kernel(int64_t BX, int cin, int cout, const float *__restrict__ d, const float *__restrict__ prm,
                              int64_t wo, int bf16, float *__restrict__ din, int add) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= BX * cin) return;
    const int64_t bx = i / cin;
    const int c = (int)(i % cin);
    float acc = 0.f;
    for (int o = 0; o < cout; ++o) acc = fmaf(wval(prm, wo + (int64_t)c * cout + o, bf16), d[bx * cout + o], acc);
    din[i] = add ? din[i] + acc : acc;
}

// dz = dh * GELU'(z)  (in place on dh), or a copy for the last layer
__global__ void gelu_back_kernel(int64_t n, const float *__restrict__ z, float *__restrict__ dh) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    dh[i] *= gelu_grad(z[i]);
}

// dG[b][k][o] = (1/X) sum_x dz[b][x][o] e^{-i theta}
__global__ void dft_adj_kernel(int B, int g, int m, int64_t X, int64_t M, int W, const float *__restrict__ dz,
                               const float2 *__restrict__ tw, float2 *__restrict__ dG) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)B * M * W) return;
    const int o = (int)(i % W);
    const int64_t k = (i / W) % M;
    const int b = (int)(i / ((int64_t)W * M));
    int kx, ky, kz;
    mode_of(k, m, kx, ky, kz);
    float re = 0.f, im = 0.f;
    const float *db = dz + (int64_t)b * X * W + o;
    for (int64_t x = 0; x < X; ++x) {
        const float2 t = tw[phase_index(kx, ky, kz, x, g)];
        const float v = db[x * W];
        re = fmaf(v, t.x, re);
        im = fmaf(-v, t.y, im);
    }
    dG[i] = make_float2(re / (float)X, im / (float)X);
}

// dR[k][c][o] += sum_b dG[b][k][o] conj(F[b][k][c])
__global__ void rgrad_kernel(int B, int64_t M, int W, const float2 *__restrict__ dG, const float2 *__restrict__ F,
                             float *__restrict__ grad, int64_t ro) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M * W * W) return;
    const int o = (int)(i % W), c = (int)((i / W) % W);
    const int64_t k = i / ((int64_t)W * W);
    float re = 0.f, im = 0.f;
    for (int b = 0; b < B; ++b) {
        const float2 d = dG[((int64_t)b * M + k) * W + o];
        const float2 f = F[((int64_t)b * M + k) * W + c];
        re += d.x * f.x + d.y * f.y;
        im += d.y * f.x - d.x * f.y;
    }
    grad[ro + i * 2] += re;
    grad[ro + i * 2 + 1] += im;
}

// dF[b][k][c] = sum_o conj(R[k][c][o]) dG[b][k][o]
__global__ void fgrad_kernel(int B, int64_t M, int W, const float2 *__restrict__ dG, const float *__restrict__ prm,
                             int64_t ro, int bf16, float2 *__restrict__ dF) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)B * M * W) return;
    const int c = (int)(i % W);
    const int64_t k = (i / W) % M;
    const int b = (int)(i / ((int64_t)W * M));
    float re = 0.f, im = 0.f;
    for (int o = 0; o < W; ++o) {
        const int64_t r = ro + ((k * W + c) * W + o) * 2;
        const float rr = wval(prm, r, bf16), ri = wval(prm, r + 1, bf16);
        const float2 d = dG[((int64_t)b * M + k) * W + o];
        re += rr * d.x + ri * d.y;
        im += rr * d.y - ri * d.x;
    }
    dF[i] = make_float2(re, im);
}

// dh[b][x][c] += Re sum_k dF[b][k][c] e^{+i theta}
__global__ void dft_back_kernel(int B, int g, int m, int64_t X, int64_t M, int W, const float2 *__restrict__ dF,
                                const float2 *__restrict__ tw, float *__restrict__ dh) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)B * X * W) return;
    const int c = (int)(i % W);
    const int64_t x = (i / W) % X;
    const int b = (int)(i / ((int64_t)W * X));
    float s = 0.f;
    const float2 *Fb = dF + (int64_t)b * M * W + c;
    for (int64_t k = 0; k < M; ++k) {
        int kx, ky, kz;
        mode_of(k, m, kx, ky, kz);
        const float2 t = tw[phase_index(kx, ky, kz, x, g)];
        const float2 f = Fb[k * W];
        s += f.x * t.x - f.y * t.y;
    }
    dh[i] += s;
}

// loss = sum (y - t)^2 / n ; dy = 2 (y - t) / n   (per-block partial sums, then one block)
__global__ void mse_kernel(int64_t n, const float *__restrict__ y, const float *__restrict__ t, float *__restrict__ dy,
                           double *__restrict__ partial) {
    __shared__ double s[256];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float e = y[i] - t[i];
        dy[i] = 2.f * e / (float)n;
        acc += (double)e * e;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = s[0];
}
__global__ void sum_kernel(int nb, int64_t n, const double *__restrict__ partial, float *__restrict__ loss) {
    __shared__ double s[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partial[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = (float)(s[0] / (double)n);
}

// Adam (Kingma & Ba, "Adam: A Method for Stochastic Optimization", ICLR 2015), bias-corrected
__global__ void adam_kernel(int64_t n, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m1,
                            float *__restrict__ m2, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float v = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = v;
    p[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
}

static unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

static int check_cfg(bdg_ctx *ctx, const bdg_fno_config *c, int B) {
    if (!c || c->g < 2 || c->width < 1 || c->modes < 1 || 2 * c->modes - 1 > c->g || c->layers < 1 || c->cin < 1 ||
        c->cout < 1 || B < 1)
        return bdg_fail(ctx, BDG_EINVAL, "fno: bad configuration (need g >= 2m-1, positive sizes)");
    return BDG_OK;
}

}  // namespace fno
}  // namespace bdg

using namespace bdg;
using namespace bdg::fno;

extern "C" {

int bdg_fno_sizes(const bdg_fno_config *cfg, int batch, int64_t *nparams, int64_t *ncache) {
    if (!cfg || batch < 1) return BDG_EINVAL;
    const Dims d = dims_of(cfg);
    if (nparams) *nparams = poff(d).total;
    if (ncache) *ncache = coff(d, batch).total;
    return BDG_OK;
}

int bdg_fno_forward(bdg_ctx *ctx, const bdg_fno_config *cfg, int batch, const float *params, const float *in,
                    float *out, float *cache, cudaStream_t st) {
    if (!ctx) return BDG_EINVAL;
    int rc = check_cfg(ctx, cfg, batch);
    if (rc) return rc;
    if (!params || !in || !out || !cache) return bdg_fail(ctx, BDG_EINVAL, "bdg_fno_forward: null pointer");
    cudaSetDevice(ctx->device);
    const Dims d = dims_of(cfg);
    const POff po = poff(d);
    const COff co = coff(d, batch);
    const int B = batch;
    const int64_t BX = (int64_t)B * d.X;
    // twiddles and the spectral scratch G live in the context arena
    ws_reset(ctx);
    rc = ws_reserve(ctx, align_up((size_t)d.g * 8) + align_up((size_t)co.spec * 4) + 4096);
    if (rc) return rc;
    float2 *tw = (float2 *)ws_take(ctx, (size_t)d.g * 8);
    float2 *G = (float2 *)ws_take(ctx, (size_t)co.spec * 4);
    twiddle_kernel<<<1, 256, 0, st>>>(d.g, tw);
    BDG_LAUNCH_CHECK(ctx);
    pointwise_kernel<<<nblk(BX * d.W), 256, 0, st>>>(BX, d.cin, d.W, in, params, po.P, po.p, d.bf16, cache + co.h(0));
    BDG_LAUNCH_CHECK(ctx);
    for (int l = 0; l < d.L; ++l) {
        const float *h = cache + co.h(l);
        float2 *F = (float2 *)(cache + co.F(l));
        dft_fwd_kernel<<<nblk((int64_t)B * d.M * d.W), 256, 0, st>>>(B, d.g, d.m, d.X, d.M, d.W, h, tw, F);
        mode_mix_kernel<<<nblk((int64_t)B * d.M * d.W), 256, 0, st>>>(B, d.M, d.W, F, params, po.Rl(l), d.bf16, G);
        float *hn = (l + 1 < d.L) ? cache + co.h(l + 1) : cache + co.hL();
        layer_out_kernel<<<nblk(BX * d.W), 256, 0, st>>>(B, d.g, d.m, d.X, d.M, d.W, G, h, params, po.Wl(l),
                                                        po.bl(l), d.bf16, tw, l + 1 < d.L, cache + co.z(l), hn);
        BDG_LAUNCH_CHECK(ctx);
    }
    pointwise_kernel<<<nblk(BX * d.cout), 256, 0, st>>>(BX, d.W, d.cout, cache + co.hL(), params, po.Q, po.q, d.bf16,
                                                       out);
    BDG_LAUNCH_CHECK(ctx);
    return BDG_OK;
}

int bdg_fno_backward(bdg_ctx *ctx, const bdg_fno_config *cfg, int batch, const float *params, const float *in,
                     const float *cache, const float *dout, float *grad, cudaStream_t st) {
    if (!ctx) return BDG_EINVAL;
    int rc = check_cfg(ctx, cfg, batch);
    if (rc) return rc;
    if (!params || !in || !cache || !dout || !grad) return bdg_fail(ctx, BDG_EINVAL, "bdg_fno_backward: null pointer");
    cudaSetDevice(ctx->device);
    const Dims d = dims_of(cfg);
    const POff po = poff(d);
    const COff co = coff(d, batch);
    const int B = batch;
    const int64_t BX = (int64_t)B * d.X;
    ws_reset(ctx);
    rc = ws_reserve(ctx, align_up((size_t)d.g * 8) + 2 * align_up((size_t)co.spec * 4) + 2 * align_up((size_t)co.act * 4) +
                             4096);
    if (rc) return rc;
    float2 *tw = (float2 *)ws_take(ctx, (size_t)d.g * 8);
    float2 *dG = (float2 *)ws_take(ctx, (size_t)co.spec * 4);
    float2 *dF = (float2 *)ws_take(ctx, (size_t)co.spec * 4);
    float *dh = (float *)ws_take(ctx, (size_t)co.act * 4);    // gradient w.r.t. the current h
    float *dh2 = (float *)ws_take(ctx, (size_t)co.act * 4);   // gradient w.r.t. the previous h
    twiddle_kernel<<<1, 256, 0, st>>>(d.g, tw);
    BDG_CUDA_TRY(ctx, cudaMemsetAsync(grad, 0, (size_t)po.total * 4, st));
    // projection
    wgrad_kernel<<<nblk((int64_t)(d.W + 1) * d.cout), 256, 0, st>>>(BX, d.W, d.cout, cache + co.hL(), dout, grad, po.Q,
                                                                    po.q);
    dinput_kernel<<<nblk(BX * d.W), 256, 0, st>>>(BX, d.W, d.cout, dout, params, po.Q, d.bf16, dh, 0);
    BDG_LAUNCH_CHECK(ctx);
    for (int l = d.L - 1; l >= 0; --l) {
        // dh holds dL/dh_{l+1}; turn it into dz_l
        if (l + 1 < d.L) gelu_back_kernel<<<nblk(BX * d.W), 256, 0, st>>>(BX * d.W, cache + co.z(l), dh);
        const float *h = cache + co.h(l);
        const float2 *F = (const float2 *)(cache + co.F(l));
        wgrad_kernel<<<nblk((int64_t)(d.W + 1) * d.W), 256, 0, st>>>(BX, d.W, d.W, h, dh, grad, po.Wl(l), po.bl(l));
        dft_adj_kernel<<<nblk((int64_t)B * d.M * d.W), 256, 0, st>>>(B, d.g, d.m, d.X, d.M, d.W, dh, tw, dG);
        rgrad_kernel<<<nblk(d.M * d.W * d.W), 256, 0, st>>>(B, d.M, d.W, dG, F, grad, po.Rl(l));
        fgrad_kernel<<<nblk((int64_t)B * d.M * d.W), 256, 0, st>>>(B, d.M, d.W, dG, params, po.Rl(l), d.bf16, dF);
        dinput_kernel<<<nblk(BX * d.W), 256, 0, st>>>(BX, d.W, d.W, dh, params, po.Wl(l), d.bf16, dh2, 0);
        dft_back_kernel<<<nblk(BX * d.W), 256, 0, st>>>(B, d.g, d.m, d.X, d.M, d.W, dF, tw, dh2);
        BDG_LAUNCH_CHECK(ctx);
        float *t = dh; dh = dh2; dh2 = t;
    }
    // lift
    wgrad_kernel<<<nblk((int64_t)(d.cin + 1) * d.W), 256, 0, st>>>(BX, d.cin, d.W, in, dh, grad, po.P, po.p);
    BDG_LAUNCH_CHECK(ctx);
    return BDG_OK;
}

int bdg_fno_mse(bdg_ctx *ctx, int64_t n, const float *y, const float *target, float *dy, float *loss_out,
                cudaStream_t st) {
    if (!ctx) return BDG_EINVAL;
    if (n < 1 || !y || !target || !dy || !loss_out) return bdg_fail(ctx, BDG_EINVAL, "bdg_fno_mse: bad arguments");
    cudaSetDevice(ctx->device);
    ws_reset(ctx);
    const int nb = (int)std::min<int64_t>(1024, (n + 255) / 256);
    int rc = ws_reserve(ctx, align_up((size_t)nb * 8) + 4096);
    if (rc) return rc;
    double *part = (double *)ws_take(ctx, (size_t)nb * 8);
    mse_kernel<<<nb, 256, 0, st>>>(n, y, target, dy, part);
    sum_kernel<<<1, 256, 0, st>>>(nb, n, part, loss_out);
    BDG_LAUNCH_CHECK(ctx);
    return BDG_OK;
}

int bdg_fno_adam(bdg_ctx *ctx, int64_t n, float *params, const float *grad, float *m1, float *m2, float lr,
                 float beta1, float beta2, float eps, int step, cudaStream_t st) {
    if (!ctx) return BDG_EINVAL;
    if (n < 1 || !params || !grad || !m1 || !m2 || step < 1 || !(lr > 0.f) || beta1 < 0.f || beta1 >= 1.f ||
        beta2 < 0.f || beta2 >= 1.f)
        return bdg_fail(ctx, BDG_EINVAL, "bdg_fno_adam: bad arguments");
    cudaSetDevice(ctx->device);
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    adam_kernel<<<nblk(n), 256, 0, st>>>(n, params, grad, m1, m2, lr, beta1, beta2, eps, c1, c2);
    BDG_LAUNCH_CHECK(ctx);
    return BDG_OK;
}

}  // extern "C"
