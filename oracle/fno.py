"""FP64 reference of the Fourier neural operator -- TEST INFRASTRUCTURE ONLY.

Same network as the library's learned SCF guess (lift, Fourier layers with a
spectral convolution truncated to the modes |k| <= m-1 per dimension, GELU
between layers, projection), written with numpy's FFT and an explicit mode
mask instead of direct DFT sums, in float64.  Gradients for the parity tests
are central finite differences of this forward.

Parameter vector layout (as the library's): P[cin][W], p[W]; per layer
W[W][W], b[W], R[M][W][W] complex as (re, im) pairs; Q[W][cout], q[cout];
M = (2m-1)^3 modes ordered with kx slowest and kz fastest, each in
-(m-1) .. m-1.
"""
from __future__ import annotations

import math

import numpy as np


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.asarray(x, dtype=np.float32).copy()
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def sizes(g, width, modes, layers, cin, cout):
    km = 2 * modes - 1
    M = km ** 3
    per_layer = width * width + width + M * width * width * 2
    return cin * width + width + layers * per_layer + width * cout + cout, M


def unpack(cfg, params):
    g, W, m, L, cin, cout = (cfg[k] for k in ("g", "width", "modes", "layers", "cin", "cout"))
    p = np.asarray(params, dtype=np.float64)
    if cfg.get("bf16_weights"):
        p = bf16_round(np.asarray(params, dtype=np.float32))
    km = 2 * m - 1
    M = km ** 3
    o = 0

    def take(n):
        nonlocal o
        v = p[o:o + n]
        o += n
        return v
    P = take(cin * W).reshape(cin, W)
    pb = take(W)
    layers = []
    for _ in range(L):
        Wl = take(W * W).reshape(W, W)
        bl = take(W)
        R = take(M * W * W * 2).reshape(M, W, W, 2)
        layers.append((Wl, bl, R[..., 0] + 1j * R[..., 1]))
    Q = take(W * cout).reshape(W, cout)
    qb = take(cout)
    assert o == p.size
    return P, pb, layers, Q, qb


def mode_indices(g, m):
    """Array indices (mod g) of the kept modes, kx slowest, kz fastest."""
    ks = np.arange(-(m - 1), m)
    kx, ky, kz = np.meshgrid(ks, ks, ks, indexing="ij")
    return kx.ravel() % g, ky.ravel() % g, kz.ravel() % g


def gelu(x):
    from scipy.special import erf
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def forward(cfg, params, inp):
    """inp (B, g^3, cin) -> out (B, g^3, cout), float64."""
    g, m, L = cfg["g"], cfg["modes"], cfg["layers"]
    P, pb, layers, Q, qb = unpack(cfg, params)
    B = inp.shape[0]
    x = np.asarray(inp, dtype=np.float64)
    h = x @ P + pb                                   # (B, X, W)
    ix, iy, iz = mode_indices(g, m)
    for l, (Wl, bl, R) in enumerate(layers):
        W = h.shape[-1]
        hg = h.reshape(B, g, g, g, W)
        F = np.fft.fftn(hg, axes=(1, 2, 3))[:, ix, iy, iz, :]      # (B, M, W): sum_x h e^{-i k.x}
        Gm = np.einsum("bkc,kco->bko", F, R)
        full = np.zeros((B, g, g, g, W), dtype=np.complex128)
        full[:, ix, iy, iz, :] = Gm
        spec = np.real(np.fft.ifftn(full, axes=(1, 2, 3))).reshape(B, g ** 3, W)   # (1/X) sum_k G e^{+i k.x}
        z = spec + h @ Wl + bl
        h = gelu(z) if l + 1 < L else z
    return h @ Q + qb


def mse(y, t):
    return float(np.mean((y - t) ** 2))


def fd_gradient(cfg, params, inp, target, idx, eps=1e-6):
    """Central finite differences of mse(forward(params), target) at the parameter indices idx."""
    p = np.asarray(params, dtype=np.float64).copy()
    out = []
    for i in idx:
        v = p[i]
        p[i] = v + eps
        lp = mse(forward(cfg, p, inp), target)
        p[i] = v - eps
        lm = mse(forward(cfg, p, inp), target)
        p[i] = v
        out.append((lp - lm) / (2 * eps))
    return np.array(out)
