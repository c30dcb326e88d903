"""Pins of the FP64 FNO reference (oracle/fno.py) against what the
mathematics fixes, independent of its own code paths."""
import numpy as np
import pytest

from oracle import fno


def _cfg(**kw):
    c = dict(g=6, width=4, modes=2, layers=2, cin=3, cout=2, bf16_weights=0)
    c.update(kw)
    return c


def _params(cfg, seed, scale=0.3):
    n, _ = fno.sizes(cfg["g"], cfg["width"], cfg["modes"], cfg["layers"], cfg["cin"], cfg["cout"])
    return np.random.default_rng(seed).standard_normal(n) * scale


def test_spectral_layer_with_identity_modes_is_a_low_pass_filter():
    """One layer, W = 0, b = 0, R = I on every kept mode, identity lift and
    projection: the output is the input with every Fourier mode outside
    |k| <= m-1 removed (computed here by an explicit DFT sum)."""
    g, m, w = 6, 2, 1
    cfg = _cfg(g=g, width=w, modes=m, layers=1, cin=1, cout=1)
    n, M = fno.sizes(g, w, m, 1, 1, 1)
    p = np.zeros(n)
    p[0] = 1.0                       # P = 1
    o = 1 + 1                        # after P and p
    o += 1 + 1                       # W_0 = 0, b_0 = 0
    R = np.zeros((M, 1, 1, 2)); R[..., 0] = 1.0
    p[o:o + M * 2] = R.ravel(); o += M * 2
    p[o] = 1.0                       # Q = 1
    x = np.random.default_rng(1).standard_normal((1, g ** 3, 1))
    y = fno.forward(cfg, p, x)[0, :, 0]
    idx = np.arange(g)
    ix, iy, iz = np.meshgrid(idx, idx, idx, indexing="ij")
    ref = np.zeros(g ** 3)
    xv = x[0, :, 0]
    ks = range(-(m - 1), m)
    for kx in ks:
        for ky in ks:
            for kz in ks:
                ph = np.exp(2j * np.pi * (kx * ix + ky * iy + kz * iz).ravel() / g)
                ref += np.real(ph * np.sum(xv * np.conj(ph))) / g ** 3
    assert np.max(np.abs(y - ref)) < 1e-12


def test_zero_spectral_weights_reduce_to_a_pointwise_mlp():
    cfg = _cfg(layers=2)
    p = _params(cfg, 3)
    g, W, m = cfg["g"], cfg["width"], cfg["modes"]
    _, M = fno.sizes(g, W, m, 2, cfg["cin"], cfg["cout"])
    o = cfg["cin"] * W + W
    per = W * W + W + M * W * W * 2
    for l in range(2):
        p[o + W * W + W:o + per] = 0.0
        o += per
    x = np.random.default_rng(4).standard_normal((2, g ** 3, cfg["cin"]))
    P, pb, layers, Q, qb = fno.unpack(cfg, p)
    from scipy.special import erf
    gelu = lambda z: 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))   # GELU from its definition
    h = x @ P + pb
    h = gelu(h @ layers[0][0] + layers[0][1])
    h = h @ layers[1][0] + layers[1][1]
    ref = h @ Q + qb
    assert np.max(np.abs(fno.forward(cfg, p, x) - ref)) < 1e-12


def test_translation_equivariance():
    """Periodic shifts of the input shift the output (every layer commutes with translations)."""
    cfg = _cfg()
    p = _params(cfg, 5)
    g = cfg["g"]
    x = np.random.default_rng(6).standard_normal((1, g ** 3, cfg["cin"]))
    y = fno.forward(cfg, p, x)
    xs = np.roll(x.reshape(1, g, g, g, -1), (1, 2, 3), axis=(1, 2, 3)).reshape(1, g ** 3, -1)
    ys = np.roll(y.reshape(1, g, g, g, -1), (1, 2, 3), axis=(1, 2, 3)).reshape(1, g ** 3, -1)
    assert np.max(np.abs(fno.forward(cfg, p, xs) - ys)) < 1e-12


def test_bf16_rounding_matches_the_definition():
    v = np.array([1.0, 1.00390625, 1.005859375, -3.14159265, 65504.0, 1e-30], dtype=np.float32)
    r = fno.bf16_round(v)
    # bf16 keeps 8 significant bits: the rounded value is within half an ulp (2^-8 relative)
    assert np.all(np.abs(r - v.astype(np.float64)) <= np.abs(v) * 2.0 ** -8 + 1e-45)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0078125   # ties to even; 1.0059 rounds up


def test_finite_difference_gradient_of_a_linear_case():
    """With one layer (no GELU) the output is linear in the projection weights:
    the finite difference equals the analytic derivative of the MSE."""
    cfg = _cfg(layers=1)
    p = _params(cfg, 7)
    g = cfg["g"]
    x = np.random.default_rng(8).standard_normal((1, g ** 3, cfg["cin"]))
    t = np.random.default_rng(9).standard_normal((1, g ** 3, cfg["cout"]))
    y = fno.forward(cfg, p, x)
    n, _ = fno.sizes(g, cfg["width"], cfg["modes"], 1, cfg["cin"], cfg["cout"])
    qb0 = n - cfg["cout"]
    analytic = 2.0 * np.mean((y - t), axis=(0, 1)) / cfg["cout"]   # d mse / d q_o
    fd = fno.fd_gradient(cfg, p, x, t, [qb0, qb0 + 1])
    assert np.max(np.abs(fd - analytic)) < 1e-8


def _single_mode_net(g, m, mode, value):
    """One layer, width 1, identity lift/projection, W = b = 0, R = value on one mode, zero elsewhere."""
    cfg = _cfg(g=g, width=1, modes=m, layers=1, cin=1, cout=1)
    n, M = fno.sizes(g, 1, m, 1, 1, 1)
    p = np.zeros(n)
    p[0] = 1.0                                   # P = 1
    o = 2 + 2                                    # skip P, p, W_0, b_0
    ks = list(range(-(m - 1), m))
    km = len(ks)
    k = (ks.index(mode[0]) * km + ks.index(mode[1])) * km + ks.index(mode[2])
    p[o + 2 * k] = value.real
    p[o + 2 * k + 1] = value.imag
    p[o + 2 * M] = 1.0                           # Q = 1
    return cfg, p


def test_plane_wave_through_one_complex_mode_fixes_the_transform_convention():
    """With DFT(h)[k] = sum_x h e^{-i k.x}, IDFT = (1/X) sum_k G e^{+i k.x} and R = i on
    the single mode k0 (zero on -k0), the input cos(k0.x) maps to Re(i e^{i k0.x} / 2)
    = -sin(k0.x) / 2.  A flipped sign convention gives +sin/2, a wrong mode index 0."""
    g, m, k0 = 6, 3, (1, 0, 2)
    cfg, p = _single_mode_net(g, m, k0, 1j)
    idx = np.arange(g)
    ix, iy, iz = np.meshgrid(idx, idx, idx, indexing="ij")
    ph = 2 * np.pi * (k0[0] * ix + k0[1] * iy + k0[2] * iz).ravel() / g
    y = fno.forward(cfg, p, np.cos(ph)[None, :, None])[0, :, 0]
    assert np.max(np.abs(y - (-np.sin(ph) / 2))) < 1e-12
