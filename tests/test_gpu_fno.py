"""FNO kernels (bdg_fno_*) against the FP64 reference oracle/fno.py, and
the gain of the learned start over the plain start of the SCF loop."""
import numpy as np
import pytest

from oracle import fno as ofno
from tests.gpu_common import ctx, torch

pytestmark = pytest.mark.gpu


def _cfg(bf16, g=6, width=8, modes=2, layers=3):
    import paper_2310_03341_b300 as bdg
    return bdg.FnoConfig(g, width, modes, layers, 5, 3, 1 if bf16 else 0)


def _odict(c):
    return dict(g=c.g, width=c.width, modes=c.modes, layers=c.layers, cin=c.cin, cout=c.cout,
                bf16_weights=c.bf16_weights)


def _setup(c, B=3, seed=0):
    n, _ = ctx().fno_sizes(c, B)
    rng = np.random.default_rng(seed)
    p = (rng.standard_normal(n) * 0.25).astype(np.float32)
    x = rng.standard_normal((B, c.g ** 3, c.cin)).astype(np.float32)
    t = rng.standard_normal((B, c.g ** 3, c.cout)).astype(np.float32)
    return p, x, t


@pytest.mark.parametrize("bf16", [False, True])
def test_forward_matches_fp64_reference(bf16):
    c = _cfg(bf16)
    p, x, _ = _setup(c)
    out, _ = ctx().fno_forward(c, torch.tensor(p, device="cuda"), torch.tensor(x, device="cuda"))
    ref = ofno.forward(_odict(c), p, x)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(out.cpu().numpy() - ref)) / scale <= 1e-5
    if bf16:
        # against FP32 weights: the bf16 rounding of the weights shows at the 1e-2 level at most
        ref32 = ofno.forward(dict(_odict(c), bf16_weights=0), p, x)
        assert np.max(np.abs(out.cpu().numpy() - ref32)) / scale <= 1e-2


def test_backward_matches_finite_differences_of_the_reference():
    c = _cfg(False)
    p, x, t = _setup(c, B=2, seed=1)
    dev = lambda a: torch.tensor(a, device="cuda")
    pd, xd, td = dev(p), dev(x), dev(t)
    out, cache = ctx().fno_forward(c, pd, xd)
    loss, dy = ctx().fno_mse(out, td)
    grad = ctx().fno_backward(c, pd, xd, cache, dy).cpu().numpy()
    ref_loss = ofno.mse(ofno.forward(_odict(c), p, x), t)
    assert abs(float(loss.item()) - ref_loss) <= 1e-5 * ref_loss
    # sampled parameters from every block: lift, each layer's W / b / R, projection
    rng = np.random.default_rng(2)
    idx = np.unique(np.concatenate([rng.choice(p.size, 40, replace=False), [0, p.size - 1, p.size - 4]]))
    fd = ofno.fd_gradient(_odict(c), p.astype(np.float64), x, t, idx, eps=1e-4)
    g = grad[idx]
    assert np.linalg.norm(g - fd) <= 2e-3 * np.linalg.norm(fd)
    big = np.abs(fd) > 1e-3 * np.max(np.abs(fd))
    assert np.max(np.abs(g[big] - fd[big]) / np.abs(fd[big])) <= 2e-2


def test_adam_step_matches_its_definition():
    n = 1000
    rng = np.random.default_rng(3)
    p = rng.standard_normal(n).astype(np.float32)
    g = rng.standard_normal(n).astype(np.float32)
    m1 = (rng.standard_normal(n) * 0.1).astype(np.float32)
    m2 = np.abs(rng.standard_normal(n) * 0.1).astype(np.float32)
    dev = lambda a: torch.tensor(a, device="cuda")
    pd, gd, m1d, m2d = dev(p), dev(g), dev(m1), dev(m2)
    ctx().fno_adam(pd, gd, m1d, m2d, 1e-2, 5, 0.9, 0.999, 1e-8)
    a = 0.9 * m1 + 0.1 * g
    v = 0.999 * m2 + 0.001 * g * g
    ref = p - 1e-2 * (a / (1 - 0.9 ** 5)) / (np.sqrt(v / (1 - 0.999 ** 5)) + 1e-8)
    assert np.max(np.abs(pd.cpu().numpy() - ref)) <= 1e-6


def test_learned_start_cuts_scf_iterations():
    """Train on SCF states the library generates (8^3 small-box recipe, fixed
    vortex phase), then compare the SCF iterations to max|dn| <= 1e-4 from the
    plain start and from the network's guess on held-out vortex states."""
    from paper_2310_03341_b300 import fno
    c = ctx()
    cfg = fno.config(8, width=16, modes=3, layers=4, bf16=True)
    train = [s for s in range(40) if fno.sample(s, 8).meta["centers"]][:6]
    X, Y, its = fno.generate(c, train, 8)
    params, hist = fno.train(c, cfg, X, Y, epochs=200, batch=6, lr=3e-3)
    assert hist[-1] < 0.2 * hist[0]
    held = [s for s in range(10_000, 10_040) if fno.sample(s, 8).meta["centers"]][:2]
    rows = fno.evaluate(c, cfg, params, held, 8)
    assert np.mean([r[2] for r in rows]) < np.mean([r[0] for r in rows])
