"""Learned initial guess for the self-consistent loop: data generation, training and use of the
Fourier neural operator whose forward, backward, loss and Adam steps are libbdg kernels
(bdg_fno_*).

The network maps per-site inputs (mu, Delta0, |ansatz|, cos theta, sin theta) of a seeded
vortex configuration to the correction that takes the plain start (uniform Hartree shift U0,
Delta = Delta0 x ansatz) to the converged (U, Re Delta, Im Delta) of the SCF loop
(bdg_scf_step with the phase of the ansatz held fixed); a uniform state, whose plain start is
already the fixed point, then maps to a correction near zero.  Training states are produced by that
same SCF loop from the plain start.  The SCF loop alone decides convergence: the network only
replaces the starting fields.

    python -m paper_2310_03341_b300.fno [--grid 8] [--train 24] [--test 8] [--epochs 300] [--tol 1e-4]
                                        [--checkpoint-dir DIR]

prints one JSON line with the mean SCF iterations and wall time to max|dn| <= tol from the
plain start and from the network's guess on held-out states.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CIN, COUT = 5, 3


def config(g: int, width: int = 32, modes: int = 4, layers: int = 4, bf16: bool = True):
    from . import FnoConfig
    return FnoConfig(g, width, min(modes, (g + 1) // 2), layers, CIN, COUT, 1 if bf16 else 0)


# ----------------------------------------------------------------------------- physics set-up
def coupling_for_gap(nx, ny, nz, mu, delta0, Ec=math.pi ** 2 / 2):
    """(g, U0) making the uniform state with gap delta0 self-consistent for the contact
    coupling with Hartree term (Delta = g nu, U = -g n / 2): bdg_gap_coupling of the library."""
    from . import gap_coupling
    return gap_coupling((nx, ny, nz), mu, delta0, Ec)


def sample(seed: int, g: int):
    """Seeded learned-guess state on g^3: the full recipe (mu ~ U[0.3, 0.7], Delta0 ~ U[0.1, 0.4],
    0-4 straight z-vortices) for g >= 16, the small-box recipe (Delta0 ~ U[0.4, 0.5], at most
    one vortex) below, where the full recipe's coherence length exceeds the box."""
    import workloads as wk
    return wk.c5_sample(seed, n=g) if g >= 16 else wk.c5_small_sample(seed, n=g)


def features(w):
    """(X, 5) float32: mu, Delta0, |ansatz|, cos theta, sin theta."""
    d0 = w.meta["Delta0"]
    ans = w.Delta / d0
    mag = np.abs(ans)
    th = np.angle(ans)
    X = w.V
    f = np.stack([np.full(X, w.mu), np.full(X, d0), mag, np.cos(th), np.sin(th)], axis=1)
    return f.astype(np.float32)


def plain_start(w, U0):
    return np.full(w.V, U0), w.Delta.copy()


def fixed_phase(w):
    ph = np.exp(1j * np.angle(w.Delta))
    return ph.astype(np.complex128)


# ----------------------------------------------------------------------------- SCF driver
def scf_solve(ctx, w, g, U, D, tol=1e-4, max_iter=120, alpha=0.7, prec="fp32", checkpoint=None,
              device="cuda"):
    """Iterate bdg_scf_step with the ansatz phase held fixed until max|dn| <= tol.

    checkpoint: optional .npz path.  The loop state is saved there after every step, and when the
    file already exists the loop resumes from it (a run that had converged returns at once).
    max_iter counts the resumed steps too.  A step whose max|dn| is not finite (NaN or Inf fields)
    raises FloatingPointError before anything is saved, so the checkpoint keeps the last finite
    state.
    Returns (iterations, seconds of this call, U, Delta, converged)."""
    import torch
    from . import scf_state
    grid = (w.nx, w.ny, w.nz)
    it, ok, hist, n0 = 0, False, [], np.zeros(w.V)
    if checkpoint is not None and os.path.exists(checkpoint):
        st = scf_state.load(checkpoint)
        scf_state.check_matches(st, grid, w.mu, g, alpha)
        U, D, n0 = st["U"], st["Delta"], st["n_prev"]
        it, hist = st["iteration"], st["dn_history"]
        ok = it > 1 and bool(hist) and hist[-1] <= tol      # judged against this call's tol
    Ud = torch.tensor(U, dtype=torch.float64, device=device)
    Dd = torch.tensor(D, dtype=torch.complex128, device=device)
    ph = torch.tensor(fixed_phase(w), device=device)
    n_prev = torch.tensor(n0, dtype=torch.float64, device=device)
    sync = torch.cuda.synchronize if torch.device(device).type == "cuda" else (lambda: None)
    sync()
    t = time.perf_counter()
    while not ok and it < max_iter:
        dn = ctx.scf_step(grid, Ud, Dd, n_prev, w.mu, g, alpha=alpha, prec=prec, refine_iters=0, phase=ph)
        it += 1
        if not math.isfinite(dn):
            raise FloatingPointError(f"SCF step {it}: max|dn| = {dn}; the fields are no longer finite")
        hist.append(float(dn))
        ok = it > 1 and dn <= tol
        if checkpoint is not None:
            scf_state.save(checkpoint, U=Ud, Delta=Dd, n_prev=n_prev, grid=grid, mu=w.mu, g=g, alpha=alpha,
                           tol=tol, iteration=it, converged=ok, dn_history=hist)
    sync()
    return it, time.perf_counter() - t, Ud.cpu().numpy(), Dd.cpu().numpy(), ok


def scf_solve_kz(ctx, w, g, U, D, tol=1e-4, max_iter=120, alpha=0.7, prec="fp32", checkpoint=None, device="cuda",
                 solver=None):
    """scf_solve for a z-invariant state through its kz blocks (kzscf.scf_step_kz): the loop runs on
    the (nx, ny) fields, nz/2 + 1 blocks of order 2 nx ny per step, with the ansatz phase held
    fixed, until max|dn| <= tol.  `solver(U2, D2) -> (solve_all, densities)` defaults to the
    library's (one bdg_heev_batched call and bdg_densities per block).  The checkpoint has the
    format of scf_solve's, with the fields on the full grid, so either loop can resume the other's.
    Returns (iterations, seconds, U, Delta, converged) with U, Delta on the full grid."""
    import torch
    from . import kzscf, scf_state
    nx, ny, nz = w.nx, w.ny, w.nz
    grid = (nx, ny, nz)
    U3, D3, P3 = np.asarray(U), np.asarray(D), fixed_phase(w)
    n3 = np.zeros(w.V)
    it, ok, hist = 0, False, []
    if checkpoint is not None and os.path.exists(checkpoint):
        st = scf_state.load(checkpoint)
        scf_state.check_matches(st, grid, w.mu, g, alpha)
        U3, D3, n3 = st["U"], st["Delta"], st["n_prev"]
        it, hist = st["iteration"], st["dn_history"]
        ok = it > 1 and bool(hist) and hist[-1] <= tol      # judged against this call's tol
    for f in (U3, D3, P3, n3):
        if not np.allclose(f.reshape(nx * ny, nz), f.reshape(nx * ny, nz)[:, :1]):
            raise ValueError("scf_solve_kz: the fields depend on z")
    U2 = torch.tensor(U3[::nz], dtype=torch.float64, device=device)       # z-fastest site order
    D2 = torch.tensor(D3[::nz], dtype=torch.complex128, device=device)
    ph = torch.tensor(P3[::nz], dtype=torch.complex128, device=device)
    n_prev = torch.tensor(n3[::nz], dtype=torch.float64, device=device)
    if solver is None:
        solver = lambda U_, D_: kzscf.library_solver(ctx, (nx, ny), w.mu, U_, D_, prec=prec)   # noqa: E731
    solve_all, dens = solver(U2, D2)
    full = lambda x: np.repeat(x.cpu().numpy(), nz)                                            # noqa: E731
    sync = torch.cuda.synchronize if torch.device(device).type == "cuda" else (lambda: None)
    sync()
    t = time.perf_counter()
    while not ok and it < max_iter:
        Un, Dn, n, _ = kzscf.scf_step_kz(nz, solve_all, dens, U2, D2, g, alpha=alpha, phase=ph)
        dn = float(torch.max(torch.abs(n - n_prev)).item())
        it += 1
        if not math.isfinite(dn):
            raise FloatingPointError(f"SCF step {it}: max|dn| = {dn}; the fields are no longer finite")
        U2.copy_(Un)
        D2.copy_(Dn)
        n_prev = n
        hist.append(dn)
        ok = it > 1 and dn <= tol
        if checkpoint is not None:
            scf_state.save(checkpoint, U=full(U2), Delta=full(D2), n_prev=full(n_prev), grid=grid, mu=w.mu, g=g,
                           alpha=alpha, tol=tol, iteration=it, converged=ok, dn_history=hist)
    sync()
    return (it, time.perf_counter() - t, np.repeat(U2.cpu().numpy(), nz), np.repeat(D2.cpu().numpy(), nz), ok)


def generate(ctx, seeds, grid, tol=1e-4, log=None, checkpoint_dir=None, kz=False):
    """Converged states from the plain start: inputs (S, X, 5), targets (S, X, 3) = converged
    minus plain start, SCF iterations.  With checkpoint_dir, each state's loop is checkpointed
    there (state_<grid>_<seed>.npz), so a restarted run skips finished states and resumes the rest.
    With kz, the loops run through the kz blocks (the states are z-invariant)."""
    xs, ys, its = [], [], []
    for s in seeds:
        w = sample(s, grid)
        gc, U0 = coupling_for_gap(w.nx, w.ny, w.nz, w.mu, w.meta["Delta0"])
        U, D = plain_start(w, U0)
        ck = os.path.join(checkpoint_dir, f"state_{grid}_{s}.npz") if checkpoint_dir else None
        if kz:
            it, dt, Uc, Dc, ok = scf_solve_kz(ctx, w, gc, U, D, tol=tol, checkpoint=ck)
        else:
            it, dt, Uc, Dc, ok = scf_solve(ctx, w, gc, U, D, tol=tol, checkpoint=ck)
        xs.append(features(w))
        ys.append(np.stack([Uc - U, (Dc - D).real, (Dc - D).imag], axis=1).astype(np.float32))
        its.append(it)
        if log:
            log(f"state {s}: {it} SCF iterations ({dt:.2f} s), converged={ok}")
    return np.stack(xs), np.stack(ys), its


def init_params(ctx, cfg, seed=0):
    """Seeded initial weights: uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) per block."""
    import torch
    n, _ = ctx.fno_sizes(cfg, 1)
    rng = np.random.default_rng(seed)
    W, cin, cout, m, L = cfg.width, cfg.cin, cfg.cout, cfg.modes, cfg.layers
    M = (2 * m - 1) ** 3
    parts = [rng.uniform(-1, 1, cin * W) / math.sqrt(cin), np.zeros(W)]
    for _ in range(L):
        parts += [rng.uniform(-1, 1, W * W) / math.sqrt(W), np.zeros(W),
                  rng.uniform(-1, 1, M * W * W * 2) / (W * math.sqrt(M))]
    parts += [rng.uniform(-1, 1, W * cout) / math.sqrt(W), np.zeros(cout)]
    p = np.concatenate(parts)
    assert p.size == n
    return torch.tensor(p, dtype=torch.float32, device="cuda")


def train(ctx, cfg, X, Y, epochs=300, batch=8, lr=2e-3, seed=0, log=None):
    """Adam on the MSE over (U, Re Delta, Im Delta); every step in libbdg kernels."""
    import torch
    params = init_params(ctx, cfg, seed)
    m1 = torch.zeros_like(params)
    m2 = torch.zeros_like(params)
    Xd = torch.tensor(X, device="cuda")
    Yd = torch.tensor(Y, device="cuda")
    S = X.shape[0]
    rng = np.random.default_rng(seed + 1)
    step, cache, hist = 0, None, []
    for ep in range(epochs):
        perm = rng.permutation(S)
        tot = 0.0
        for b0 in range(0, S, batch):
            idx = torch.tensor(perm[b0:b0 + batch], device="cuda")
            xb, yb = Xd[idx].contiguous(), Yd[idx].contiguous()
            out, cache = ctx.fno_forward(cfg, params, xb, cache)
            loss, dy = ctx.fno_mse(out, yb)
            grad = ctx.fno_backward(cfg, params, xb, cache, dy)
            step += 1
            rate = lr * 0.5 * (1.0 + math.cos(math.pi * ep / epochs))   # cosine schedule
            ctx.fno_adam(params, grad, m1, m2, max(rate, lr * 1e-2), step)
            tot += float(loss.item()) * xb.shape[0]
        hist.append(tot / S)
        if log and (ep % 50 == 0 or ep == epochs - 1):
            log(f"epoch {ep}: mse {hist[-1]:.3e}")
    return params, hist


def predict(ctx, cfg, params, w, U0):
    """Starting fields: the plain start plus the network's correction."""
    import torch
    x = torch.tensor(features(w)[None], device="cuda")
    out, _ = ctx.fno_forward(cfg, params, x)
    y = out[0].double().cpu().numpy()
    U, D = plain_start(w, U0)
    return U + y[:, 0], D + (y[:, 1] + 1j * y[:, 2])


def evaluate(ctx, cfg, params, seeds, grid, tol=1e-4, log=None, kz=False):
    """Per held-out state: (plain iterations, plain s, learned iterations, learned s, converged, vortices).
    With kz, both loops run through the kz blocks; the network's start is projected onto z-invariant
    fields first (its mean over z), since the kz reduction needs them."""
    rows = []
    solve = scf_solve_kz if kz else scf_solve
    for s in seeds:
        w = sample(s, grid)
        gc, U0 = coupling_for_gap(w.nx, w.ny, w.nz, w.mu, w.meta["Delta0"])
        U, D = plain_start(w, U0)
        it0, t0, *_ , ok0 = solve(ctx, w, gc, U, D, tol=tol)
        Up, Dp = predict(ctx, cfg, params, w, U0)
        if kz:
            Up = np.repeat(Up.reshape(-1, w.nz).mean(axis=1), w.nz)
            Dp = np.repeat(Dp.reshape(-1, w.nz).mean(axis=1), w.nz)
        it1, t1, *_, ok1 = solve(ctx, w, gc, Up, Dp, tol=tol)
        rows.append((it0, t0, it1, t1, ok0 and ok1, len(w.meta["centers"])))
        if log:
            log(f"held-out {s}: plain {it0} it {t0:.2f} s | learned {it1} it {t1:.2f} s")
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, default=8)
    ap.add_argument("--train", type=int, default=24)
    ap.add_argument("--test", type=int, default=8)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--fp32-weights", action="store_true")
    ap.add_argument("--vortex-only", action="store_true", help="train and evaluate on states with a vortex")
    ap.add_argument("--kz", action="store_true",
                    help="run every SCF loop through the kz blocks of the z-invariant states (kzscf)")
    ap.add_argument("--checkpoint-dir", default=None,
                    help="checkpoint every training state's SCF loop here; a rerun resumes from them")
    a = ap.parse_args()
    import torch
    from . import Context
    ctx = Context(0)
    log = lambda s: print(s, file=sys.stderr, flush=True)
    cfg = config(a.grid, bf16=not a.fp32_weights)
    t = time.perf_counter()
    keep = (lambda s: bool(sample(s, a.grid).meta["centers"])) if a.vortex_only else (lambda s: True)
    train_seeds = [s for s in range(10 * a.train + 40) if keep(s)][:a.train]
    test_seeds = [s for s in range(10_000, 10_000 + 10 * a.test + 40) if keep(s)][:a.test]
    X, Y, its = generate(ctx, train_seeds, a.grid, a.tol, log, checkpoint_dir=a.checkpoint_dir, kz=a.kz)
    t_gen = time.perf_counter() - t
    t = time.perf_counter()
    params, hist = train(ctx, cfg, X, Y, epochs=a.epochs, log=log)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t
    rows = evaluate(ctx, cfg, params, test_seeds, a.grid, a.tol, log, kz=a.kz)
    r = np.array([[x[0], x[1], x[2], x[3]] for x in rows])
    vx = np.array([x[5] > 0 for x in rows])
    print(json.dumps({
        "workload": f"learned SCF guess, {a.grid}^3 grid (N={2 * a.grid ** 3}), {a.train} training states, "
                    f"{a.test} held-out" + (", vortex states only" if a.vortex_only else "")
                    + (", SCF through the kz blocks" if a.kz else ""), "tol": a.tol,
        "fno": {"width": cfg.width, "modes": cfg.modes, "layers": cfg.layers, "bf16_weights": bool(cfg.bf16_weights)},
        "scf_iterations": {"plain": float(r[:, 0].mean()), "learned": float(r[:, 2].mean())},
        "scf_seconds": {"plain": float(r[:, 1].mean()), "learned": float(r[:, 3].mean())},
        "with_vortices": {"states": int(vx.sum()),
                          "scf_iterations": {"plain": float(r[vx, 0].mean()) if vx.any() else None,
                                             "learned": float(r[vx, 2].mean()) if vx.any() else None}},
        "all_converged": bool(all(x[4] for x in rows)),
        "train_mse_final": hist[-1], "data_seconds": t_gen, "train_seconds": t_train,
        "training_scf_iterations_mean": float(np.mean(its))}))


if __name__ == "__main__":
    main()
