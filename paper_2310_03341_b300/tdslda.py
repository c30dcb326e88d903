"""Time evolution of the quasiparticle wavefunctions on the GPU: throughput and roofline.

    python -m paper_2310_03341_b300.tdslda [--workload C2] [--steps K] [--warmup W] [--dt DT]

The initial states are the quasiparticle wavefunctions of the static problem with 0 < E < Ec
(mixed-precision eigensolve refined to 1e-10, the benchmark's path) of the chosen workload; they
are evolved under Eq. (TDSLDA) with the contact functional (U = U_ext - g n / 2, Delta = g nu,
U_ext the workload's U and g from the uniform gap equation at |Delta| = 0.3), so the state is not
stationary.  One bdg_td_evolve call runs the RK4 start and the ABM steps; the timed region is
K ABM steps (a call of W + K steps minus a call of W steps, both timed with CUDA events on the
launching stream).  Printed as one JSON line: time steps per second, quasiparticle
wavefunction-steps per second, and the FP64 rate of the evaluations (two per ABM step, each
dominated by H applied to every state through the Kronecker-sum kinetic operator).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def h_apply_flops(nx: int, ny: int, nz: int) -> float:
    """Real flops of H applied to one state: per site, for u and v, the three line sums of the
    kinetic operator (nx + ny + nz complex-by-real taps, 4 flops each) plus the diagonal and
    pairing terms (about 24 flops)."""
    V = nx * ny * nz
    return V * (2 * (nx + ny + nz) * 4 + 24)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="C2")
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=8)
    ap.add_argument("--dt", type=float, default=0.01)
    a = ap.parse_args()
    import torch
    import paper_2310_03341_b300 as bdg
    import workloads as wk
    from paper_2310_03341_b300 import fno
    w = wk.by_name(a.workload)
    grid = (w.nx, w.ny, w.nz)
    ctx = bdg.Context(0)
    U = torch.tensor(w.U, dtype=torch.float64, device="cuda")
    D = torch.tensor(w.Delta, dtype=torch.complex128, device="cuda")
    H = ctx.build(grid, w.mu, U, D)
    ev, Z = ctx.heev(H, "bf16x9", overwrite=True, ph=True)
    del H
    ctx.refine(grid, w.mu, U, D, ev, Z, 6, 1e-10, orth=False)
    sel = torch.nonzero((ev > 0) & (ev < math.pi ** 2 / 2)).flatten()
    E0 = ev[sel].contiguous()
    Psi0 = bdg.colmajor(Z[:, sel])
    del Z
    torch.cuda.empty_cache()
    nq = E0.shape[0]
    g, _ = fno.coupling_for_gap(w.nx, w.ny, w.nz, w.mu, 0.3)

    def run(nsteps):
        P = Psi0.mT.clone().mT
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        ctx.td_evolve(grid, E0, P, a.dt, nsteps, w.mu, g, U_ext=U, densities=False)
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, P

    run(a.warmup)                                  # warm up
    t_w, _ = run(a.warmup)
    t_all, P = run(a.warmup + a.steps)
    t = (t_all - t_w) / a.steps                    # seconds per ABM step
    G = P.mT.conj() @ P
    orth = float(torch.max(torch.abs(G - torch.eye(nq, dtype=G.dtype, device=G.device))).item())
    fl = 2 * nq * h_apply_flops(w.nx, w.ny, w.nz)  # two evaluations per ABM step
    print(json.dumps({"workload": f"{w.name} (N = {w.N})", "states": nq, "dt": a.dt, "steps_timed": a.steps,
                      "seconds_per_step": t, "steps_per_second": 1.0 / t,
                      "state_steps_per_second": nq / t, "h_apply_tflops": fl / t / 1e12,
                      "orthogonality_after": orth}))


if __name__ == "__main__":
    main()
