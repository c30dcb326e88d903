"""A fixed, bounded profiling case for the kernels of libbdg.

    python -m paper_2310_03341_b300.profile_case [--grid NX NY NZ] [--prec P] [--iters K]

builds the vortex-pairing BdG matrix of a random_small workload on the grid
(default 12 x 12 x 16, N = 4608: the refinement's sliced operands are larger
than L2 while the whole case holds about 3 GB of device memory), runs one
mixed-precision particle-hole solve and K refinement iterations (default 1),
and prints the stage times.  It exists so that profiler captures of single
kernels (the sliced products, the back-transformations) run on a small,
reproducible case of the real path.
"""
import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, nargs=3, default=[12, 12, 16])
    ap.add_argument("--prec", default="bf16x9")
    ap.add_argument("--iters", type=int, default=1)
    a = ap.parse_args()
    import torch
    import paper_2310_03341_b300 as bdg
    import workloads as wk
    w = wk.random_small(*a.grid, seed=5, n_vortices=2)
    grid = (w.nx, w.ny, w.nz)
    ctx = bdg.Context(0)
    ctx.set_timing(True)
    U = torch.tensor(w.U, dtype=torch.float64, device="cuda")
    D = torch.tensor(w.Delta, dtype=torch.complex128, device="cuda")
    H = ctx.build(grid, w.mu, U, D)
    ev, Z = ctx.heev(H, a.prec, overwrite=True, ph=True)
    st_h = ctx.stage_times()
    r, _, it, _ = ctx.refine(grid, w.mu, U, D, ev, Z, a.iters, 1e-14, orth=False)
    st_r = ctx.stage_times()
    torch.cuda.synchronize()
    print(f"N={w.N} resid after {it} iterations: {r:.3e}")
    for k, v in st_h + st_r:
        print(f"  {k:16s} {v:10.3f} ms")


if __name__ == "__main__":
    main()
