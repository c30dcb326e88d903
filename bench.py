"""Benchmark of the BdG eigensolve hot path on B300.

One step = one diagonalisation of the dense BdG matrix of the static SLDA
loop at the vortex-lattice workload (24 x 24 x 32 grid, N = 36864 by
default): bdg_build -> bdg_heev (reduced precision, tensor-core products) ->
bdg_refine (Ogita-Aishima, FP64-accurate, to a residual <= 1e-10 rho) ->
bdg_densities.  Throughput is reported as F(N)/t with the standard credited
flop count of a complex Hermitian eigendecomposition with all vectors,
F(N) = (16/3 + 8) N^3 real flops.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload C3|C2|C1|C4]
                  [--impl ours|reference] [--prec bf16x9|fp64|...] [--fp64-steps S]
                  [--e2e-steps E]

With --prec fp64 the step is the same library's all-FP64 path (build -> FP64
heev -> densities, no refinement): the "FP64 GPU" side of the metric.
The end-to-end leg (host buffers in and out) runs a fixed E steps (default 2)
after the device-timed K steps; the line states E.

Multi-GPU (torchrun): every rank solves its own replica of the workload
(independent diagonalisations, no collective in the data path): weak scaling.
The reference arm (--impl reference) times the FP64 CPU oracle, as it stands,
on a bounded sample of the workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "BdG eigensolve sec and TFLOP/s at N=36864, mixed vs FP64 GPU, at 1e-10 residual"
UNIT = "TFLOP/s"


def flops(N: int) -> float:
    return (40.0 / 3.0) * float(N) ** 3


def workload(name: str):
    import workloads as wk
    return wk.by_name(name)


def cpu_sample_workload():
    """Bounded CPU sample: the vortex-lattice recipe of the benchmark workload
    (four +-1 straight vortices, |Delta| = 0.25, U = -0.4 + 0.05 * smooth field,
    mu = 0.5) on an 8 x 16 x 8 grid (N = 2048)."""
    import workloads as wk
    nx, ny, nz = 8, 16, 8
    centers = [(-2.0, -4.0), (2.0, 4.0), (-2.0, 4.0), (2.0, -4.0)]
    D = wk.vortex_pairing(nx, ny, nz, 0.25, centers, [1, -1, 1, -1])
    U = -0.4 + wk.smooth_field((nx, ny, nz), 3.0, 3, 0.05)
    return wk.Workload("C3_recipe_sample_8x16x8", nx, ny, nz, 0.5, U, D, {})


def time_oracle(threads: int):
    import oracle
    w = cpu_sample_workload()
    H = oracle.build(w)
    t = time.perf_counter()
    oracle.heev(H, vectors=True, threads=threads)
    dt = time.perf_counter() - t
    return w.N, dt


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clocks and throttle reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank: int):
        # the device's UUID names the physical GPU whatever CUDA_VISIBLE_DEVICES remaps; the
        # logical index is the fallback when the UUID is unavailable or not accepted
        self.ids = []
        try:
            import torch
            uuid = getattr(torch.cuda.get_device_properties(local_rank), "uuid", None)
            if uuid is not None:
                self.ids.append("GPU-" + str(uuid))
        except Exception:
            pass
        self.ids.append(str(local_rank))
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.ids[0]}", f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                if out.returncode == 0 and out.stdout.strip():
                    self.samples.append([x.strip() for x in out.stdout.strip().split(",")])
                elif not self.samples and len(self.ids) > 1:
                    self.ids.pop(0)
                    continue
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace('.', '', 1).isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace('.', '', 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for k, name in enumerate(names):
                if len(s) > 5 + k and s[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2310_03341_b300 as bdg

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = workload(args.workload)
    N, V = w.N, w.V
    grid = (w.nx, w.ny, w.nz)
    ctx = bdg.Context(local_rank)
    U0 = torch.tensor(w.U, dtype=torch.float64, device=dev)
    D0 = torch.tensor(w.Delta, dtype=torch.complex128, device=dev)
    # persistent device buffers (inputs resident in HBM before timing)
    Hbuf = torch.empty(N, N, dtype=torch.complex128, device=dev)
    Zbuf = torch.empty(N, N, dtype=torch.complex128, device=dev)
    wv = torch.empty(N, dtype=torch.float64, device=dev)
    nd = torch.empty(V, dtype=torch.float64, device=dev)
    nu = torch.empty(V, dtype=torch.complex128, device=dev)
    L = bdg.lib()
    gptr = bdg.Grid(*grid, 1.0)
    import ctypes as C
    stream = torch.cuda.current_stream(dev)
    sptr = C.c_void_p(stream.cuda_stream)
    phf = 0 if args.no_ph else bdg.HEEV_PH   # particle-hole half solve (BDG_HEEV_PH)
    prec = bdg.PREC[args.prec] | phf
    fp64_mode = args.prec == "fp64"
    info = {}

    stages = {"heev": {}, "refine": {}}
    oz = {"ms": {}, "stages": {}}      # by slices per operand: summed ms and number of product stages

    def add_stages(kind, st, record):
        if not record:
            return
        for k, v in st:
            stages[kind][k] = stages[kind].get(k, 0.0) + v
            if kind == "refine" and k.startswith(("ref_oz_gram_s", "ref_oz_s_s")):
                sl = int(k.rsplit("_s", 1)[1])
                oz["ms"][sl] = oz["ms"].get(sl, 0.0) + v
                oz["stages"][sl] = oz["stages"].get(sl, 0) + 1

    def step(U, D, record=False):
        rc = L.bdg_build(ctx._h, C.byref(gptr), float(w.mu), C.c_void_p(U.data_ptr()), C.c_void_p(D.data_ptr()),
                         C.c_void_p(Hbuf.data_ptr()), N, sptr)
        ctx._check(rc)
        ctx._check(L.bdg_heev(ctx._h, N, C.c_void_p(Hbuf.data_ptr()), N, C.c_void_p(wv.data_ptr()),
                              C.c_void_p(Zbuf.data_ptr()), N, prec, sptr))
        add_stages("heev", ctx.stage_times() if record else [], record)
        if fp64_mode:
            info.update(resid=None, iters=0, converged=None)
        else:
            refine(U, D, record)
        ctx._check(L.bdg_densities(ctx._h, C.byref(gptr), N, C.c_void_p(wv.data_ptr()), C.c_void_p(Zbuf.data_ptr()),
                                   N, 0.0, math.pi ** 2 / 2, C.c_void_p(nd.data_ptr()), C.c_void_p(nu.data_ptr()),
                                   sptr))

    def refine(U, D, record):
        r, it = C.c_double(), C.c_int()
        # the timed step does not ask for the orthogonality (that would add one
        # Gram product); it is measured on the final vectors after timing
        rc = L.bdg_refine(ctx._h, C.byref(gptr), float(w.mu), C.c_void_p(U.data_ptr()), C.c_void_p(D.data_ptr()), N,
                          C.c_void_p(wv.data_ptr()), C.c_void_p(Zbuf.data_ptr()), N, args.refine_iters,
                          args.tol, C.byref(r), None, C.byref(it), sptr)
        if rc not in (0, -4):
            ctx._check(rc)
        add_stages("refine", ctx.stage_times() if record else [], record)
        info.update(resid=r.value, iters=it.value, converged=(rc == 0))

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        step(U0, D0)
    torch.cuda.synchronize()

    # ---- device-timed steps (inputs resident; H = 16 N^2 bytes >> L2, so no flush is needed).
    # Stage events (CUDA events on the launching stream) stay on: they time the
    # dominant kernel live inside the timed region.
    ctx.set_timing(True)
    l0 = ctx.launch_count()
    ev_s = torch.cuda.Event(enable_timing=True)
    ev_e = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as cs:
        ev_s.record(stream)
        for _ in range(args.steps):
            step(U0, D0, record=True)
        ev_e.record(stream)
        torch.cuda.synchronize()
    launches = ctx.launch_count() - l0
    modes = ctx.last_modes()
    ctx.set_timing(False)
    ms_total = ev_s.elapsed_time(ev_e)
    ms = ms_total / args.steps
    if world > 1:
        from paper_2310_03341_b300.sharding import max_over_ranks
        ms = max_over_ranks(ms, device=dev)
    clocks = cs.summary()
    heev_stages = [(k, v / args.steps) for k, v in stages["heev"].items()]
    ref_stages = [(k, v / args.steps) for k, v in stages["refine"].items()]

    # ---- accuracy of the final pairs (untimed): residual and orthogonality
    r, o, it = C.c_double(), C.c_double(), C.c_int()
    L.bdg_refine(ctx._h, C.byref(gptr), float(w.mu), C.c_void_p(U0.data_ptr()), C.c_void_p(D0.data_ptr()), N,
                 C.c_void_p(wv.data_ptr()), C.c_void_p(Zbuf.data_ptr()), N, 0, args.tol,
                 C.byref(r), C.byref(o), C.byref(it), sptr)
    info.update(resid_check=r.value, orth=o.value)

    # ---- e2e: host buffers in, eigenvalues + densities out, copies inside the timed region
    e2e = None
    e2e_steps = max(1, args.e2e_steps)
    if not args.no_e2e:
        Uh = torch.tensor(w.U, dtype=torch.float64).pin_memory()
        Dh = torch.tensor(w.Delta, dtype=torch.complex128).pin_memory()
        wh = torch.empty(N, dtype=torch.float64).pin_memory()
        nh = torch.empty(V, dtype=torch.float64).pin_memory()
        nuh = torch.empty(V, dtype=torch.complex128).pin_memory()
        Ud = torch.empty_like(U0)
        Dd = torch.empty_like(D0)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            Ud.copy_(Uh, non_blocking=True)
            Dd.copy_(Dh, non_blocking=True)
            step(Ud, Dd)
            wh.copy_(wv, non_blocking=True)
            nh.copy_(nd, non_blocking=True)
            nuh.copy_(nu, non_blocking=True)
            torch.cuda.synchronize()
        t_e2e = (time.perf_counter() - t0) / e2e_steps
        if world > 1:
            from paper_2310_03341_b300.sharding import max_over_ranks
            t_e2e = max_over_ranks(t_e2e, device=dev)
        h2d = Uh.numel() * 8 + Dh.numel() * 16
        d2h = wh.numel() * 8 + nh.numel() * 8 + nuh.numel() * 16
        e2e = {"value": world * flops(N) / t_e2e / 1e12, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "seconds_per_step": t_e2e, "steps": e2e_steps,
               "path": "pinned host U, Delta -> device; build, heev, refine, densities; eigenvalues and "
                       "densities -> pinned host"}

    # ---- optional FP64 GPU path (same library, all-FP64)
    fp64 = None
    if args.fp64_steps > 0:
        ctx.set_timing(True)
        tt = []
        for _ in range(args.fp64_steps):
            ctx._check(L.bdg_build(ctx._h, C.byref(gptr), float(w.mu), C.c_void_p(U0.data_ptr()),
                                   C.c_void_p(D0.data_ptr()), C.c_void_p(Hbuf.data_ptr()), N, sptr))
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx._check(L.bdg_heev(ctx._h, N, C.c_void_p(Hbuf.data_ptr()), N, C.c_void_p(wv.data_ptr()),
                                  C.c_void_p(Zbuf.data_ptr()), N, bdg.PREC["fp64"] | phf, sptr))
            b.record(stream)
            torch.cuda.synchronize()
            tt.append(a.elapsed_time(b) / 1e3)
        fp64 = {"seconds": min(tt), "tflops": flops(N) / min(tt) / 1e12, "steps": args.fp64_steps,
                "stages_ms": {k: round(v, 2) for k, v in ctx.stage_times()}}
        ctx.set_timing(False)

    # ---- optional: the library's own SCF step (bdg_scf_step: build, heev, refine, densities, update)
    scf = None
    if args.scf_steps > 0:
        Hbuf = Zbuf = None                           # the SCF step owns its H and Z
        torch.cuda.empty_cache()
        from paper_2310_03341_b300 import fno
        g_c, _ = fno.coupling_for_gap(w.nx, w.ny, w.nz, w.mu, 0.25)
        Us, Ds = U0.clone(), D0.clone()
        n_prev = torch.zeros(V, dtype=torch.float64, device=dev)
        prec_s = "fp64" if fp64_mode else args.prec
        ctx.scf_step(grid, Us, Ds, n_prev, w.mu, g_c, alpha=0.3, prec=prec_s, refine_iters=args.refine_iters,
                     refine_tol=args.tol)          # untimed: sizes the workspace
        tt, dn = [], None
        for _ in range(args.scf_steps):
            a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            dn = ctx.scf_step(grid, Us, Ds, n_prev, w.mu, g_c, alpha=0.3, prec=prec_s,
                              refine_iters=args.refine_iters, refine_tol=args.tol)
            b_.record(stream)
            torch.cuda.synchronize()
            tt.append(a.elapsed_time(b_) / 1e3)
        scf = {"seconds_per_step": statistics.median(tt), "steps": args.scf_steps, "max_dn_last": dn,
               "call": "bdg_scf_step (build, heev, refine, densities, mixed update; contact coupling for "
                       "|Delta0| = 0.25, alpha = 0.3)"}

    return dict(w=w, N=N, ms=ms, info=info, clocks=clocks, e2e=e2e, launches=launches, heev_stages=heev_stages,
                ref_stages=ref_stages, fp64=fp64, oz=oz, steps=args.steps, refine_ph=modes[1], heev_ph=modes[0],
                scf=scf)


def run_c4(args):
    """The batched tube workload (C4): Nx = Ny in {16, 24, 32, 48}, Nz = 64, one vortex and a seeded
    U field per geometry, 256 kz blocks of orders 512 / 1152 / 2048 / 4608.  One step = build every
    block (bdg_build on the L x L x 1 grid with mu - kz^2/2) and solve them all with one
    bdg_heev_batched call (BF16X9, particle-hole half solve, no refinement).  Throughput is
    sum_i F(n_i) / t.  Printed as its own JSON line (not the headline metric)."""
    import torch
    import paper_2310_03341_b300 as bdg
    import workloads as wk
    ctx = bdg.Context(0)
    geoms = wk.c4_tubes()
    fields = [(g["L"], g["mu"], torch.tensor(g["U"].reshape(-1), dtype=torch.float64, device="cuda"),
               torch.tensor(g["Delta"].reshape(-1), dtype=torch.complex128, device="cuda"), g["kz"]) for g in geoms]
    sizes = [2 * L * L for L, _, _, _, kz in fields for _ in kz]
    F = sum(flops(n) for n in sizes)

    def step():
        blocks = []
        for L, mu, U, D, kz in fields:
            blocks += ctx.build_kz_blocks((L, L), mu, U, D, kz)
        return ctx.heev_batched(blocks, args.prec, ph=not args.no_ph, overwrite=True)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = ctx.launch_count()
    with ClockSampler(0) as cs:
        e0.record(st)
        for _ in range(args.steps):
            step()
        e1.record(st)
        torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / args.steps
    launches = ctx.launch_count() - l0
    print(json.dumps({"metric": "batched BdG eigensolve TFLOP/s, sum F(n_i)/t over 256 kz blocks (C4)",
                      "value": F / t / 1e12, "unit": UNIT, "seconds_per_step": t, "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                      "dtype": args.prec + " (no refinement)", "data": "synthetic",
                      "config": {"workload": "C4_tubes_L16-48_nz64", "blocks": len(sizes),
                                 "orders": sorted(set(sizes)), "particle_hole_half_solve": not args.no_ph},
                      "clocks": cs.summary(), "gpu_launches": launches}))
    return 0


def precision_label(prec):
    if prec == "fp64":
        return "fp64 reduction and back-transformation (all-FP64 GPU path, no refinement)"
    return prec + " reduction, FP64-accurate refinement"


def arm_config(args, w, world=1, heev_ph=None, refine_ph=None):
    """The config object of the GPU arm's JSON line: the workload it solved."""
    c = {"workload": w.name, "N": w.N, "grid": [w.nx, w.ny, w.nz],
         "precision": precision_label(args.prec),
         "refine_tol": None if args.prec == "fp64" else args.tol,
         "l2": "inputs larger than L2 (H is 16 N^2 bytes)",
         "parallelism": f"replicas x{world}"}
    if heev_ph is not None:
        c["particle_hole_half_solve"] = bool(heev_ph)
        c["particle_hole_refinement"] = bool(refine_ph)
    return c


def reference_config(args, w, world=1):
    """The config object of the reference arm's line: the bounded sample the oracle
    actually solved (its N, grid and FP64 arithmetic), next to the workload it stands for."""
    ws = cpu_sample_workload()
    return {"workload": ws.name, "N": ws.N, "grid": [ws.nx, ws.ny, ws.nz],
            "precision": "fp64 (CPU oracle: unblocked Householder, implicit QR, all eigenpairs)",
            "stands_for": {"workload": w.name, "N": w.N, "grid": [w.nx, w.ny, w.nz]},
            "rate": "F(N)/t at the sample's N; not extrapolated to the workload's N",
            "parallelism": f"host cores, rank 0 of {world}"}


OZ_TILE_WIDTH = {4: 32, 5: 24, 6: 16}      # output columns per tile of the sliced product, by slices


def oz_tiles(m: int, N: int, tn: int = 16):
    """Output tiles (128 x tn) of one sliced-product launch that touch the upper triangle of the
    m x m result, and the 64-wide chunks of its padded contraction axis (u and v halves of the
    BdG vectors, each padded to 64)."""
    V = N // 2
    kp = 2 * ((V + 63) // 64) * 64
    tm = 128
    mt, nt = (m + tm - 1) // tm, (m + tn - 1) // tn
    tiles = sum(min(nt, nt - (i * tm) // tn) for i in range(mt))   # tiles with j*tn+tn-1 >= i*128
    return tiles, kp // 64


def oz_issued_flop(m: int, N: int, slices: int) -> int:
    """bf16 tensor-core flops one launch issues: on every tile and chunk, for each slice a of X,
    two MMAs of 128 x 2 tn (S - a) x 64 (levels a .. S-1, real and imaginary part)."""
    tn = OZ_TILE_WIDTH[slices]
    tiles, kblocks = oz_tiles(m, N, tn)
    pairs_cols = tn * slices * (slices + 1) // 2          # sum over slices a of tn (S - a)
    return tiles * kblocks * 4 * 128 * 64 * 2 * pairs_cols


def roofline(res, peaks):
    """Dominant kernel = the FP64-accurate sliced product of the refinement,
    timed live with CUDA events on its stream over the timed steps.
    Two work counts per launch, both reported:
    * issued: the bf16 tensor-core flops it issues (S(S+1)/2 slice pairs x 4
      real products on every 128 x tn tile touching the upper triangle, tn = 32, 24, 16 for
      S = 4, 5, 6);
      frac = issued rate / the measured bf16 peak: how well the kernel uses
      the tensor pipe;
    * method: the complex product it delivers, 8 real flops per complex MAC
      over the upper triangle, m (m + 1) / 2 entries x N terms; frac_method =
      that rate / the same peak.
    m = N/2 and two launches per product stage with the particle-hole
    reduction, m = N and one launch per stage without."""
    N = res["N"]
    if not res["oz"]["stages"]:
        return None
    ph = res.get("refine_ph", False)
    m = N // 2 if ph else N
    per_stage = 2 if ph else 1
    ms = sum(res["oz"]["ms"].values())
    n_launch = per_stage * sum(res["oz"]["stages"].values())
    issued = sum(per_stage * c * oz_issued_flop(m, N, sl) for sl, c in res["oz"]["stages"].items())
    method = n_launch * 8.0 * (m * (m + 1) / 2) * N
    achieved = issued / (ms * 1e-3) / 1e12
    achieved_m = method / (ms * 1e-3) / 1e12
    peak = peaks.get("bf16_tflops_sustained")
    src = "bf16_tflops_sustained of measured"
    if not peak:
        peak, src = 1400.0, "1.4 PFLOP/s sustained bf16 of fallback"
    return {"kernel": "ozaki_kernel (FP64-accurate X^H Y / X^T C Y, refinement)", "bound": "tensor",
            "achieved": round(achieved, 2), "peak": peak, "unit": "TFLOP/s",
            "frac": round(achieved / peak, 4), "traffic": res.get("oz_traffic"),
            "achieved_method": round(achieved_m, 2), "frac_method": round(achieved_m / peak, 4),
            "peak_source": src, "launches_timed": n_launch,
            "launches_by_slices": {str(sl): per_stage * c for sl, c in sorted(res["oz"]["stages"].items())},
            "ms_per_launch": round(ms / n_launch, 3), "issued_flop": issued,
            "method_flop_per_launch": method / n_launch, "result_order": m}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="C3")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16x9", choices=["fp32", "bf16x3", "bf16x6", "bf16x9", "fp64"])
    ap.add_argument("--refine-iters", type=int, default=6)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--fp64-steps", type=int, default=0)
    ap.add_argument("--scf-steps", type=int, default=0, help="also time S calls of bdg_scf_step (SCF throughput)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2, help="steps of the end-to-end leg (host buffers)")
    ap.add_argument("--no-ph", action="store_true", help="full spectrum solve (no particle-hole half solve)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return 0
        import oracle
        threads = os.cpu_count() or 1
        for _ in range(min(args.warmup, 1)):
            time_oracle(threads)
        tt = [time_oracle(threads)[1] for _ in range(max(args.steps, 1))]
        n_s = cpu_sample_workload().N
        t = statistics.median(tt)
        val = flops(n_s) / t / 1e12
        sample = f"FP64 CPU oracle, full eigenpairs of the benchmark recipe on an 8x16x8 grid (N={n_s}), {t:.2f} s"
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": reference_config(args, workload(args.workload), args.gpus),
                          "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                                           "sample": sample},
                          "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return 0

    if args.workload == "C4":
        if world > 1 and rank != 0:
            return 0
        return run_c4(args)

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")

    res = run_ours(args, rank, world, local_rank)
    if rank != 0:
        return 0
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    N = res["N"]
    secs = res["ms"] / 1e3
    value = world * flops(N) / secs / 1e12
    cpu = None
    if not args.no_cpu_baseline and world == 1:      # the host baseline is taken at N = 1 only
        import oracle
        threads = os.cpu_count() or 1
        n_s, t = time_oracle(threads)
        cpu = {"value": flops(n_s) / t / 1e12, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
               "sample": f"FP64 CPU oracle, full eigenpairs of the benchmark recipe on an 8x16x8 grid "
                         f"(N={n_s}) in {t:.2f} s, scaled as F(N)/t"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["ms"], "seconds_per_solve": secs, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32+f64"}.get(args.prec, args.prec + "+f64"),
        "data": "synthetic",
        "config": arm_config(args, res["w"], world, res["heev_ph"], res["refine_ph"]),
        "accuracy": {"resid_over_rho": res["info"].get("resid"), "orth": res["info"].get("orth"),
                     "resid_recheck": res["info"].get("resid_check"),
                     "refine_iters": res["info"].get("iters"), "converged": res["info"].get("converged")},
        "clocks": res["clocks"], "e2e": res["e2e"], "gpu_launches": res["launches"],
        "roofline": roofline(res, peaks), "cpu_baseline": cpu,
        "stages_ms": {"heev": {k: round(v, 2) for k, v in res["heev_stages"]},
                      "refine": {k: round(v, 2) for k, v in res["ref_stages"]}},
    }
    if res["fp64"]:
        line["fp64_gpu"] = res["fp64"]
    if res.get("scf"):
        line["scf"] = res["scf"]
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
