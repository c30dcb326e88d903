"""Host-side logic of bench.py: the algorithmic work credited to the sliced-product kernel,
the config object shared by both arms, and the clock sampler's choice of device (no GPU)."""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _brute_force_flops(m, kp, slices=6, tn=16):
    """S(S+1)/2 slice pairs x 4 real products x 2 flop per MAC on every 128 x tn tile with a column >=
    its first row."""
    tiles = 0
    for i in range(0, (m + 127) // 128):
        for j in range(0, (m + tn - 1) // tn):
            if j * tn + tn - 1 >= i * 128:
                tiles += 1
    return tiles * (kp // 64) * 4 * 128 * 64 * 2 * tn * sum(range(1, slices + 1))


def test_roofline_credits_the_kernel_work():
    for N, ph in [(8192, True), (8192, False), (4608, True), (36864, True)]:
        res = {"N": N, "oz": {"ms": {6: 1000.0}, "stages": {6: 1}}, "refine_ph": ph}
        r = bench.roofline(res, {"bf16_tflops_sustained": 1000.0})
        m = N // 2 if ph else N
        kp = 2 * ((N // 2 + 63) // 64) * 64
        launches = 2 if ph else 1
        assert r["issued_flop"] == launches * _brute_force_flops(m, kp)
        assert r["launches_timed"] == launches
        assert abs(r["achieved"] - r["issued_flop"] / 1e12) <= 0.005 + 1e-9 * r["achieved"]   # rounded to 0.01
        assert abs(r["method_flop_per_launch"] - 4.0 * m * (m + 1) * N) <= 1e-6 * r["method_flop_per_launch"]


def test_roofline_counts_fewer_slice_pairs_for_cheaper_products():
    """S slices keep S (S + 1) / 2 slice pairs: 10, 15 and 21 for 4, 5 and 6."""
    N = 8192
    kp = 2 * ((N // 2 + 63) // 64) * 64
    f = {sl: bench.oz_issued_flop(N // 2, N, sl) for sl in (4, 5, 6)}
    for sl, tn in ((4, 32), (5, 24), (6, 16)):
        assert f[sl] == _brute_force_flops(N // 2, kp, sl, tn)
    res = {"N": N, "oz": {"ms": {4: 500.0, 6: 500.0}, "stages": {4: 2, 6: 2}}, "refine_ph": True}
    r = bench.roofline(res, {"bf16_tflops_sustained": 1000.0})
    assert r["launches_by_slices"] == {"4": 4, "6": 4} and r["issued_flop"] == 4 * (f[4] + f[6])


def test_arm_configs_name_what_each_arm_ran():
    """The GPU arm names the workload it solved; the reference arm names the bounded
    sample the oracle solved (its N and FP64 arithmetic) and the workload it stands for."""
    import workloads as wk
    args = argparse.Namespace(prec="bf16x9", tol=1e-10)
    w = wk.c3_vortex_lattice()
    c_ours = bench.arm_config(args, w, 1, True, True)
    assert c_ours["N"] == w.N == 36864 and c_ours["workload"] == w.name
    c_ref = bench.reference_config(args, w, 1)
    s = bench.cpu_sample_workload()
    assert c_ref["N"] == s.N == 2048 and c_ref["workload"] == s.name
    assert c_ref["grid"] == [8, 16, 8] and c_ref["precision"].startswith("fp64")
    assert c_ref["stands_for"]["N"] == w.N
    c64 = bench.arm_config(argparse.Namespace(prec="fp64", tol=1e-10), w, 1)
    assert c64["precision"].startswith("fp64") and c64["refine_tol"] is None


def test_clock_sampler_falls_back_from_uuid_to_index(monkeypatch):
    """nvidia-smi is asked for the device by UUID first; when that is refused before any
    sample, the sampler uses the logical index (a fake nvidia-smi stands in)."""
    import subprocess
    import types
    calls = []

    def fake_run(cmd, **kw):
        ident = [a for a in cmd if a.startswith("--id=")][0][5:]
        calls.append(ident)
        if ident.startswith("GPU-"):
            return types.SimpleNamespace(returncode=6, stdout="")
        return types.SimpleNamespace(returncode=0, stdout="0, 2032, 2032, 700.5, Active, Not Active, Not Active, "
                                                            "Not Active, Active\n")

    monkeypatch.setattr(subprocess, "run", fake_run)
    cs = bench.ClockSampler(0)
    cs.ids = ["GPU-00000000-0000-0000-0000-000000000000", "0"]
    import time
    with cs:
        time.sleep(0.5)
    assert calls[0].startswith("GPU-") and calls[1] == "0" and cs.ids == ["0"]
    s = cs.summary()
    assert s["sm_mhz"] == 2032.0 and s["reasons"] == ["sw_power_cap"]
