"""Checkpoint and resume of the self-consistent loop (host logic, CPU).

The loop driver is the one the learned-guess pipeline uses; the GPU step is stood in for by a
deterministic host contraction with the same in-place interface as Context.scf_step, so an
interrupted-and-resumed run must end bit for bit where an uninterrupted run ends."""
import os

import numpy as np
import pytest
import torch

import workloads as wk
from paper_2310_03341_b300 import fno, scf_state


class FakeScf:
    """In-place update of (U, Delta, n_prev) toward a fixed point; returns max|dn|."""

    def __init__(self):
        self.calls = 0

    def scf_step(self, grid, U, D, n_prev, mu, g, alpha=0.3, prec="fp64", refine_iters=0, phase=None):
        self.calls += 1
        n = 0.5 + 0.2 * torch.tanh(U + D.abs())
        nu = 0.1 * torch.cos(U) * phase
        U.mul_(1 - alpha).add_(alpha * (-g * n / 2))
        D.mul_(1 - alpha).add_(alpha * g * nu)
        dn = float((n - n_prev).abs().max())
        n_prev.copy_(n)
        return dn


def _case():
    w = wk.random_small(4, 4, 2, seed=3, n_vortices=1)
    return w, 1.3, np.full(w.V, -0.2), w.Delta.copy()


def test_resume_matches_uninterrupted_run(tmp_path):
    w, g, U, D = _case()
    it_ref, _, U_ref, D_ref, ok_ref = fno.scf_solve(FakeScf(), w, g, U, D, tol=1e-10, max_iter=200,
                                                    alpha=0.5, device="cpu")
    assert ok_ref and it_ref > 10
    ck = str(tmp_path / "state.npz")
    first = FakeScf()
    it1, _, _, _, ok1 = fno.scf_solve(first, w, g, U, D, tol=1e-10, max_iter=7, alpha=0.5,
                                      checkpoint=ck, device="cpu")      # interrupted after 7 steps
    assert (it1, ok1, first.calls) == (7, False, 7)
    st = scf_state.load(ck)
    assert st["iteration"] == 7 and len(st["dn_history"]) == 7 and not st["converged"]
    second = FakeScf()
    it2, _, U2, D2, ok2 = fno.scf_solve(second, w, g, U, D, tol=1e-10, max_iter=200, alpha=0.5,
                                        checkpoint=ck, device="cpu")
    assert ok2 and it2 == it_ref and second.calls == it_ref - 7
    assert np.array_equal(U2, U_ref) and np.array_equal(D2, D_ref)
    # a converged checkpoint returns at once
    third = FakeScf()
    it3, _, U3, _, ok3 = fno.scf_solve(third, w, g, U, D, tol=1e-10, max_iter=200, alpha=0.5,
                                       checkpoint=ck, device="cpu")
    assert ok3 and it3 == it_ref and third.calls == 0 and np.array_equal(U3, U_ref)
    # a tighter tolerance than the one it converged to resumes the loop
    fourth = FakeScf()
    _, _, _, _, ok4 = fno.scf_solve(fourth, w, g, U, D, tol=1e-14, max_iter=400, alpha=0.5,
                                    checkpoint=ck, device="cpu")
    assert fourth.calls > 0 and ok4


def test_checkpoint_of_another_problem_is_refused(tmp_path):
    w, g, U, D = _case()
    ck = str(tmp_path / "state.npz")
    fno.scf_solve(FakeScf(), w, g, U, D, tol=1e-10, max_iter=3, alpha=0.5, checkpoint=ck, device="cpu")
    with pytest.raises(ValueError, match="checkpoint is for"):
        fno.scf_solve(FakeScf(), w, g * 1.01, U, D, tol=1e-10, max_iter=5, alpha=0.5, checkpoint=ck,
                      device="cpu")
    with pytest.raises(ValueError, match="checkpoint is for"):
        fno.scf_solve(FakeScf(), w, g, U, D, tol=1e-10, max_iter=5, alpha=0.7, checkpoint=ck, device="cpu")


def test_checkpoint_write_is_atomic_and_validated(tmp_path):
    w, g, U, D = _case()
    ck = str(tmp_path / "sub" / "state.npz")
    scf_state.save(ck, U=U, Delta=D, n_prev=np.zeros(w.V), grid=(w.nx, w.ny, w.nz), mu=w.mu, g=g,
                   alpha=0.5, tol=1e-6, iteration=2, converged=False, dn_history=[0.3, 0.1])
    assert os.listdir(tmp_path / "sub") == ["state.npz"]       # no temporary file left behind
    st = scf_state.load(ck)
    assert np.array_equal(st["Delta"], D) and st["grid"] == (w.nx, w.ny, w.nz)
    bad = str(tmp_path / "bad.npz")
    np.savez(bad, U=U, Delta=D[:-1], n_prev=np.zeros(w.V), grid=np.array([w.nx, w.ny, w.nz]), mu=0.5, g=g,
             alpha=0.5, tol=1e-6, iteration=1, converged=False, dn_history=np.zeros(1))
    with pytest.raises(ValueError, match="field Delta"):
        scf_state.load(bad)
    np.savez(bad, U=U)
    with pytest.raises(ValueError, match="not an SCF checkpoint"):
        scf_state.load(bad)


def test_non_finite_step_stops_the_loop_and_keeps_the_last_finite_checkpoint(tmp_path):
    """Fault injected on the host: the step poisons U with NaN at step 5."""
    w, g, U, D = _case()

    class Poisoned(FakeScf):
        def scf_step(self, grid, U, D, n_prev, *a, **k):
            if self.calls == 4:
                U[0] = float("nan")
            return super().scf_step(grid, U, D, n_prev, *a, **k)

    ck = str(tmp_path / "state.npz")
    with pytest.raises(FloatingPointError, match="SCF step 5"):
        fno.scf_solve(Poisoned(), w, g, U, D, tol=1e-10, max_iter=50, alpha=0.5, checkpoint=ck, device="cpu")
    st = scf_state.load(ck)
    assert st["iteration"] == 4 and np.all(np.isfinite(st["U"])) and np.all(np.isfinite(st["dn_history"]))
