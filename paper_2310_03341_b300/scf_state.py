"""Checkpoints of the self-consistent loop: the fields and counters of a run of bdg_scf_step,
saved after each step as one .npz file, so that an interrupted loop resumes where it stopped
(the same U, Delta and previous density, the same iteration count and residual history) and the
converged states of a data-generation run can be collected without repeating finished work.

A checkpoint holds
  U (V float64), Delta (V complex128), n_prev (V float64)   the loop's fields after `iteration`
                                                            steps (n_prev: the density of the
                                                            last step, which the next step's
                                                            max|dn| is measured against);
  grid (3 ints), mu, g, alpha, tol                          the problem and loop parameters;
  iteration, converged, dn_history                          the counters.
It is written to a temporary file in the same directory and renamed over the old one, so an
interruption during the write leaves the previous checkpoint intact.
"""
from __future__ import annotations

import os

import numpy as np

_KEYS = ("U", "Delta", "n_prev", "grid", "mu", "g", "alpha", "tol", "iteration", "converged",
         "dn_history")


def save(path: str, *, U, Delta, n_prev, grid, mu: float, g: float, alpha: float, tol: float,
         iteration: int, converged: bool, dn_history) -> None:
    """Write one checkpoint atomically (host arrays or tensors on any device)."""
    def host(x, dtype):
        x = x.detach().cpu().numpy() if hasattr(x, "detach") else np.asarray(x)
        return np.ascontiguousarray(x, dtype=dtype).reshape(-1)

    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    tmp = os.path.join(d, f".{os.path.basename(path)}.{os.getpid()}.tmp")
    with open(tmp, "wb") as f:
        np.savez(f, U=host(U, np.float64), Delta=host(Delta, np.complex128),
                 n_prev=host(n_prev, np.float64), grid=np.asarray(grid, dtype=np.int64),
                 mu=np.float64(mu), g=np.float64(g), alpha=np.float64(alpha), tol=np.float64(tol),
                 iteration=np.int64(iteration), converged=np.bool_(converged),
                 dn_history=np.asarray(dn_history, dtype=np.float64))
        f.flush()
        os.fsync(f.fileno())
    os.replace(tmp, path)


def load(path: str) -> dict:
    """Read a checkpoint; raises ValueError if a field is missing or has the wrong length."""
    with np.load(path) as z:
        missing = [k for k in _KEYS if k not in z.files]
        if missing:
            raise ValueError(f"{path}: not an SCF checkpoint (missing {', '.join(missing)})")
        st = {k: z[k] for k in _KEYS}
    V = int(np.prod(st["grid"]))
    for k in ("U", "Delta", "n_prev"):
        if st[k].shape != (V,):
            raise ValueError(f"{path}: field {k} has {st[k].size} entries, the grid has {V} sites")
    for k in ("mu", "g", "alpha", "tol"):
        st[k] = float(st[k])
    st["iteration"] = int(st["iteration"])
    st["converged"] = bool(st["converged"])
    st["grid"] = tuple(int(x) for x in st["grid"])
    st["dn_history"] = [float(x) for x in st["dn_history"]]
    return st


def check_matches(st: dict, grid, mu: float, g: float, alpha: float) -> None:
    """Refuse to resume a checkpoint of another problem or another mixing."""
    want = (tuple(int(x) for x in grid), float(mu), float(g), float(alpha))
    have = (st["grid"], st["mu"], st["g"], st["alpha"])
    if want != have:
        raise ValueError(f"checkpoint is for (grid, mu, g, alpha) = {have}, not {want}")
