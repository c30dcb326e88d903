"""Helpers shared by the GPU parity tests: run the CUDA path and the oracle on
the same seeded inputs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def have_gpu():
    return torch.cuda.is_available()


_ctx = None


def ctx():
    global _ctx
    import paper_2310_03341_b300 as bdg
    if _ctx is None:
        _ctx = bdg.Context(0)
    return _ctx


def dev_fields(w):
    U = torch.tensor(w.U, dtype=torch.float64, device="cuda")
    D = torch.tensor(w.Delta, dtype=torch.complex128, device="cuda")
    return U, D


def gpu_eig(w, prec, refine=0, tol=1e-12, ph=False):
    U, D = dev_fields(w)
    c = ctx()
    H = c.build((w.nx, w.ny, w.nz), w.mu, U, D)
    ev, Z = c.heev(H, prec, overwrite=True, ph=ph)
    info = None
    if refine:
        info = c.refine((w.nx, w.ny, w.nz), w.mu, U, D, ev, Z, refine, tol)
    torch.cuda.synchronize()
    return ev.cpu().numpy(), Z.cpu().numpy(), info


def isolated(ev, rel=1e-6):
    rho = np.max(np.abs(ev))
    gl = np.abs(np.diff(ev, prepend=-np.inf))
    gr = np.abs(np.diff(ev, append=np.inf))
    return np.nonzero(np.minimum(gl, gr) > rel * rho)[0]
