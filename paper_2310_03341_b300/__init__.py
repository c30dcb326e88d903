"""Python binding of libbdg, the B300 (sm_103a) dense BdG eigensolver.

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libbdg.so`` (built from ``csrc/`` by ``build.py``).  PyTorch
provides device memory and the current stream.  There is no CPU fallback:
if the library is missing or no CUDA device is present the calls raise.

Matrix convention: the library is column-major.  A column-major N x N buffer
is exposed to torch as ``buf.mT`` of a contiguous (N, N) tensor ``buf``, so
``Z[:, j]`` is eigenvector j.  ``colmajor()`` converts any torch matrix into
that layout.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbdg.so")

BDG_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENOCONV", -5: "ETIMEOUT", -6: "EUNSUPPORTED"}
ERRORS_BY_NAME = {v: k for k, v in ERRORS.items()}
PREC = {"fp64": 0, "fp32": 1, "bf16x3": 2, "bf16x6": 3, "bf16x9": 4}
HEEV_PH = 0x100   # BDG_HEEV_PH
EXPORTS = ("bdg_create", "bdg_destroy", "bdg_last_error", "bdg_build", "bdg_heev_workspace", "bdg_heev",
           "bdg_refine", "bdg_densities", "bdg_scf_step", "bdg_heev_batched", "bdg_set_timing", "bdg_stage_times",
           "bdg_launch_count", "bdg_densities_noalloc", "bdg_last_modes", "bdg_fno_sizes", "bdg_fno_forward",
           "bdg_fno_backward", "bdg_fno_mse", "bdg_fno_adam", "bdg_kinetic_current_densities", "bdg_set_wait_limit", "bdg_td_evolve", "bdg_gap_coupling")

_lib = None


class BdgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx", C.c_double)]


class FnoConfig(C.Structure):
    _fields_ = [("g", C.c_int), ("width", C.c_int), ("modes", C.c_int), ("layers", C.c_int), ("cin", C.c_int),
                ("cout", C.c_int), ("bf16_weights", C.c_int)]


class TdParams(C.Structure):
    _fields_ = [("mu", C.c_double), ("g", C.c_double), ("T", C.c_double), ("dt", C.c_double),
                ("U_ext", C.c_void_p)]


class ScfParams(C.Structure):
    _fields_ = [("mu", C.c_double), ("g", C.c_double), ("alpha", C.c_double), ("T", C.c_double),
                ("Ec", C.c_double), ("prec", C.c_int), ("refine_iters", C.c_int), ("refine_tol", C.c_double),
                ("phase", C.c_void_p), ("n_prev", C.c_void_p)]


def lib():
    """Load libbdg.so (building it first if the sources are newer)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            from . import build as _b
            _b.build()
        L = C.CDLL(LIB_PATH)
        P, i64 = C.c_void_p, C.c_int64
        L.bdg_create.argtypes = [C.c_int, C.POINTER(P)]
        L.bdg_destroy.argtypes = [P]
        L.bdg_destroy.restype = None
        L.bdg_last_error.argtypes = [P]
        L.bdg_last_error.restype = C.c_char_p
        L.bdg_build.argtypes = [P, C.POINTER(Grid), C.c_double, P, P, P, i64, P]
        L.bdg_heev_workspace.argtypes = [P, i64, C.c_int, C.POINTER(C.c_size_t)]
        L.bdg_heev.argtypes = [P, i64, P, i64, P, P, i64, C.c_int, P]
        L.bdg_refine.argtypes = [P, C.POINTER(Grid), C.c_double, P, P, i64, P, P, i64, C.c_int, C.c_double,
                                 C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int), P]
        L.bdg_densities.argtypes = [P, C.POINTER(Grid), i64, P, P, i64, C.c_double, C.c_double, P, P, P]
        L.bdg_kinetic_current_densities.argtypes = [P, C.POINTER(Grid), i64, P, P, i64, C.c_double, C.c_double,
                                                     P, P, P]
        L.bdg_densities_noalloc.argtypes = [C.POINTER(Grid), i64, P, P, i64, C.c_double, C.c_double, P, P, P,
                                             C.c_char_p, C.c_size_t]
        L.bdg_scf_step.argtypes = [P, C.POINTER(Grid), C.POINTER(ScfParams), P, P, C.POINTER(C.c_double), P]
        L.bdg_heev_batched.argtypes = [P, C.c_int, C.POINTER(i64), C.POINTER(P), C.POINTER(P), C.POINTER(P),
                                       C.c_int, P]
        L.bdg_set_timing.argtypes = [P, C.c_int]
        L.bdg_set_wait_limit.argtypes = [P, C.c_longlong]
        L.bdg_gap_coupling.argtypes = [C.POINTER(Grid), C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double),
                                       C.POINTER(C.c_double)]
        L.bdg_td_evolve.argtypes = [P, C.POINTER(Grid), C.POINTER(TdParams), i64, P, P, i64, C.c_int, P, P, P]
        L.bdg_launch_count.argtypes = [P, C.POINTER(C.c_longlong)]
        L.bdg_last_modes.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.bdg_fno_sizes.argtypes = [C.POINTER(FnoConfig), C.c_int, C.POINTER(i64), C.POINTER(i64)]
        L.bdg_fno_forward.argtypes = [P, C.POINTER(FnoConfig), C.c_int, P, P, P, P, P]
        L.bdg_fno_backward.argtypes = [P, C.POINTER(FnoConfig), C.c_int, P, P, P, P, P, P]
        L.bdg_fno_mse.argtypes = [P, i64, P, P, P, P, P]
        L.bdg_fno_adam.argtypes = [P, i64, P, P, P, P, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int, P]
        L.bdg_stage_times.argtypes = [P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_char_p), C.POINTER(C.c_int)]
        for name in EXPORTS:
            if name not in ("bdg_destroy", "bdg_last_error"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _ptr(t: torch.Tensor):
    return C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def colmajor(M: torch.Tensor) -> torch.Tensor:
    """Same matrix, stored column-major (returned as the .mT view of a contiguous buffer)."""
    if M.dim() == 2 and M.stride(0) == 1 and M.stride(1) == M.shape[0]:
        return M
    return M.mT.contiguous().mT


def _buf(M: torch.Tensor) -> torch.Tensor:
    """The contiguous buffer behind a column-major view."""
    assert M.stride(0) == 1 and M.stride(1) == M.shape[0], "matrix must be column-major (use colmajor())"
    return M.mT


def gap_coupling(grid, mu, delta0, Ec=None):
    """bdg_gap_coupling: (g, U0) of the contact functional that make the uniform state with gap
    delta0 self-consistent (host computation in the library; no device needed)."""
    import math
    g = Grid(*grid, 1.0)
    go, uo = C.c_double(), C.c_double()
    rc = lib().bdg_gap_coupling(C.byref(g), float(mu), float(delta0), math.pi ** 2 / 2 if Ec is None else float(Ec),
                                C.byref(go), C.byref(uo))
    if rc != BDG_OK:
        raise BdgError(rc, "bdg_gap_coupling: no solution for these arguments")
    return go.value, uo.value


def densities_noalloc(grid, w, Z, n_out, nu_out, T=0.0, Ec=None, stream=None):
    """bdg_densities_noalloc: the densities into caller-owned ``n_out`` (V
    float64) and ``nu_out`` (V complex128) without any device allocation
    (library-internal fixed scratch; V <= 174720).  ``Z`` must already be
    column-major (``colmajor()`` would allocate); only its columns with
    0 < w < Ec are read.  Every tensor must be on one device; the call runs
    there.  Calls that overlap on one device race on the shared scratch."""
    import math
    g = Grid(*grid, 1.0)
    V = grid[0] * grid[1] * grid[2]
    n = w.shape[0]
    dev = w.device
    if dev.type != "cuda" or any(t.device != dev for t in (Z, n_out, nu_out)):
        raise ValueError("densities_noalloc: w, Z, n_out and nu_out must be on one CUDA device")
    if w.dtype != torch.float64 or w.dim() != 1 or n != 2 * V or not w.is_contiguous():
        raise ValueError(f"densities_noalloc: w must be a contiguous float64 vector of 2V = {2 * V} entries")
    if Z.dtype != torch.complex128 or Z.dim() != 2 or Z.shape[0] != n:
        raise ValueError(f"densities_noalloc: Z must be complex128 with {n} rows")
    if n_out.dtype != torch.float64 or n_out.numel() != V or not n_out.is_contiguous():
        raise ValueError(f"densities_noalloc: n_out must be a contiguous float64 tensor of V = {V} entries")
    if nu_out.dtype != torch.complex128 or nu_out.numel() != V or not nu_out.is_contiguous():
        raise ValueError(f"densities_noalloc: nu_out must be a contiguous complex128 tensor of V = {V} entries")
    Ec = math.pi ** 2 / 2 if Ec is None else Ec
    msg = C.create_string_buffer(256)
    with torch.cuda.device(dev):
        st = _stream() if stream is None else C.c_void_p(stream.cuda_stream)
        rc = lib().bdg_densities_noalloc(C.byref(g), n, _ptr(w), _ptr(_buf(Z)), n, float(T), float(Ec),
                                         _ptr(n_out), _ptr(nu_out), st, msg, 256)
    if rc != BDG_OK:
        raise BdgError(rc, msg.value.decode())


class Context:
    """A libbdg context on one CUDA device (owns the device workspace)."""

    def __init__(self, device: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("libbdg needs a CUDA device; no CPU fallback exists")
        self.device = device
        self._h = C.c_void_p()
        rc = lib().bdg_create(device, C.byref(self._h))
        if rc != BDG_OK:
            raise BdgError(rc, "bdg_create failed")

    def close(self):
        if self._h:
            lib().bdg_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != BDG_OK:
            raise BdgError(rc, lib().bdg_last_error(self._h).decode())

    # -- instrumentation -----------------------------------------------------
    def set_timing(self, enable: bool = True):
        self._check(lib().bdg_set_timing(self._h, 1 if enable else 0))

    def set_wait_limit(self, cycles: int = 0):
        """Cap every bounded device wait of this context at `cycles` SM clock cycles (0: default)."""
        self._check(lib().bdg_set_wait_limit(self._h, int(cycles)))

    def launch_count(self) -> int:
        out = C.c_longlong()
        self._check(lib().bdg_launch_count(self._h, C.byref(out)))
        return out.value

    def last_modes(self):
        """(heev_ph, refine_ph): whether the last heev / refine used the particle-hole reduction."""
        a, b = C.c_int(), C.c_int()
        self._check(lib().bdg_last_modes(self._h, C.byref(a), C.byref(b)))
        return bool(a.value), bool(b.value)

    # -- Fourier neural operator (learned SCF initial guess) ------------------
    def fno_sizes(self, cfg: "FnoConfig", batch: int):
        npar, ncache = C.c_int64(), C.c_int64()
        self._check(lib().bdg_fno_sizes(C.byref(cfg), int(batch), C.byref(npar), C.byref(ncache)))
        return npar.value, ncache.value

    def fno_forward(self, cfg, params, inp, cache=None):
        """inp (B, X, cin) float32 -> (out (B, X, cout), cache)."""
        B = inp.shape[0]
        _, nc = self.fno_sizes(cfg, B)
        if cache is None or cache.numel() < nc:
            cache = torch.empty(nc, dtype=torch.float32, device=inp.device)
        out = torch.empty(B, inp.shape[1], cfg.cout, dtype=torch.float32, device=inp.device)
        self._check(lib().bdg_fno_forward(self._h, C.byref(cfg), B, _ptr(params), _ptr(inp), _ptr(out), _ptr(cache),
                                          _stream()))
        return out, cache

    def fno_backward(self, cfg, params, inp, cache, dout, grad=None):
        if grad is None:
            grad = torch.empty_like(params)
        self._check(lib().bdg_fno_backward(self._h, C.byref(cfg), inp.shape[0], _ptr(params), _ptr(inp), _ptr(cache),
                                           _ptr(dout), _ptr(grad), _stream()))
        return grad

    def fno_mse(self, y, target, dy=None, loss=None):
        if dy is None:
            dy = torch.empty_like(y)
        if loss is None:
            loss = torch.empty(1, dtype=torch.float32, device=y.device)
        self._check(lib().bdg_fno_mse(self._h, y.numel(), _ptr(y), _ptr(target), _ptr(dy), _ptr(loss), _stream()))
        return loss, dy

    def fno_adam(self, params, grad, m1, m2, lr, step, beta1=0.9, beta2=0.999, eps=1e-8):
        self._check(lib().bdg_fno_adam(self._h, params.numel(), _ptr(params), _ptr(grad), _ptr(m1), _ptr(m2),
                                       float(lr), float(beta1), float(beta2), float(eps), int(step), _stream()))

    def stage_times(self):
        """[(stage, ms)] of the last bdg_heev / bdg_refine call with timing enabled."""
        ms = (C.c_double * 64)()
        names = (C.c_char_p * 64)()
        cnt = C.c_int()
        self._check(lib().bdg_stage_times(self._h, 64, ms, names, C.byref(cnt)))
        return [(names[i].decode(), ms[i]) for i in range(cnt.value)]

    # -- entry points --------------------------------------------------------
    def build(self, grid, mu, U: torch.Tensor, Delta: torch.Tensor) -> torch.Tensor:
        """Dense H (N x N complex128, column-major view) of Eq. (stHpsi)."""
        g = Grid(*grid, 1.0)
        N = 2 * grid[0] * grid[1] * grid[2]
        buf = torch.empty(N, N, dtype=torch.complex128, device=U.device)
        self._check(lib().bdg_build(self._h, C.byref(g), float(mu), _ptr(U), _ptr(Delta), _ptr(buf), N,
                                    _stream()))
        return buf.mT

    def heev_workspace(self, n: int, prec: str = "fp64") -> int:
        out = C.c_size_t()
        self._check(lib().bdg_heev_workspace(self._h, n, PREC[prec], C.byref(out)))
        return out.value

    def heev(self, A: torch.Tensor, prec: str = "fp64", overwrite: bool = False, ph: bool = False):
        """All eigenpairs of the Hermitian A -> (w ascending, Z column-major).
        ph=True asserts that A is a BdG matrix (particle-hole half solve)."""
        n = A.shape[0]
        A = colmajor(A)
        if not overwrite:
            A = A.mT.clone().mT
        w = torch.empty(n, dtype=torch.float64, device=A.device)
        zb = torch.empty(n, n, dtype=torch.complex128, device=A.device)
        code = PREC[prec] | (HEEV_PH if ph else 0)
        self._check(lib().bdg_heev(self._h, n, _ptr(_buf(A)), n, _ptr(w), _ptr(zb), n, code, _stream()))
        return w, zb.mT

    def refine(self, grid, mu, U, Delta, w: torch.Tensor, Z: torch.Tensor, max_iter=3, tol=1e-11, orth=True):
        """In-place Ogita-Aishima refinement of (w, Z) -> (resid, orth, iters, converged).
        With orth=False the final Gram matrix is not formed and orth is None."""
        g = Grid(*grid, 1.0)
        n = w.shape[0]
        r, o, it = C.c_double(), C.c_double(), C.c_int()
        rc = lib().bdg_refine(self._h, C.byref(g), float(mu), _ptr(U), _ptr(Delta), n, _ptr(w), _ptr(_buf(Z)), n,
                              int(max_iter), float(tol), C.byref(r), C.byref(o) if orth else None, C.byref(it),
                              _stream())
        if rc not in (BDG_OK, -4):
            self._check(rc)
        return r.value, (o.value if orth else None), it.value, rc == BDG_OK

    def kinetic_current_densities(self, grid, w, Z, T=0.0, Ec=None):
        """bdg_kinetic_current_densities: (tau (V,), j (3, V)) float64 on the device of w."""
        import math
        g = Grid(*grid, 1.0)
        n = w.shape[0]
        V = n // 2
        Ec = math.pi ** 2 / 2 if Ec is None else Ec
        tau = torch.empty(V, dtype=torch.float64, device=w.device)
        j = torch.empty(3, V, dtype=torch.float64, device=w.device)
        self._check(lib().bdg_kinetic_current_densities(self._h, C.byref(g), n, _ptr(w), _ptr(_buf(Z)), n,
                                                        float(T), float(Ec), _ptr(tau), _ptr(j), _stream()))
        return tau, j

    def densities(self, grid, w, Z, T=0.0, Ec=None):
        import math
        g = Grid(*grid, 1.0)
        n = w.shape[0]
        V = n // 2
        Ec = math.pi ** 2 / 2 if Ec is None else Ec
        nd = torch.empty(V, dtype=torch.float64, device=w.device)
        nu = torch.empty(V, dtype=torch.complex128, device=w.device)
        self._check(lib().bdg_densities(self._h, C.byref(g), n, _ptr(w), _ptr(_buf(Z)), n, float(T), float(Ec),
                                        _ptr(nd), _ptr(nu), _stream()))
        return nd, nu

    def scf_step(self, grid, U, Delta, n_prev, mu, g, alpha=0.3, T=0.0, Ec=None, prec="fp64", refine_iters=2,
                 refine_tol=1e-11, phase=None):
        import math
        gr = Grid(*grid, 1.0)
        p = ScfParams(float(mu), float(g), float(alpha), float(T), math.pi ** 2 / 2 if Ec is None else float(Ec),
                      PREC[prec], int(refine_iters), float(refine_tol),
                      C.c_void_p(phase.data_ptr()) if phase is not None else None, C.c_void_p(n_prev.data_ptr()))
        dn = C.c_double()
        self._check(lib().bdg_scf_step(self._h, C.byref(gr), C.byref(p), _ptr(U), _ptr(Delta), C.byref(dn),
                                       _stream()))
        return dn.value

    def td_evolve(self, grid, E0: torch.Tensor, Psi: torch.Tensor, dt: float, nsteps: int, mu: float, g: float,
                  T: float = 0.0, U_ext: torch.Tensor = None, densities: bool = True):
        """bdg_td_evolve: evolve the states Psi (2V x nq, column-major view, updated in place) for nsteps
        steps of dt -> (n, nu) at the final time (None when densities=False)."""
        gr = Grid(*grid, 1.0)
        V = grid[0] * grid[1] * grid[2]
        nq = E0.shape[0]
        assert Psi.shape == (2 * V, nq) and Psi.dtype == torch.complex128
        p = TdParams(float(mu), float(g), float(T), float(dt), C.c_void_p(U_ext.data_ptr()) if U_ext is not None
                     else None)
        nd = nu = None
        if densities:
            nd = torch.empty(V, dtype=torch.float64, device=E0.device)
            nu = torch.empty(V, dtype=torch.complex128, device=E0.device)
        self._check(lib().bdg_td_evolve(self._h, C.byref(gr), C.byref(p), nq, _ptr(E0), _ptr(_buf(Psi)), 2 * V,
                                        int(nsteps), _ptr(nd) if densities else None,
                                        _ptr(nu) if densities else None, _stream()))
        return nd, nu

    def heev_batched(self, blocks, prec: str = "fp64", ph: bool = False, overwrite: bool = False):
        """bdg_heev_batched: blocks is a list of Hermitian matrices of any sizes -> list of (w, Z).
        ph=True asserts that every block is a BdG matrix (particle-hole half solve per block)."""
        sizes, As, ws, zs, keep = [], [], [], [], []
        for A in blocks:
            n = A.shape[0]
            Ac = colmajor(A)
            if not overwrite or Ac is not A:
                Ac = Ac.mT.clone().mT if Ac is A else Ac
            w = torch.empty(n, dtype=torch.float64, device=A.device)
            zb = torch.empty(n, n, dtype=torch.complex128, device=A.device)
            keep += [Ac, w, zb]
            sizes.append(n)
            As.append(_buf(Ac).data_ptr())
            ws.append(w.data_ptr())
            zs.append(zb.data_ptr())
        nb = len(blocks)
        arr = lambda xs, t: (t * nb)(*xs)
        code = PREC[prec] | (HEEV_PH if ph else 0)
        self._check(lib().bdg_heev_batched(self._h, nb, arr(sizes, C.c_int64), arr(As, C.c_void_p),
                                           arr(ws, C.c_void_p), arr(zs, C.c_void_p), code, _stream()))
        return [(keep[3 * i + 1], keep[3 * i + 2].mT) for i in range(nb)]

    def build_kz_blocks(self, grid2d, mu, U2d, Delta2d, kz):
        """The kz blocks H_kz = H_perp + (kz^2/2) tau_z of a z-invariant system, each built by
        bdg_build on the (nx, ny, 1) grid with mu - kz^2/2 (tau_z = +1 on u, -1 on v)."""
        nx, ny = grid2d
        return [self.build((nx, ny, 1), float(mu) - 0.5 * float(k) ** 2, U2d, Delta2d) for k in kz]
