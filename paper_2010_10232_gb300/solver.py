"""Python binding of the C ABI: argument marshalling only.

Every computation happens in the CUDA library; this module converts torch
tensors (complex128, on the context's device) to pointers and raises on error
status.  PyTorch provides device memory and the stream.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _ffi


class IgaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_ffi.STATUS.get(status, status)}: {msg}")
        self.status = status


def _ptr(t: torch.Tensor) -> int:
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("tensor must be contiguous and on the CUDA device")
    return t.data_ptr()


class Helmholtz:
    """One IgA Helmholtz problem on the unit interval/square (homogeneous
    Dirichlet data), set up on the current CUDA device and stream.

    kfield: either a number (constant k) or an object with ``values`` (k per
    layer) and ``lines`` (each with a, b, c: layer index = number of lines with
    a*x + b*y + c >= 0)."""

    def __init__(self, dim=2, p=3, n_el=32, kfield=10.0, beta=(1.0, 0.5), eps=0.0, nu_pre=1, nu_post=1,
                 omega=0.6, n_vcycles=1, precision=0, flexible=0, skip_deflation=0, host_loop=0, arnoldi=None,
                 fused_vcycle=0, stream=None, precond=0, deflation=1, robin=0):
        self._L = _ffi.lib()
        prm = _ffi.IgaParams()
        self._L.iga_default_params(C.byref(prm))
        prm.dim, prm.p, prm.n_el = int(dim), int(p), int(n_el)
        if isinstance(kfield, (int, float)):
            prm.n_lines = 0
            prm.k_values[0] = float(kfield)
        else:
            lines = list(kfield.lines)
            vals = list(kfield.values)
            if len(lines) > _ffi.IGA_MAX_LINES or len(vals) != len(lines) + 1:
                raise ValueError("bad k field description")
            prm.n_lines = len(lines)
            for i, ln in enumerate(lines):
                prm.lines[i][0], prm.lines[i][1], prm.lines[i][2] = float(ln.a), float(ln.b), float(ln.c)
            for i, v in enumerate(vals):
                prm.k_values[i] = float(v)
        prm.beta1, prm.beta2 = float(beta[0]), float(beta[1])
        prm.eps = float(eps)
        prm.nu_pre, prm.nu_post = int(nu_pre), int(nu_post)
        prm.omega = float(omega)
        prm.n_vcycles = int(n_vcycles)
        prm.precision = int(precision)
        prm.flexible = int(flexible)
        prm.skip_deflation = int(skip_deflation)
        prm.host_loop = int(host_loop)
        if arnoldi is not None:
            prm.arnoldi = int(arnoldi)
        prm.fused_vcycle = int(fused_vcycle)
        prm.precond = int(precond)
        prm.deflation = int(deflation)
        prm.robin = int(robin)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        prm.stream = C.c_void_p(stream.cuda_stream)
        self.params = prm
        self.device = torch.device("cuda", torch.cuda.current_device())
        h = C.c_void_p()
        st = self._L.iga_setup(C.byref(prm), C.byref(h))
        if st != 0:
            raise IgaError(st, "iga_setup failed (see stderr)")
        self._h = h
        self.n = int(self._L.iga_ndof(h))
        self.m = int(self._L.iga_coarse_ndof(h))
        self.levels = int(self._L.iga_num_levels(h))
        self.dim, self.p, self.n_el = int(dim), int(p), int(n_el)

    # ------------------------------------------------------------ plumbing
    def close(self):
        if getattr(self, "_h", None):
            self._L.iga_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st < 0:
            raise IgaError(st, self._L.iga_last_error(self._h).decode())
        return st

    def vec(self, n=None):
        return torch.zeros(self.n if n is None else n, dtype=torch.complex128, device=self.device)

    def level_nx(self, level: int) -> int:
        return int(self._L.iga_level_nx(self._h, level))

    def tile(self, level: int, precision: int = 0) -> int:
        return int(self._L.iga_tile_choice(self._h, level, precision))

    def set_tile(self, level: int, precision: int, tile: int) -> None:
        self._check(self._L.iga_set_tile(self._h, level, precision, tile))

    def level_n(self, level: int) -> int:
        return self.level_nx(level) ** self.dim

    def level_nel(self, level: int) -> int:
        return int(self._L.iga_level_nel(self._h, level))

    # ------------------------------------------------------------ setup queries
    def knots(self, level: int = 0) -> np.ndarray:
        n = self.level_nel(level) + 2 * self.p + 1
        out = np.zeros(n)
        self._check(self._L.iga_get_knots(self._h, level, out.ctypes.data, n))
        return out

    def band(self, level: int, which: int) -> np.ndarray:
        nx = self.level_nx(level)
        out = np.zeros(nx * (2 * self.p + 1))
        self._check(self._L.iga_get_band(self._h, level, which, out.ctypes.data, out.size))
        return out.reshape(nx, 2 * self.p + 1)

    def prolongation(self, level: int) -> np.ndarray:
        nf, nc = self.level_nx(level), self.level_nx(level + 1)
        out = np.zeros(nf * nc)
        self._check(self._L.iga_get_prolongation(self._h, level, out.ctypes.data, out.size))
        return out.reshape(nf, nc)

    # ------------------------------------------------------------ operators
    def apply_A(self, x, y=None):
        y = self.vec() if y is None else y
        self._check(self._L.iga_apply_A(self._h, _ptr(x), _ptr(y)))
        return y

    def apply_Mshift(self, level, x, y=None):
        y = self.vec(self.level_n(level)) if y is None else y
        self._check(self._L.iga_apply_Mshift(self._h, level, _ptr(x), _ptr(y)))
        return y

    def jacobi(self, level, b, x, sweeps=1):
        xin = x.clone()
        out = torch.empty_like(x)
        self._check(self._L.iga_jacobi(self._h, level, _ptr(b), _ptr(xin), _ptr(out), int(sweeps)))
        return out

    def vec32(self, n=None):
        return torch.zeros(self.n if n is None else n, dtype=torch.complex64, device=self.device)

    def apply_Mshift32(self, level, x, y=None):
        y = self.vec32(self.level_n(level)) if y is None else y
        self._check(self._L.iga_apply_Mshift32(self._h, level, _ptr(x), _ptr(y)))
        return y

    def jacobi32(self, level, b, x, out=None):
        out = torch.empty_like(x) if out is None else out
        self._check(self._L.iga_jacobi32(self._h, level, _ptr(b), _ptr(x), _ptr(out)))
        return out

    def restrict(self, level, fine):
        c = self.vec(self.level_n(level + 1))
        self._check(self._L.iga_restrict(self._h, level, _ptr(fine), _ptr(c)))
        return c

    def prolong_add(self, level, coarse, fine):
        self._check(self._L.iga_prolong_add(self._h, level, _ptr(coarse), _ptr(fine)))
        return fine

    def coarse_solve(self, b):
        x = torch.empty_like(b)
        self._check(self._L.iga_coarse_solve(self._h, _ptr(b), _ptr(x)))
        return x

    def vcycle(self, r, z=None):
        z = self.vec() if z is None else z
        self._check(self._L.iga_vcycle_cslp(self._h, _ptr(r), _ptr(z)))
        return z

    def precond(self, r, z=None):
        """z = M~^{-1} r as the solve applies it (V-cycles, exact CSLP or identity)."""
        z = self.vec() if z is None else z
        self._check(self._L.iga_precond(self._h, _ptr(r), _ptr(z)))
        return z

    def set_wait_limit(self, polls=0, phantom_arrivals=0):
        self._check(self._L.iga_set_wait_limit(self._h, int(polls), int(phantom_arrivals)))

    def zt(self, x):
        c = self.vec(self.m)
        self._check(self._L.iga_zt(self._h, _ptr(x), _ptr(c)))
        return c

    def z(self, c):
        x = self.vec()
        self._check(self._L.iga_z(self._h, _ptr(c), _ptr(x)))
        return x

    def esolve(self, t):
        s = self.vec(self.m)
        self._check(self._L.iga_esolve(self._h, _ptr(t), _ptr(s)))
        return s

    def deflate(self, x, y=None):
        y = self.vec() if y is None else y
        self._check(self._L.iga_deflate(self._h, _ptr(x), _ptr(y)))
        return y

    def point_source(self, x0, y0=0.5, f=None):
        f = self.vec() if f is None else f
        self._check(self._L.iga_load_point_source(self._h, float(x0), float(y0), _ptr(f)))
        return f

    def dirichlet_load(self, g=1.0, f=None):
        """Right-hand side of u(0) = g for an MP 1-A context (robin = 1)."""
        f = self.vec() if f is None else f
        g = complex(g)
        self._check(self._L.iga_load_dirichlet(self._h, g.real, g.imag, _ptr(f)))
        return f

    def mgs(self, V, j, w):
        """V: (k, n) complex128 rows = basis vectors; w updated in place."""
        h = self.vec(j + 2)
        self._check(self._L.iga_mgs(self._h, _ptr(V), V.shape[1], int(j), _ptr(w), _ptr(h)))
        return h

    # ------------------------------------------------------------ solve
    def solve(self, f, tol=1e-7, maxit=100, x=None):
        """Returns (x, iters, res_hist (numpy), true_res, status)."""
        x = self.vec() if x is None else x
        iters = C.c_int(0)
        hist = np.zeros(maxit + 1)
        tr = C.c_double(0.0)
        st = self._check(self._L.iga_solve(self._h, _ptr(f), _ptr(x), float(tol), int(maxit), C.byref(iters),
                                           hist.ctypes.data, C.byref(tr)))
        return x, iters.value, hist[:iters.value + 1], tr.value, st

    def solve_host(self, f: np.ndarray, tol=1e-7, maxit=100):
        """Host-memory solve: f (numpy complex128) -> x (numpy complex128); the
        copies to and from the device are part of the call."""
        f = np.ascontiguousarray(f, dtype=np.complex128)
        x = np.zeros_like(f)
        iters = C.c_int(0)
        hist = np.zeros(maxit + 1)
        tr = C.c_double(0.0)
        st = self._check(self._L.iga_solve_host(self._h, f.ctypes.data, x.ctypes.data, float(tol), int(maxit),
                                                C.byref(iters), hist.ctypes.data, C.byref(tr)))
        return x, iters.value, hist[:iters.value + 1], tr.value, st


def solve_batched(contexts, rhs, x=None, tol=1e-7, maxit=100, stream=None):
    """Solve every contexts[b] for the right-hand sides rhs[b] (tensor of shape
    (nrhs_b, n_b), complex128, CUDA) in one graph launch.  Returns (x list,
    iterations list of arrays, status list of arrays, overall status)."""
    L = _ffi.lib()
    nb = len(contexts)
    rhs = [r.reshape(-1, c.n).contiguous() for r, c in zip(rhs, contexts)]
    if x is None:
        x = [torch.zeros_like(r) for r in rhs]
    nr = [int(r.shape[0]) for r in rhs]
    tot = sum(nr)
    H = (C.c_void_p * nb)(*[c._h.value for c in contexts])
    R = (C.c_void_p * nb)(*[_ptr(r) for r in rhs])
    X = (C.c_void_p * nb)(*[_ptr(v) for v in x])
    N = (C.c_int * nb)(*nr)
    it = (C.c_int * tot)()
    stt = (C.c_int * tot)()
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = L.iga_solve_batched(H, nb, R, X, N, float(tol), int(maxit), it, stt, C.c_void_p(s.cuda_stream))
    if rc < 0:
        raise IgaError(rc, contexts[0]._L.iga_last_error(contexts[0]._h).decode())
    its, sts, k = [], [], 0
    for n_r in nr:
        its.append(np.array(it[k:k + n_r]))
        sts.append(np.array(stt[k:k + n_r]))
        k += n_r
    return x, its, sts, rc


def from_problem(pr, **kw) -> Helmholtz:
    """Build a context from a workloads.Problem-like description."""
    kf = pr.kfield
    kfield = float(kf.values[0]) if len(kf.lines) == 0 else kf
    if not getattr(pr, "shift_uses_mass", True):
        raise ValueError("the identity-shift CSLP is not built on the GPU (see the CSLP reading of Section 3)")
    args = dict(dim=pr.dim, p=pr.p, n_el=pr.n_el, kfield=kfield, beta=pr.shift, eps=pr.eps, nu_pre=pr.nu_pre,
                nu_post=pr.nu_post, omega=pr.omega, n_vcycles=pr.n_vcycles,
                precond={"mg": 0, "exact": 1}[getattr(pr, "precond", "mg")],
                deflation=1 if getattr(pr, "deflation", True) else 0,
                robin=1 if getattr(pr, "robin", False) else 0)
    args.update(kw)
    return Helmholtz(**args)
