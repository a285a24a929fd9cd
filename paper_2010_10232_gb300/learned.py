"""Learned correction of the FP32 CSLP V-cycle: network handle, training-data
generation from the solver's own preconditioner inputs, and training.

Argument marshalling and the training loop's bookkeeping only: every
computation (V-cycles, residuals, packing, convolutions, gradients, Adam) runs
in the CUDA library.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _ffi
from .solver import Helmholtz, IgaError, _ptr


class Net:
    """The 3 -> 32 -> 32 -> 32 -> 2 convolution network (BF16 kernels, FP32 master weights)."""

    def __init__(self, seed: int = 0):
        self._L = _ffi.lib()
        h = C.c_void_p()
        st = self._L.iga_net_create(C.c_ulonglong(seed), C.byref(h))
        if st != 0:
            raise IgaError(st, "iga_net_create failed")
        self._h = h
        self.num_params = int(self._L.iga_net_num_params())

    def close(self):
        if getattr(self, "_h", None):
            self._L.iga_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st < 0:
            raise IgaError(st, self._L.iga_net_last_error(self._h).decode())
        return st

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.num_params, dtype=np.float32)
        self._check(self._L.iga_net_get_params(self._h, out.ctypes.data, out.size))
        return out

    def set_params(self, theta) -> None:
        theta = np.ascontiguousarray(theta, dtype=np.float32)
        self._check(self._L.iga_net_set_params(self._h, theta.ctypes.data, theta.size))

    def save(self, path: str) -> None:
        np.save(path, self.get_params())

    def load(self, path: str) -> None:
        self.set_params(np.load(path))

    @staticmethod
    def _stream():
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        """x: (B, H, W, 16) bfloat16 on the GPU -> (B, H, W, 2) float32."""
        B, H, Wd, _ = x.shape
        y = torch.empty(B, H, Wd, 2, dtype=torch.float32, device=x.device)
        self._check(self._L.iga_net_forward(self._h, C.c_void_p(_ptr(x)), C.c_void_p(_ptr(y)), B, H, Wd,
                                            self._stream()))
        return y

    def grad(self, x: torch.Tensor, t: torch.Tensor):
        B, H, Wd, _ = x.shape
        g = np.zeros(self.num_params, dtype=np.float32)
        loss = C.c_float(0.0)
        self._check(self._L.iga_net_grad(self._h, C.c_void_p(_ptr(x)), C.c_void_p(_ptr(t)), B, H, Wd,
                                         g.ctypes.data, C.byref(loss), self._stream()))
        return g, float(loss.value)

    def train_step(self, x: torch.Tensor, t: torch.Tensor, lr: float = 1e-3) -> float:
        B, H, Wd, _ = x.shape
        loss = C.c_float(0.0)
        self._check(self._L.iga_net_train_step(self._h, C.c_void_p(_ptr(x)), C.c_void_p(_ptr(t)), B, H, Wd,
                                               C.c_float(lr), C.byref(loss), self._stream()))
        return float(loss.value)


def _attach(self: Helmholtz, net: Net | None, gamma: float = 1.0) -> None:
    self._check(self._L.iga_attach_net(self._h, net._h if net is not None else None, float(gamma)))
    self._net = net          # keep the network alive while attached


Helmholtz.attach = _attach


def preconditioner_inputs(h: Helmholtz, f: torch.Tensor, count: int):
    """Vectors of the kind the preconditioner sees inside FGMRES: v0 = P f / |P f|,
    v_{j+1} = P A M~^{-1} v_j / |.| (the Krylov directions before orthogonalisation)."""
    v = h.deflate(f)
    v = v / torch.linalg.vector_norm(v)
    out = []
    for _ in range(count):
        out.append(v)
        z = h.vcycle(v)
        w = h.deflate(h.apply_A(z))
        v = w / torch.linalg.vector_norm(w)
    return out


def make_pairs(h: Helmholtz, vectors, crops_per_vector: int, crop: int, gamma: float, cycles: int, rng):
    """Training samples (X bf16 (N, crop, crop, 16), T f32 (N, crop, crop, 2)) from
    preconditioner inputs: e = (I - V M_beta)^cycles V(v), r~ = M_beta e (so
    e = M_beta^{-1} r~ exactly), random crops."""
    L = h._L
    nx = h.level_nx(0)
    Xs, Ts = [], []
    rt = h.vec()
    e = h.vec()
    for v in vectors:
        h._check(L.iga_precond_pair(h._h, C.c_void_p(_ptr(v)), C.c_void_p(_ptr(rt)), C.c_void_p(_ptr(e)), int(cycles)))
        for _ in range(crops_per_vector):
            x0 = int(rng.integers(0, max(1, nx - crop + 1)))
            y0 = int(rng.integers(0, max(1, nx - crop + 1)))
            X = torch.empty(crop, crop, 16, dtype=torch.bfloat16, device="cuda")
            T = torch.empty(crop, crop, 2, dtype=torch.float32, device="cuda")
            h._check(L.iga_net_pack(h._h, C.c_void_p(_ptr(rt)), C.c_void_p(_ptr(e)), x0, y0, crop, crop,
                                    C.c_void_p(_ptr(X)), C.c_void_p(_ptr(T)), float(gamma)))
            Xs.append(X)
            Ts.append(T)
    return torch.stack(Xs), torch.stack(Ts)


def target_scale(h: Helmholtz, v: torch.Tensor, cycles: int = 1) -> float:
    """RMS(e) / RMS(r~) for one preconditioner input: the normalisation that makes
    the network's targets O(1)."""
    rt, e = h.vec(), h.vec()
    h._check(h._L.iga_precond_pair(h._h, C.c_void_p(_ptr(v)), C.c_void_p(_ptr(rt)), C.c_void_p(_ptr(e)), int(cycles)))
    return float(torch.linalg.vector_norm(e) / torch.linalg.vector_norm(rt))
