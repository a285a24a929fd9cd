"""Small, self-contained launch sequences for Nsight Compute captures.

    python -m measure.profile_cases apply   # FP64 constant-k apply, bench size
    python -m measure.profile_cases apply32 # FP32 V-cycle, 4097^2 dofs
    python -m measure.profile_cases solve   # one bench solve
    python -m measure.profile_cases solve_host  # same, iterations launched from the host
    python -m measure.profile_cases sweep32     # FP32 Jacobi sweep on level 0, 4097^2 dofs
    python -m measure.profile_cases cnn         # network forward pass, 1281^2 pixels
    python -m measure.profile_cases esolve1d    # 1D E solve at k = 10^6 (band solver)
    python -m measure.profile_cases solve1d     # 1D deflated GMRES at k = 10^6, p = 5, 12 iterations

The solve, apply32, sweep32, cnn, esolve1d and solve1d cases open a profiler range around the
timed launches only (capture them with `ncu --profile-from-start off`).

Each case launches a handful of kernels on inputs of the bench problem so a
capture (-k <kernel> -c <count>) ends in seconds.
"""
from __future__ import annotations

import sys

import torch

from paper_2010_10232_gb300.solver import Helmholtz


def main(case: str) -> None:
    torch.cuda.set_device(0)
    if case == "apply":
        h = Helmholtz(dim=2, p=3, n_el=320, kfield=200.0, skip_deflation=1)
        x = torch.randn(h.n, dtype=torch.complex128, device="cuda")
        y = h.vec()
        for _ in range(4):
            h.apply_A(x, y)
    elif case == "apply32":
        h = Helmholtz(dim=2, p=3, n_el=4096, kfield=2560.0, skip_deflation=1, precision=1)
        x = torch.randn(h.n, dtype=torch.complex128, device="cuda")
        z = h.vec()
        h.vcycle(x, z)
        torch.cuda.synchronize()
        # one V-cycle inside the profiler range (ncu --profile-from-start off);
        # the setup's launches, the tile autotuner's included, stay outside
        torch.cuda.profiler.start()
        h.vcycle(x, z)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    elif case == "sweep32":
        # one FP32 Jacobi sweep on level 0 at 4097^2 dofs inside the profiler
        # range (capture with ncu --profile-from-start off)
        h = Helmholtz(dim=2, p=3, n_el=4096, kfield=2560.0, skip_deflation=1, precision=1)
        xs = torch.randn(h.n, dtype=torch.complex64, device="cuda")
        bs = torch.randn(h.n, dtype=torch.complex64, device="cuda")
        xo = torch.empty_like(xs)
        h.jacobi32(0, bs, xs, xo)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        for _ in range(2):
            h.jacobi32(0, bs, xs, xo)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    elif case == "esolve1d":
        # one solve with the 1D deflation matrix E at k = 10^6, p = 1 (799 999
        # unknowns, band solver) inside the profiler range
        h = Helmholtz(dim=1, p=1, n_el=1600000, kfield=1e6)
        t = torch.randn(h.m, dtype=torch.complex128, device="cuda")
        h.esolve(t)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        h.esolve(t)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    elif case == "solve1d":
        # MP 1-B at k = 10^6, p = 5 (1.6 10^6 dofs), deflation alone (D): one
        # solve of 12 iterations inside the profiler range
        h = Helmholtz(dim=1, p=5, n_el=1600000, kfield=1e6, n_vcycles=0)
        f = h.point_source(0.5)
        x = h.vec()
        h.solve(f, x=x, tol=0.0, maxit=12)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        h.solve(f, x=x, tol=0.0, maxit=12)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    elif case == "cnn":
        # one forward pass of the correction network at 1281^2 pixels (the
        # 1280^2-element grid) inside the profiler range
        from paper_2010_10232_gb300.learned import Net
        net = Net(seed=0)
        x = torch.zeros(1, 1281, 1281, 16, dtype=torch.bfloat16, device="cuda")
        x[..., :3] = torch.randn(1, 1281, 1281, 3, device="cuda").to(torch.bfloat16)
        net.forward(x)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        net.forward(x)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    elif case in ("solve", "solve_host"):
        h = Helmholtz(dim=2, p=3, n_el=320, kfield=200.0, host_loop=int(case == "solve_host"))
        f = h.point_source(0.5, 0.5)
        torch.cuda.synchronize()
        # the solve alone is the profiler range (ncu --profile-from-start off):
        # the setup's launches, the tile autotuner's included, stay outside
        torch.cuda.profiler.start()
        h.solve(f)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    else:
        raise SystemExit(f"unknown case {case}")
    torch.cuda.synchronize()
    print("ok", case)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "apply")
