"""GMRES and flexible GMRES (paper Section 3 uses GMRES; Section 4.3: stop at
relative residual 1e-7, at most 100 iterations).

Test infrastructure only (see oracle/__init__.py).

Readings: no restart, x0 = 0, modified Gram-Schmidt Arnoldi with the
Hermitian inner product, complex Givens rotations on the Hessenberg matrix.
``gmres`` is left preconditioned in the sense that the caller passes the full
operator v -> B v (e.g. M^{-1} P A); its stopping test is on the residual of
that operator.  ``fgmres`` is right preconditioned with a per-iteration
preconditioner whose outputs z_j are stored.

Pins (tests/test_oracle_krylov.py): the iterate x_j equals the brute-force
minimiser over the explicit Krylov space; residual history non-increasing;
FGMRES with a fixed preconditioner equals GMRES on B M^{-1}.
"""
from __future__ import annotations

import numpy as np


def _givens(a, b):
    """Rotation (c real, s complex) with [c, s; -conj(s), c] [a; b] = [r; 0]."""
    if b == 0:
        return 1.0, 0.0 + 0.0j
    if a == 0:
        return 0.0, np.conj(b) / abs(b)
    t = np.hypot(abs(a), abs(b))
    c = abs(a) / t
    s = (a / abs(a)) * np.conj(b) / t
    return c, s


class KrylovResult:
    def __init__(self, x, iters, hist, converged, y=None, V=None):
        self.x, self.iters, self.hist, self.converged = x, iters, hist, converged
        self.y, self.V = y, V


def gmres(op, b, tol=1e-7, maxit=100, x_at=None):
    """Solve op(x) = b from x0 = 0.  Returns KrylovResult with the residual
    history |g_{j+1}| / beta.  If x_at is an int, the iterate after exactly
    x_at iterations is also returned as result.x_at."""
    n = b.shape[0]
    beta = np.linalg.norm(b)
    V = np.zeros((n, maxit + 1), dtype=np.complex128)
    H = np.zeros((maxit + 1, maxit), dtype=np.complex128)
    cs = np.zeros(maxit)
    sn = np.zeros(maxit, dtype=np.complex128)
    g = np.zeros(maxit + 1, dtype=np.complex128)
    hist = [1.0]
    if beta == 0:
        return KrylovResult(np.zeros(n, np.complex128), 0, hist, True)
    V[:, 0] = b / beta
    g[0] = beta
    j_done = 0
    converged = False
    xs = {}
    for j in range(maxit):
        w = op(V[:, j])
        for i in range(j + 1):                      # modified Gram-Schmidt
            H[i, j] = np.vdot(V[:, i], w)
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] != 0:
            V[:, j + 1] = w / H[j + 1, j]
        Hj = H[:, j].copy()
        for i in range(j):                          # previous rotations
            t = cs[i] * Hj[i] + sn[i] * Hj[i + 1]
            Hj[i + 1] = -np.conj(sn[i]) * Hj[i] + cs[i] * Hj[i + 1]
            Hj[i] = t
        c, s = _givens(Hj[j], Hj[j + 1])
        cs[j], sn[j] = c, s
        Hj[j] = c * Hj[j] + s * Hj[j + 1]
        Hj[j + 1] = 0.0
        H[:, j] = Hj                                # H now holds the rotated R
        g[j + 1] = -np.conj(s) * g[j]
        g[j] = c * g[j]
        res = abs(g[j + 1]) / beta
        hist.append(res)
        j_done = j + 1
        if x_at is not None and j_done == x_at:
            y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
            xs[j_done] = V[:, :j_done] @ y
        if res <= tol:
            converged = True
            break
    y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
    x = V[:, :j_done] @ y
    out = KrylovResult(x, j_done, hist, converged, y=y, V=V[:, :j_done])
    out.x_at = xs.get(x_at)
    return out


def fgmres(op, prec, b, tol=1e-7, maxit=100):
    """Right-preconditioned flexible GMRES: z_j = prec(v_j), w = op(z_j);
    x = sum_j y_j z_j.  Stops on |g_{j+1}| / ||b||."""
    n = b.shape[0]
    beta = np.linalg.norm(b)
    V = np.zeros((n, maxit + 1), dtype=np.complex128)
    Zs = np.zeros((n, maxit), dtype=np.complex128)
    H = np.zeros((maxit + 1, maxit), dtype=np.complex128)
    cs = np.zeros(maxit)
    sn = np.zeros(maxit, dtype=np.complex128)
    g = np.zeros(maxit + 1, dtype=np.complex128)
    hist = [1.0]
    if beta == 0:
        return KrylovResult(np.zeros(n, np.complex128), 0, hist, True)
    V[:, 0] = b / beta
    g[0] = beta
    j_done, converged = 0, False
    for j in range(maxit):
        Zs[:, j] = prec(V[:, j])
        w = op(Zs[:, j])
        for i in range(j + 1):
            H[i, j] = np.vdot(V[:, i], w)
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] != 0:
            V[:, j + 1] = w / H[j + 1, j]
        Hj = H[:, j].copy()
        for i in range(j):
            t = cs[i] * Hj[i] + sn[i] * Hj[i + 1]
            Hj[i + 1] = -np.conj(sn[i]) * Hj[i] + cs[i] * Hj[i + 1]
            Hj[i] = t
        c, s = _givens(Hj[j], Hj[j + 1])
        cs[j], sn[j] = c, s
        Hj[j] = c * Hj[j] + s * Hj[j + 1]
        Hj[j + 1] = 0.0
        H[:, j] = Hj
        g[j + 1] = -np.conj(s) * g[j]
        g[j] = c * g[j]
        res = abs(g[j + 1]) / beta
        hist.append(res)
        j_done = j + 1
        if res <= tol:
            converged = True
            break
    y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
    x = Zs[:, :j_done] @ y
    return KrylovResult(x, j_done, hist, converged, y=y)
