"""Adapted deflation preconditioner (ADP) (paper Section 3: Eq. adef1 and the
quadratic rational-Bezier stencils for Z and Z^T, with the epsilon-weighted
variant).

Test infrastructure only (see oracle/__init__.py).

Readings:
* indices are 1-based interior indices; coarse dof i sits at fine dof 2i;
  m_x = floor(n_x / 2); stencil terms outside 1..n_x (fine) or 1..m_x
  (coarse) are dropped (they are Dirichlet zeros);
* the paper's printed Z^T row repeats the index 2j+1; it is read as the
  transpose of Z, i.e. (1, 4, 6 - eps, 4, 1)/8 on fine dofs 2j-2 .. 2j+2;
* 2D deflation space is the tensor product Z_y (x) Z_x.

Pins (tests/test_oracle_deflation.py): Z 1 = 1 and Z (linear) = linear in the
interior, E complex symmetric, P^2 = P, P A Z = 0, M^{-1} P A has exactly m
zero eigenvalues, A u = f after recovery.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def z_matrix_1d(n_x: int, eps: float = 0.0):
    """n_x x m_x deflation matrix of Section 3: even fine dof j = 2i gets
    (6 - eps)/8 of coarse dof i and 1/8 of i-1 and i+1; odd fine dof j gets 1/2 of
    coarse (j-1)/2 and (j+1)/2."""
    m_x = n_x // 2
    Z = np.zeros((n_x, m_x))
    for j in range(1, n_x + 1):                  # 1-based fine index
        if j % 2 == 0:
            terms = [((j - 2) // 2, 1.0 / 8.0), (j // 2, (6.0 - eps) / 8.0), ((j + 2) // 2, 1.0 / 8.0)]
        else:
            terms = [((j - 1) // 2, 0.5), ((j + 1) // 2, 0.5)]
        for i, w in terms:
            if 1 <= i <= m_x:
                Z[j - 1, i - 1] += w
    return sp.csr_matrix(Z)


def z_matrix(dim: int, n_x: int, eps: float = 0.0):
    Z1 = z_matrix_1d(n_x, eps)
    return Z1 if dim == 1 else sp.kron(Z1, Z1).tocsr()


class Deflation:
    """P = I - A Q, Q = Z E^{-1} Z^T, E = Z^T A Z (Eq. adef1)."""

    def __init__(self, A, Z):
        self.A = A.tocsr()
        self.Z = Z.tocsr()
        self.E = (self.Z.T @ self.A @ self.Z).tocsc()
        self.lu = spla.splu(self.E)

    @property
    def m(self) -> int:
        return self.Z.shape[1]

    def Q(self, v):
        return self.Z @ self.lu.solve(np.asarray(self.Z.T @ v, dtype=np.complex128))

    def P(self, v):
        """y = v - A Z E^{-1} Z^T v."""
        return v - self.A @ self.Q(v)

    def PT(self, v):
        """P^T v = v - Q A v  (A and Q complex symmetric)."""
        return v - self.Q(self.A @ v)
