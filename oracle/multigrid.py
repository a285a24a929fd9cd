"""Geometric multigrid approximation of the CSLP inverse (paper Section 3, CSLP
paragraph: damped Jacobi with omega = 0.6; Section 4.2: V-cycle structure and
the transfer operators).

Test infrastructure only (see oracle/__init__.py).

Readings taken where the paper is silent:
* levels: halve n_el while it is even and >= 8 (coarsest n_el in 4..7), with a
  dense direct solve on the coarsest level;
* coarse operators by rediscretisation (same quadrature, k^2 at the coarse
  Gauss points), identical to the Galerkin product for constant k;
* transfers: B-spline knot insertion between the nested knot vectors (the
  paper's linear interpolation is the p = 1 case); restriction is the
  transpose of prolongation;
* shift: M_beta = S - (beta1 - i beta2) M^{k^2}.

Pins (tests/test_oracle_multigrid.py): P reproduces the coarse spline
pointwise, interior mask 2^{-p} C(p+1, j), rediscretised = Galerkin for
constant k, V-cycle iteration converges to M_beta^{-1} b, explicit two-level
matrix on a tiny case.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import bspline
from .assembly import Discretization


def level_sizes(n_el: int) -> list[int]:
    """n_el per level: halve while even and >= 8."""
    out = [n_el]
    while out[-1] % 2 == 0 and out[-1] >= 8:
        out.append(out[-1] // 2)
    return out


def boehm_insert(knots: np.ndarray, p: int, rows: list, u: float):
    """Insert one knot u (Boehm's algorithm).  rows holds one sparse row
    {column: value} per basis function (the coefficients of any number of
    splines, one per column).  With t[k] <= u < t[k+1], rows i <= k - p are
    kept, rows i > k shift by one, and rows k - p < i <= k become
    (1 - a_i) c_{i-1} + a_i c_i with a_i = (u - t_i) / (t_{i+p} - t_i).
    Returns (new_knots, new_rows)."""
    t = knots
    k = int(np.searchsorted(t, u, side='right') - 1)      # t[k] <= u < t[k+1]
    mid = []
    for i in range(k - p + 1, k + 1):
        a = (u - t[i]) / (t[i + p] - t[i])
        lo, hi = rows[i - 1], rows[i]
        mid.append({c: (1.0 - a) * lo.get(c, 0.0) + a * hi.get(c, 0.0) for c in set(lo) | set(hi)})
    return np.insert(t, k + 1, u), rows[:k - p + 1] + mid + rows[k:]


def prolongation_1d_sparse(n_el_coarse: int, p: int) -> sp.csr_matrix:
    """Knot-insertion matrix (full bases): fine coefficients of each coarse
    basis function, obtained by inserting the midpoints of all coarse spans
    one at a time into the identity (one column per coarse function)."""
    tc = bspline.open_uniform_knots(n_el_coarse, p)
    nbc = n_el_coarse + p
    t, rows = tc.copy(), [{j: 1.0} for j in range(nbc)]
    n_f = 2 * n_el_coarse
    for i in range(n_el_coarse):
        u = float(2 * i + 1) / float(n_f)
        t, rows = boehm_insert(t, p, rows, u)
    tf = bspline.open_uniform_knots(n_f, p)
    assert np.array_equal(t, tf), "knot insertion did not produce the fine knot vector"
    ri = [i for i, r in enumerate(rows) for _ in r]
    ci = [c for r in rows for c in r]
    vals = [v for r in rows for v in r.values()]
    return sp.csr_matrix((vals, (ri, ci)), shape=(len(rows), nbc))


def prolongation_1d(n_el_coarse: int, p: int) -> np.ndarray:
    """The knot-insertion matrix, dense."""
    return prolongation_1d_sparse(n_el_coarse, p).toarray()


def prolongation_interior_1d(n_el_coarse: int, p: int, robin: bool = False, sparse: bool = False):
    """Interior rows/columns of the knot-insertion matrix.  A coarse spline
    with zero end coefficients refines to a fine spline with zero end
    coefficients, so the Dirichlet-eliminated transfer is the submatrix (with
    the Sommerfeld end at x = 1, only the first row and column are dropped).
    Dense unless sparse=True (CSR)."""
    P = prolongation_1d_sparse(n_el_coarse, p)
    P = P[1:, 1:] if robin else P[1:-1, 1:-1]
    return P.tocsr() if sparse else P.toarray()


class Level:
    def __init__(self, disc: Discretization, beta1: float, beta2: float, uses_mass: bool = True):
        self.disc = disc
        self.Mb = disc.shifted(beta1, beta2, uses_mass)
        self.D = self.Mb.diagonal()


class MGHierarchy:
    """Rediscretised CSLP levels plus transfers for one problem description."""

    def __init__(self, dim, p, n_el, kfield, beta1, beta2, omega=0.6, nu_pre=1, nu_post=1,
                 fine_disc: Discretization | None = None, uses_mass: bool = True, robin: bool = False):
        self.sizes = level_sizes(n_el)
        self.omega, self.nu_pre, self.nu_post = omega, nu_pre, nu_post
        self.levels = []
        self.P = []
        for li, ne in enumerate(self.sizes):
            disc = fine_disc if (li == 0 and fine_disc is not None) else Discretization(dim, p, ne, kfield, robin)
            self.levels.append(Level(disc, beta1, beta2, uses_mass))
            if li > 0:
                P1 = prolongation_interior_1d(ne, p, robin, sparse=True)
                self.P.append(P1 if dim == 1 else sp.kron(P1, P1).tocsr())
        self.coarse_dense = self.levels[-1].Mb.toarray()

    def jacobi(self, lvl: Level, x, b, sweeps):
        """Damped Jacobi: x <- x + omega D^{-1} (b - M_beta x)."""
        for _ in range(sweeps):
            x = x + self.omega * (b - lvl.Mb @ x) / lvl.D
        return x

    def vcycle(self, b, li: int = 0):
        """One V-cycle for M_beta x = b from x = 0."""
        lvl = self.levels[li]
        if li == len(self.levels) - 1:
            return np.linalg.solve(self.coarse_dense, b)
        x = np.zeros_like(b)
        x = self.jacobi(lvl, x, b, self.nu_pre)
        r = b - lvl.Mb @ x
        bc = self.P[li].T @ r
        xc = self.vcycle(bc, li + 1)
        x = x + self.P[li] @ xc
        x = self.jacobi(lvl, x, b, self.nu_post)
        return x

    def apply(self, b, n_cycles: int = 1):
        """j V-cycles as a stationary iteration from x = 0:
        x <- x + V(b - M_beta x)."""
        x = self.vcycle(b, 0)
        Mb = self.levels[0].Mb
        for _ in range(n_cycles - 1):
            x = x + self.vcycle(b - Mb @ x, 0)
        return x
