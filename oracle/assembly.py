"""Galerkin assembly of the IgA Helmholtz operator (paper Section 2.3, Eq. linearsystem1).

Test infrastructure only (see oracle/__init__.py).

S_ij = int grad Phi_i . grad Phi_j,  M_ij = int Phi_i Phi_j,
M^{k^2}_ij = int k(x)^2 Phi_i Phi_j, all by (p+1)-point Gauss quadrature per
knot span (per element in 2D, tensor Gauss rule).  The operator is
A = S - M^{k^2}: the reading of the paper's sign conflict that matches its
model problems (-Delta u - k^2 u = f) and the exact solution e^{ikx}.
Homogeneous Dirichlet conditions are imposed by deleting the first and last
basis function in each direction (the open knot vector makes them the only
functions that are non-zero on the boundary).

Index convention: interior coefficient (ix, iy) sits at flat index
iy * n_x + ix (x fastest), ix = bx - 1 for full basis index bx.

Pins (tests/test_oracle_assembly.py): p=1 textbook element matrices, zero row
sums of S before Dirichlet elimination, sum(M) = |Omega|, symmetry,
generalised eigenvalues -> j^2 pi^2 at rate h^{2p}, manufactured-solution
L2 rates O(h^{p+1}), MP 1-B Green's function, MP 1-A Table 1 rates.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import bspline


# ---------------------------------------------------------------- k field
def k_of(kfield, x, y=None):
    """Piecewise-constant wave number: values[count of lines with a*x+b*y+c >= 0],
    the sum evaluated as ((a*x) + (b*y)) + c."""
    x = np.asarray(x, dtype=np.float64)
    if len(kfield.lines) == 0:
        return np.full(x.shape, float(kfield.values[0]))
    y = np.asarray(y, dtype=np.float64)
    count = np.zeros(x.shape, dtype=np.int64)
    for ln in kfield.lines:
        s = (ln.a * x + ln.b * y) + ln.c
        count += (s >= 0.0)
    return np.asarray(kfield.values, dtype=np.float64)[count]


# ---------------------------------------------------------------- 1D tables
def local_tables(n_el: int, p: int):
    """Per element e and Gauss point q: values B[e,q,a] and derivatives
    D[e,q,a] of the p+1 functions a = 0..p that are active on span e
    (full basis index e + a), Gauss points xq[e,q] and weights wq[e,q]."""
    t = bspline.open_uniform_knots(n_el, p)
    xq, wq, spans = bspline.element_quadrature(t, p)
    assert len(spans) == n_el
    nq = p + 1
    B = np.zeros((n_el, nq, p + 1))
    D = np.zeros((n_el, nq, p + 1))
    if n_el <= 256:
        pts = xq.reshape(-1)
        phi = bspline.basis_all(t, p, pts)
        dphi = bspline.basis_deriv_all(t, p, pts)
        for e in range(n_el):
            cols = slice(e * nq, (e + 1) * nq)
            # every function outside e..e+p must vanish on span e
            mask = np.ones(phi.shape[0], bool)
            mask[e:e + p + 1] = False
            assert np.all(phi[mask, cols] == 0.0)
            B[e] = phi[e:e + p + 1, cols].T
            D[e] = dphi[e:e + p + 1, cols].T
    else:
        # the functions e..e+p active on span e depend only on the knots
        # t[e .. e+2p+1]: the same recursion on that window gives the same
        # values (no Gauss point is a knot) without evaluating all n_el + p
        # functions at every point
        tw = np.stack([t[e:e + 2 * p + 2] for e in range(n_el)])
        B[:] = bspline.basis_windows(tw, p, xq).transpose(0, 2, 1)
        D[:] = bspline.basis_deriv_windows(tw, p, xq).transpose(0, 2, 1)
    return B, D, xq, wq


def assemble_1d(n_el: int, p: int, k2_fn=None):
    """Full (boundary functions included) 1D stiffness K, mass M and, if
    k2_fn is given, the weighted mass int k^2 phi_i phi_j, as CSR matrices."""
    B, D, xq, wq = local_tables(n_el, p)
    nb = n_el + p
    k2 = k2_fn(xq) if k2_fn is not None else None
    # element e, functions a, c: sum over q of w_q f_a(x_q) g_c(x_q), the
    # products formed left to right and summed over q in order, for all
    # (e, a, c) at once; entry (e + a, e + c) (duplicates add up)
    e_, a_, c_ = np.meshgrid(np.arange(n_el), np.arange(p + 1), np.arange(p + 1), indexing="ij")
    rows, cols = (e_ + a_).reshape(-1), (e_ + c_).reshape(-1)
    w4 = wq[:, :, None, None]
    kv = np.sum(w4 * D[:, :, :, None] * D[:, :, None, :], axis=1).reshape(-1)
    mv = np.sum(w4 * B[:, :, :, None] * B[:, :, None, :], axis=1).reshape(-1)
    if k2 is not None:
        mkv = np.sum(w4 * k2[:, :, None, None] * B[:, :, :, None] * B[:, :, None, :], axis=1).reshape(-1)
    K = sp.csr_matrix((kv, (rows, cols)), shape=(nb, nb))
    M = sp.csr_matrix((mv, (rows, cols)), shape=(nb, nb))
    Mk = sp.csr_matrix((mkv, (rows, cols)), shape=(nb, nb)) if k2 is not None else None
    return K, M, Mk


def interior_1d(mat):
    """Delete the first and last row/column (homogeneous Dirichlet)."""
    n = mat.shape[0]
    return mat[1:n - 1, :][:, 1:n - 1].tocsr()


def assemble_2d(n_el: int, p: int, kfield, chunk: int = 32):
    """Full 2D stiffness S, plain mass M and weighted mass M^{k^2} on the unit
    square by tensor Gauss quadrature on each element (ex, ey).  k^2 is
    evaluated at every Gauss point.  Returns CSR matrices over the full
    (n_el+p)^2 basis, flat index by * nb + bx."""
    B, D, xq, wq = local_tables(n_el, p)
    nb = n_el + p
    q1 = p + 1
    S_parts, M_parts, Mk_parts = [], [], []
    a_idx = np.arange(q1)
    for ey0 in range(0, n_el, chunk):
        ey1 = min(n_el, ey0 + chunk)
        ey = np.arange(ey0, ey1)
        ex = np.arange(n_el)
        # Gauss points of elements (ex, ey): X[ex,qx], Y[ey,qy]
        Xg = xq[ex][:, None, :, None]             # ex, 1, qx, 1
        Yg = xq[ey][None, :, None, :]             # 1, ey, 1, qy
        Xb, Yb = np.broadcast_arrays(Xg, Yg)
        k = k_of(kfield, Xb, Yb)                  # ex, ey, qx, qy
        W = wq[ex][:, None, :, None] * wq[ey][None, :, None, :]
        Bx, Dx = B[ex], D[ex]                     # ex, qx, a
        By, Dy = B[ey], D[ey]                     # ey, qy, b
        # local matrices [ex, ey, a, b, c, d]: row (a,b), column (c,d)
        Ml = np.einsum('xyqr,xqa,xqc,yrb,yrd->xyabcd', W, Bx, Bx, By, By, optimize=True)
        Mkl = np.einsum('xyqr,xqa,xqc,yrb,yrd->xyabcd', W * k * k, Bx, Bx, By, By, optimize=True)
        Sl = (np.einsum('xyqr,xqa,xqc,yrb,yrd->xyabcd', W, Dx, Dx, By, By, optimize=True)
              + np.einsum('xyqr,xqa,xqc,yrb,yrd->xyabcd', W, Bx, Bx, Dy, Dy, optimize=True))
        gx = ex[:, None, None, None, None, None] + a_idx[None, None, :, None, None, None]
        gy = ey[None, :, None, None, None, None] + a_idx[None, None, None, :, None, None]
        hx = ex[:, None, None, None, None, None] + a_idx[None, None, None, None, :, None]
        hy = ey[None, :, None, None, None, None] + a_idx[None, None, None, None, None, :]
        shape = Ml.shape
        r = np.broadcast_to(gy * nb + gx, shape).reshape(-1)
        c = np.broadcast_to(hy * nb + hx, shape).reshape(-1)
        S_parts.append(sp.coo_matrix((Sl.reshape(-1), (r, c)), shape=(nb * nb, nb * nb)).tocsr())
        M_parts.append(sp.coo_matrix((Ml.reshape(-1), (r, c)), shape=(nb * nb, nb * nb)).tocsr())
        Mk_parts.append(sp.coo_matrix((Mkl.reshape(-1), (r, c)), shape=(nb * nb, nb * nb)).tocsr())
    S = S_parts[0]
    M = M_parts[0]
    Mk = Mk_parts[0]
    for i in range(1, len(S_parts)):
        S = S + S_parts[i]
        M = M + M_parts[i]
        Mk = Mk + Mk_parts[i]
    return S.tocsr(), M.tocsr(), Mk.tocsr()


def interior_index_2d(nb: int) -> np.ndarray:
    """Flat full indices of the interior functions, in interior lexicographic
    order (x fastest)."""
    i = np.arange(1, nb - 1)
    return (i[:, None] * nb + i[None, :]).reshape(-1)


def interior_2d(mat, nb: int):
    idx = interior_index_2d(nb)
    return mat[idx, :][:, idx].tocsr()


# ---------------------------------------------------------------- operators
class Discretization:
    """Interior (Dirichlet-eliminated) S, M, M^{k^2} and A = S - M^{k^2} for one
    problem description (dim, p, n_el, kfield).

    robin=True (1D only): the Sommerfeld condition u' - i k u = 0 at x = 1 of
    MP 1-A (Section 2.1): the last basis function stays an unknown and the weak
    form adds the boundary mass, A = S - M^{k^2} - i k N with N = phi_last(1)^2
    at x = 1 (Section 2.3, Eq. linearsystem1's N term, read with the sign of the
    model problem); x = 0 keeps its Dirichlet condition, whose data enter the
    right-hand side through `dirichlet_lift`.  Pins: tests/test_oracle_robin.py."""

    def __init__(self, dim: int, p: int, n_el: int, kfield, robin: bool = False):
        self.dim, self.p, self.n_el, self.kfield = dim, p, n_el, kfield
        self.robin = bool(robin)
        if self.robin and dim != 1:
            raise ValueError("the Sommerfeld boundary is built for the 1D problem (MP 1-A)")
        self.nb = n_el + p
        self.n_x = n_el + p - 2 + (1 if self.robin else 0)
        if dim == 1:
            k2 = (lambda x: k_of(kfield, x) ** 2)
            K, M, Mk = assemble_1d(n_el, p, k2)
            if self.robin:
                cut = lambda mat: mat[1:, :][:, 1:].tocsr()
                self.S, self.M, self.Mk = cut(K), cut(M), cut(Mk)
                # coupling of the unknowns to the Dirichlet function at x = 0
                self.col0 = np.asarray((K - Mk)[1:, 0].toarray()).reshape(-1).astype(np.complex128)
                self.k_boundary = float(k_of(kfield, np.array([1.0]))[0])
                nb = self.S.shape[0]
                self.N = sp.csr_matrix(([1.0], ([nb - 1], [nb - 1])), shape=(nb, nb))
            else:
                self.S = interior_1d(K)
                self.M = interior_1d(M)
                self.Mk = interior_1d(Mk)
        else:
            S, M, Mk = assemble_2d(n_el, p, kfield)
            self.S = interior_2d(S, self.nb)
            self.M = interior_2d(M, self.nb)
            self.Mk = interior_2d(Mk, self.nb)
        self.A = (self.S - self.Mk).astype(np.complex128).tocsr()
        if self.robin:
            self.A = (self.A - 1j * self.k_boundary * self.N).tocsr()

    def dirichlet_lift(self, g0) -> np.ndarray:
        """Right-hand side of the inhomogeneous Dirichlet value u(0) = g0 (the
        first, interpolatory coefficient is g0): f = -g0 A[unknowns, 0]."""
        if not self.robin:
            raise ValueError("the lift is defined for the MP 1-A discretisation")
        return -complex(g0) * self.col0

    @property
    def n(self) -> int:
        return self.S.shape[0]

    def shifted(self, beta1: float, beta2: float, uses_mass: bool = True):
        """CSLP operator of Section 3 (CSLP equation).

        uses_mass=True (the reading used everywhere): M_beta = S - (beta1 -
        i beta2) M^{k^2}, the shift on the mass matrix.  uses_mass=False: the
        equation as printed, M = A + i beta2 k^2 I with A = S - beta1 M^{k^2}
        (beta1 = 1 in the paper), the shift on the identity; defined here for
        constant k only (the printed form does not say where a variable k^2
        would be sampled).

        Pins: tests/test_oracle_cslp.py (1D p = 1 closed-form eigenvalues of
        both forms; the paper's Table 2 C_ex counts, met by the mass form only)."""
        if uses_mass:
            out = (self.S - (beta1 - 1j * beta2) * self.Mk).astype(np.complex128).tocsr()
            if self.robin:      # the boundary term is not shifted
                out = (out - 1j * self.k_boundary * self.N).tocsr()
            return out
        if len(self.kfield.lines) != 0:
            raise ValueError("identity-shift CSLP is defined for constant k only")
        k2 = float(self.kfield.values[0]) ** 2
        ident = sp.identity(self.S.shape[0], format='csr')
        return (self.S - beta1 * self.Mk + 1j * beta2 * k2 * ident).astype(np.complex128).tocsr()


def point_source(dim: int, p: int, n_el: int, pos, robin: bool = False) -> np.ndarray:
    """Load vector of a unit point source: f_i = Phi_i(pos), interior functions
    (with robin, every function but the first)."""
    t = bspline.open_uniform_knots(n_el, p)
    vx = bspline.basis_all(t, p, [pos[0]])[:, 0][1:] if robin else bspline.basis_all(t, p, [pos[0]])[:, 0][1:-1]
    if dim == 1:
        return vx.astype(np.complex128)
    vy = bspline.basis_all(t, p, [pos[1]])[:, 0][1:-1]
    return np.outer(vy, vx).reshape(-1).astype(np.complex128)


def l2_load_1d(n_el: int, p: int, f_fn, nq: int | None = None) -> np.ndarray:
    """f_i = int f phi_i by Gauss quadrature with nq points per span (interior i)."""
    t = bspline.open_uniform_knots(n_el, p)
    nq = nq or (p + 4)
    xq, wq, _ = bspline.element_quadrature(t, p, nq)
    pts = xq.reshape(-1)
    phi = bspline.basis_all(t, p, pts)
    vals = f_fn(pts) * wq.reshape(-1)
    return (phi @ vals)[1:-1]


def eval_spline_1d(n_el: int, p: int, coef_full: np.ndarray, x) -> np.ndarray:
    t = bspline.open_uniform_knots(n_el, p)
    return coef_full @ bspline.basis_all(t, p, x)


def l2_error_1d(n_el: int, p: int, coef_full: np.ndarray, u_exact, nq: int = 10) -> float:
    """Continuous L2 error of a spline (full coefficient vector) vs u_exact by
    nq-point Gauss quadrature per span."""
    t = bspline.open_uniform_knots(n_el, p)
    xq, wq, _ = bspline.element_quadrature(t, p, nq)
    pts = xq.reshape(-1)
    uh = coef_full @ bspline.basis_all(t, p, pts)
    d = uh - u_exact(pts)
    return float(np.sqrt(np.sum(wq.reshape(-1) * np.abs(d) ** 2)))


def mp1a_solve(n_el: int, p: int, k: float):
    """MP 1-A (Section 2.1): -u'' - k^2 u = 0 on [0, 1], u(0) = 1,
    u'(1) - i k u(1) = 0.  Weak form gives A = K - k^2 M - i k N with the
    boundary mass N = phi_last(1)^2 at x = 1; the Dirichlet value enters as the
    first (interpolatory) coefficient.  Returns the full coefficient vector."""
    K, M, _ = assemble_1d(n_el, p)
    nb = n_el + p
    Nb = sp.csr_matrix(([1.0], ([nb - 1], [nb - 1])), shape=(nb, nb))
    A = (K - k * k * M - 1j * k * Nb).tocsc().astype(np.complex128)
    import scipy.sparse.linalg as spla
    rhs = -np.asarray(A[1:, 0].toarray()).reshape(-1)
    c = spla.spsolve(A[1:, 1:].tocsc(), rhs)
    return np.concatenate([[1.0 + 0j], c])
