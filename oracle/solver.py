"""End-to-end deflated, CSLP-preconditioned GMRES solve (paper Section 3,
deflated preconditioned system; Section 4.3 settings and the preconditioner
list D, D_eps, C_ex, DC_MG^j, D_eps C_MG^j), plus the direct solve.

Test infrastructure only (see oracle/__init__.py).

Preconditioner M~^{-1} (problem.precond):
* 'mg' (default): n_vcycles V-cycles of the CSLP hierarchy (oracle.multigrid);
  n_vcycles = 0 means no CSLP at all (the deflation-only D / D_eps of
  Section 4.3.1, Tables 2 and 3);
* 'exact': the CSLP matrix inverted by sparse LU (C_ex of Section 4.3).

Operator ordering (reading of the paper's P^T M^{-1} A u = P^T M^{-1} f, which
taken literally is singular and gives no recovery formula):

* 'def1' (default): GMRES on M~^{-1} P A x^ = M~^{-1} P f from x^ = 0, then
  u = Q f + P^T x^, with P = I - A Q, Q = Z E^{-1} Z^T, P^T = I - Q A.
* 'literal': GMRES on P^T M~^{-1} A u = P^T M~^{-1} f from u = 0; the iterate is
  used as u directly.
* flexible=True: right-preconditioned FGMRES on P A (M~^{-1} y) = P f, stopping
  on ||P (f - A x^)|| / ||P f||, recovery as for 'def1'.
* problem.deflation = False: no deflation (C_ex or C_MG alone): GMRES on
  M~^{-1} A u = M~^{-1} f (FGMRES on A M~^{-1} y = f), u = x^.

Pins (tests/test_oracle_solver.py, tests/test_oracle_cslp.py): recovery gives
A u = f; the 'literal' iterate equals the brute-force Krylov minimiser for the
dense P^T M~^{-1} A; Tables 2, 4 and 5 soft pins (iteration counts); the C_ex
preconditioned spectrum lies on the circle |mu - 1/2| = 1/2.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .assembly import Discretization, point_source
from .multigrid import MGHierarchy
from .deflation import Deflation, z_matrix
from .krylov import gmres, fgmres


class Solver:
    def __init__(self, problem, disc: Discretization | None = None):
        pr = problem
        self.problem = pr
        robin = bool(getattr(pr, "robin", False))
        self.disc = disc or Discretization(pr.dim, pr.p, pr.n_el, pr.kfield, robin)
        b1, b2 = pr.shift
        uses_mass = getattr(pr, "shift_uses_mass", True)
        kind = getattr(pr, "precond", "mg")
        if kind == "mg" and pr.n_vcycles == 0:
            kind = "none"
        if kind not in ("mg", "exact", "none"):
            raise ValueError(kind)
        self.precond_kind = kind
        self.mg = None
        self.cslp_lu = None
        if kind == "mg":
            self.mg = MGHierarchy(pr.dim, pr.p, pr.n_el, pr.kfield, b1, b2, omega=pr.omega,
                                  nu_pre=pr.nu_pre, nu_post=pr.nu_post, fine_disc=self.disc,
                                  uses_mass=uses_mass, robin=robin)
        elif kind == "exact":
            self.cslp = self.disc.shifted(b1, b2, uses_mass).tocsc()
            self.cslp_lu = spla.splu(self.cslp)
        self.deflated = bool(getattr(pr, "deflation", True))
        self.Z = z_matrix(pr.dim, self.disc.n_x, pr.eps)
        self.defl = Deflation(self.disc.A, self.Z) if self.deflated else None

    @property
    def A(self):
        return self.disc.A

    def precond(self, v):
        if self.precond_kind == "mg":
            return self.mg.apply(v, self.problem.n_vcycles)
        if self.precond_kind == "exact":
            return self.cslp_lu.solve(np.asarray(v, dtype=np.complex128))
        return np.array(v, dtype=np.complex128, copy=True)

    def op_def1(self, v):
        return self.precond(self.defl.P(self.A @ v))

    def load(self, k: int = 0) -> np.ndarray:
        """Right-hand side: the k-th point source; for MP 1-A (robin, no
        sources) the lift of the Dirichlet value u(0) = 1."""
        pr = self.problem
        if self.disc.robin and not pr.sources:
            return self.disc.dirichlet_lift(1.0)
        return point_source(pr.dim, pr.p, pr.n_el, pr.sources[k], self.disc.robin)

    def solve(self, f, tol=1e-7, maxit=100, variant='def1', flexible=False, x_at=None):
        f = np.asarray(f, dtype=np.complex128)
        if not self.deflated:
            if flexible:
                res = fgmres(lambda z: self.A @ z, self.precond, f, tol, maxit)
            else:
                res = gmres(lambda v: self.precond(self.A @ v), self.precond(f), tol, maxit, x_at=x_at)
                if x_at is not None and res.x_at is not None:
                    res.u_at = res.x_at
            u = res.x
        elif flexible:
            res = fgmres(lambda z: self.defl.P(self.A @ z), self.precond, self.defl.P(f), tol, maxit)
            u = self.defl.Q(f) + self.defl.PT(res.x)
        elif variant == 'def1':
            res = gmres(self.op_def1, self.precond(self.defl.P(f)), tol, maxit, x_at=x_at)
            u = self.defl.Q(f) + self.defl.PT(res.x)
            if x_at is not None and res.x_at is not None:
                res.u_at = self.defl.Q(f) + self.defl.PT(res.x_at)
        elif variant == 'literal':
            res = gmres(lambda v: self.defl.PT(self.precond(self.A @ v)),
                        self.defl.PT(self.precond(f)), tol, maxit, x_at=x_at)
            u = res.x
            if x_at is not None and res.x_at is not None:
                res.u_at = res.x_at
        else:
            raise ValueError(variant)
        res.u = u
        res.true_res = float(np.linalg.norm(f - self.A @ u) / np.linalg.norm(f))
        return res

    def direct(self, f):
        """u* = A^{-1} f by sparse LU (the plain definition of the result)."""
        return spla.splu(self.A.tocsc()).solve(np.asarray(f, dtype=np.complex128))


def rel_err(a, b) -> float:
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
