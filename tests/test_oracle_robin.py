"""Pins for the oracle's Sommerfeld boundary and Dirichlet lifting (MP 1-A,
Section 2.1; the boundary mass N of Section 2.3's linear system), written
independently of oracle.assembly.mp1a_solve, which is a plain direct
assembly of the same problem."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import assembly as asm
from oracle import multigrid as mg
from oracle.solver import Solver, rel_err

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("k", [1.0, 20.0])
def test_robin_discretisation_matches_direct_assembly(p, k):
    """The Solver's MP 1-A system (last function kept, -i k N, the lift of
    u(0) = 1) has the solution of the plain direct assembly."""
    pr = W.mp1a(k, p, 32)
    s = Solver(pr)
    assert s.disc.n_x == pr.n_x == 32 + p - 1 and pr.ndof == s.disc.n
    assert W.small_2d(n_el=32, p=p).n_x == 32 + p - 2
    u = s.direct(s.load())
    np.testing.assert_allclose(u, asm.mp1a_solve(32, p, k)[1:], rtol=0, atol=1e-12 * np.abs(u).max())


@pytest.mark.parametrize("p", [1, 2, 3])
def test_robin_gmres_table1_rates(p):
    """MP 1-A at k = 1 (Section 4.1, Table 1) solved by the deflated,
    CSLP-preconditioned GMRES: the L2 error against exp(i k x) decays as
    h^{p+1}, as the paper's table does."""
    g = json.load(open(os.path.join(GOLD, "table1_mp1a_l2.json")))
    errs = []
    for n_el in g["n_el"][:3]:
        s = Solver(W.mp1a(1.0, p, n_el))
        r = s.solve(s.load(), tol=1e-12, maxit=200)
        assert r.converged and r.true_res < 1e-10
        full = np.concatenate([[1.0 + 0j], r.u])
        errs.append(asm.l2_error_1d(n_el, p, full, lambda x: np.exp(1j * x), nq=12))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - (p + 1)) < 0.3), rates


@pytest.mark.parametrize("p", [1, 2, 3])
def test_robin_coarse_levels_are_galerkin(p):
    """With the Sommerfeld end kept, knot insertion keeps the last coefficient,
    so the rediscretised coarse CSLP operator (including its boundary term)
    equals the Galerkin product P^T M_beta P for constant k."""
    h = mg.MGHierarchy(1, p, 32, W.constant_k(7.0), 1.0, 0.5, robin=True)
    for li in range(len(h.levels) - 1):
        gal = (h.P[li].T @ h.levels[li].Mb @ h.P[li]).toarray()
        np.testing.assert_allclose(gal, h.levels[li + 1].Mb.toarray(), atol=1e-10 * np.abs(gal).max())


def test_robin_boundary_term_sign():
    """A plane wave exp(i k x) sampled by the exact solution satisfies the
    outgoing condition: the continuous problem's solution is reproduced to
    discretisation error, and the opposite sign of the boundary term (an
    incoming condition) is not (its solution differs at O(1))."""
    k, p, n_el = 10.0, 3, 64
    s = Solver(W.mp1a(k, p, n_el))
    full = np.concatenate([[1.0 + 0j], s.direct(s.load())])
    err = asm.l2_error_1d(n_el, p, full, lambda x: np.exp(1j * k * x), nq=12)
    assert err < 1e-5
    bad = s.disc.A + 2j * k * s.disc.N          # the same system with +i k N
    import scipy.sparse.linalg as spla
    fb = np.concatenate([[1.0 + 0j], spla.spsolve(bad.tocsc(), s.load())])
    assert asm.l2_error_1d(n_el, p, fb, lambda x: np.exp(1j * k * x), nq=12) > 0.1
