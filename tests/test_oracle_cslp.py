"""Pins for the oracle's CSLP operator and its preconditioner modes (paper
Section 3, CSLP equation; Section 4.3.1, Tables 2 and 3: D, C_ex; Section
4.3.2, Table 5).

The shift form is pinned two ways: by closed-form eigenvalues (1D, p = 1,
uniform knots: S, M and I share the eigenvectors sin(j pi x_i)), and by the
paper's own Table 2, whose C_ex counts (5 for every k and p) the mass-matrix
form reproduces and the identity form printed in the CSLP equation does not.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import assembly as asm
from oracle import multigrid as mg
from oracle.krylov import gmres
from oracle.solver import Solver, rel_err

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("uses_mass", [True, False])
def test_shift_forms_closed_form_eigenvalues(uses_mass):
    """1D, p = 1, n_el uniform elements, Dirichlet: interior S = (1/h)
    tridiag(-1, 2, -1), M = (h/6) tridiag(1, 4, 1); v_j = sin(j pi i h) gives
    S v = (2/h)(1 - cos(j pi h)) v and M v = (h/3)(2 + cos(j pi h)) v.  Hence
    M_beta v = (lS - (b1 - i b2) k^2 lM) v for the mass form and
    (lS - b1 k^2 lM + i b2 k^2) v for the identity form."""
    n_el, k, b1, b2 = 24, 7.0, 1.0, 0.5
    h = 1.0 / n_el
    d = asm.Discretization(1, 1, n_el, W.constant_k(k))
    Mb = d.shifted(b1, b2, uses_mass)
    i = np.arange(1, n_el)
    for j in (1, 5, 17, 23):
        v = np.sin(j * np.pi * i * h)
        lS = (2.0 / h) * (1.0 - np.cos(j * np.pi * h))
        lM = (h / 3.0) * (2.0 + np.cos(j * np.pi * h))
        lam = lS - (b1 - 1j * b2) * k * k * lM if uses_mass else lS - b1 * k * k * lM + 1j * b2 * k * k
        np.testing.assert_allclose(Mb @ v, lam * v, rtol=0, atol=1e-11 * abs(lam))


def _table2():
    return json.load(open(os.path.join(GOLD, "table2_3_mp1b_iterations.json")))


def _mp1b(k, p, **kw):
    n_el = int(round(k / W.KH))
    return W.Problem(dim=1, p=p, n_el=n_el, kfield=W.constant_k(k), sources=[(0.5,)], **kw)


@pytest.mark.parametrize("k", [100.0, 1000.0])
def test_cex_table2_soft_pin(k):
    """C_ex with beta_2 = 1/k (Section 4.3.1, Table 2): the paper prints 5
    iterations for every k and p.  The mass-shift reading gives a count within
    one of that, the same for every p and both k; the identity form printed in
    the CSLP equation needs 40 or more (up to the 100 cap), so the paper's
    numbers were not produced by it."""
    g = _table2()
    counts = []
    for p in (1, 2, 3, 4, 5):
        s = Solver(_mp1b(k, p, shift=(1.0, 1.0 / k), precond="exact", deflation=False))
        r = s.solve(s.load())
        assert r.converged and r.true_res < 1e-6
        assert abs(r.iters - g["cex"][str(p)]) <= 1, (p, r.iters)
        counts.append(r.iters)
    assert len(set(counts)) == 1, counts
    s = Solver(_mp1b(k, 2, shift=(1.0, 1.0 / k), precond="exact", deflation=False, shift_uses_mass=False))
    r = s.solve(s.load())
    assert r.iters >= 40, r.iters


def test_deflation_only_table2_soft_pin():
    """D (ADP alone, no CSLP; Section 4.3.1, Table 2) at k = 100 and 1000:
    within three iterations of the paper's counts (its level of detail leaves
    the Z boundary rows and the stopping residual open)."""
    g = _table2()
    for k in (100.0, 1000.0):
        for p in (1, 2, 3, 4, 5):
            s = Solver(_mp1b(k, p, n_vcycles=0))
            assert s.precond_kind == "none"
            r = s.solve(s.load())
            paper = g["d"][str(int(k))][str(p)]
            assert r.converged and abs(r.iters - paper) <= 3, (k, p, r.iters, paper)
            assert rel_err(r.u, s.direct(s.load())) < 1e-5


@pytest.mark.parametrize("uses_mass", [True, False])
def test_cex_spectrum_on_circle(uses_mass):
    """beta_1 = 1: A = M_beta - i beta_2 k^2 B (B = M or I), so every
    eigenvalue mu of M_beta^{-1} A is x / (x + i b) with x real, i.e. on the
    circle |mu - 1/2| = 1/2 (2D constant k, dense)."""
    pr = W.small_2d(n_el=8, p=2, k=9.0)
    pr.shift = (1.0, 0.3)
    d = asm.Discretization(2, 2, 8, pr.kfield)
    Mb = d.shifted(1.0, 0.3, uses_mass).toarray()
    mu = np.linalg.eigvals(np.linalg.solve(Mb, d.A.toarray()))
    np.testing.assert_allclose(np.abs(mu - 0.5), 0.5, atol=1e-10)


def test_cex_without_deflation_solves():
    """C_ex alone (no deflation): GMRES on M_beta^{-1} A u = M_beta^{-1} f gives
    the direct solution; its iterate after j steps is the brute-force
    minimiser over the Krylov space of the dense M_beta^{-1} A."""
    pr = W.small_2d(n_el=12, p=3, k=10.0)
    pr.precond, pr.deflation, pr.shift = "exact", False, (1.0, 1.0 / 30.0)
    s = Solver(pr)
    f = s.load()
    r = s.solve(f, tol=1e-12, maxit=200)
    assert r.converged and rel_err(r.u, s.direct(f)) < 1e-9
    B = np.linalg.solve(s.cslp.toarray(), s.A.toarray())
    b = np.linalg.solve(s.cslp.toarray(), f)
    for j in (2, 5):
        rj = s.solve(f, tol=0.0, maxit=j)
        K = np.stack([np.linalg.matrix_power(B, i) @ b for i in range(j)], axis=1)
        c, *_ = np.linalg.lstsq(B @ K, b, rcond=None)
        np.testing.assert_allclose(rj.u, K @ c, rtol=1e-8, atol=1e-12 * np.abs(K @ c).max())


@pytest.mark.parametrize("p,grows", [(1, False), (2, False), (3, True)])
def test_twelve_cycle_iteration_with_jacobi_smoother(p, grows):
    """Section 4.3.2's C_MG^12 setting (beta_2 = 4.2, three pre- and
    post-sweeps) with Section 3's damped Jacobi (omega = 0.6) as the
    stationary iteration x <- x + V(b - M_beta x): it contracts for p <= 2
    and grows for p = 3, where omega times the largest eigenvalue of
    D^{-1} M_beta on the mass-dominated modes passes 2."""
    n_el, k = 64, 40.0
    pr = W.small_2d(n_el=n_el, p=p, k=k)
    hier = mg.MGHierarchy(2, p, n_el, pr.kfield, 1.0, 4.2, nu_pre=3, nu_post=3)
    b = W.seeded_complex_vector(pr.n_x ** 2, 1)
    Mb = hier.levels[0].Mb
    x = np.zeros_like(b)
    for _ in range(12):
        x = x + hier.vcycle(b - Mb @ x)
    res = np.linalg.norm(b - Mb @ x) / np.linalg.norm(b)
    assert (res > 1e3) if grows else (res < 1e-3), res
