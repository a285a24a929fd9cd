"""MP 1-A on the GPU (Section 2.1: Sommerfeld condition u' - i k u = 0 at x = 1,
Dirichlet u(0) = 1; Section 2.3: the boundary mass N of the linear system;
Section 4.1, Table 1) against the oracle, through the C ABI: every piece of
the path with the last basis function kept as an unknown, the deflation solve
with the boundary term in E, the Dirichlet lift, full solves, and the paper's
convergence rates from GPU solutions."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import assembly as asm
from oracle import multigrid as mg
from oracle.solver import Solver, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2010_10232_gb300.solver import Helmholtz, IgaError, from_problem  # noqa: E402

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def to_t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def to_n(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


CASES = [(1, 32, 20.0), (2, 40, 20.0), (3, 32, 12.0), (4, 64, 40.0), (5, 48, 30.0)]


@pytest.mark.parametrize("p,n_el,k", CASES)
def test_robin_operators_and_transfers(p, n_el, k):
    pr = W.mp1a(k, p, n_el)
    h, s = from_problem(pr), Solver(pr)
    assert h.n == n_el + p - 1 == s.disc.n
    x = W.seeded_complex_vector(h.n, 1)
    assert rel_err(to_n(h.apply_A(to_t(x))), s.A @ x) <= 1e-13
    for l, lvl in enumerate(s.mg.levels):
        xl = W.seeded_complex_vector(lvl.Mb.shape[0], 2 + l)
        assert rel_err(to_n(h.apply_Mshift(l, to_t(xl))), lvl.Mb @ xl) <= 1e-13, l
        b, x0 = W.seeded_complex_vector(lvl.Mb.shape[0], 20 + l), W.seeded_complex_vector(lvl.Mb.shape[0], 30 + l)
        got = to_n(h.jacobi(l, to_t(b), to_t(x0), 2))
        assert rel_err(got, s.mg.jacobi(lvl, x0.copy(), b, 2)) <= 1e-13, l
    for l in range(h.levels - 1):
        ref = mg.prolongation_interior_1d(h.level_nel(l + 1), p, robin=True)
        np.testing.assert_allclose(h.prolongation(l), ref, rtol=0, atol=1e-14)
    r = W.seeded_complex_vector(h.n, 3)
    assert rel_err(to_n(h.vcycle(to_t(r))), s.mg.apply(r, 1)) <= 1e-11


@pytest.mark.parametrize("p,n_el,k", CASES)
def test_robin_deflation_boundary_term(p, n_el, k):
    """E = Z^T A Z carries the boundary term -i k Z^T N Z in its last rows; the
    device's band LU of the probed E against the oracle's sparse LU of the
    assembled E, and the projector P."""
    pr = W.mp1a(k, p, n_el)
    h, s = from_problem(pr), Solver(pr)
    t = W.seeded_complex_vector(h.m, 4)
    assert rel_err(to_n(h.esolve(to_t(t))), s.defl.lu.solve(t)) <= 1e-10
    x = W.seeded_complex_vector(h.n, 5)
    assert rel_err(to_n(h.deflate(to_t(x))), s.defl.P(x)) <= 1e-10


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_dirichlet_lift(p):
    pr = W.mp1a(7.0, p, 16)
    h, s = from_problem(pr), Solver(pr)
    got = to_n(h.dirichlet_load(1.0))
    ref = s.disc.dirichlet_lift(1.0)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14 * np.abs(ref).max())
    got2 = to_n(h.dirichlet_load(0.3 - 2.0j))
    np.testing.assert_allclose(got2, s.disc.dirichlet_lift(0.3 - 2.0j), rtol=0, atol=1e-14 * np.abs(got2).max())


@pytest.mark.parametrize("p,n_el,k", CASES + [(2, 160, 100.0)])
def test_mp1a_solve(p, n_el, k):
    """The deflated, CSLP-preconditioned GMRES solve of MP 1-A: iteration
    count within one of the oracle's, iterates at fixed counts to 1e-10, and
    the solution against the direct one."""
    pr = W.mp1a(k, p, n_el)
    h, s = from_problem(pr), Solver(pr)
    f = h.dirichlet_load(1.0)
    fo = s.load()
    x, it, hist, tr, st = h.solve(f)
    r = s.solve(fo)
    assert st == 0 and abs(it - r.iters) <= 1, (it, r.iters)
    for j in (1, 3):
        xj, itj, *_ = h.solve(f, tol=0.0, maxit=j)
        assert rel_err(to_n(xj), s.solve(fo, tol=0.0, maxit=j).u) <= 1e-10
    assert rel_err(to_n(x), s.direct(fo)) <= 1e-5


@pytest.mark.parametrize("p", [1, 2, 3])
def test_table1_rates_from_gpu_solutions(p):
    """Section 4.1, Table 1 (MP 1-A, k = 1): the L2 error of the GPU solution
    (solved to 1e-12) against exp(i k x) decays as h^{p+1}."""
    g = json.load(open(os.path.join(GOLD, "table1_mp1a_l2.json")))
    errs = []
    for n_el in g["n_el"][:3]:
        h = from_problem(W.mp1a(1.0, p, n_el))
        x, it, hist, tr, st = h.solve(h.dirichlet_load(1.0), tol=1e-12, maxit=200)
        assert st == 0
        full = np.concatenate([[1.0 + 0j], to_n(x)])
        ref = asm.mp1a_solve(n_el, p, 1.0)
        assert rel_err(full, ref) <= 1e-9
        errs.append(asm.l2_error_1d(n_el, p, full, lambda x_: np.exp(1j * x_), nq=12))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    print(f"p={p}: L2 errors {errs}, rates {rates}")
    assert np.all(np.abs(rates - (p + 1)) < 0.3), rates


def test_robin_argument_errors():
    with pytest.raises(IgaError) as ei:
        Helmholtz(dim=2, p=2, n_el=16, kfield=5.0, robin=1)
    assert ei.value.status == -7
    h = Helmholtz(dim=1, p=2, n_el=16, kfield=5.0)
    with pytest.raises(IgaError):
        h.dirichlet_load(1.0)                       # needs the Sommerfeld end
