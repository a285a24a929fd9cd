"""The 1D band solver (partitioned LU with partial pivoting, spikes and an
interface system) in its three uses, against the oracle's sparse / dense LU:
E = Z^T A Z of the deflation (Section 3, Eq. adef1: E inverted exactly), the
exactly inverted CSLP C_ex (Section 4.3) and a coarsest multigrid level above
the dense-inverse limit; then the 1D scaling of Section 4.3.1 (Tables 2-4)
at k = 10^4 against the oracle and at k = 10^5 by the true residual."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import multigrid as mg
from oracle.solver import Solver, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2010_10232_gb300.solver import from_problem  # noqa: E402

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def to_t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def to_n(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def mp1b(k, p, n_el=None, **kw):
    """MP 1-B (Section 2.1): 1D Dirichlet, point source at x = 1/2, kh = 0.625."""
    n_el = n_el or int(round(k / W.KH))
    return W.Problem(dim=1, p=p, n_el=n_el, kfield=W.constant_k(k), sources=[(0.5,)], **kw)


# n_el = 40: a small constant-k E (m_x <= 192), solved by the dense fast
# diagonalisation; 400 / 2000: the band solver with several partitions and the
# interface system
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("n_el,k", [(40, 20.0), (400, 250.0), (2000, 1250.0)])
def test_banded_E_solve(p, n_el, k):
    pr = mp1b(k, p, n_el)
    h, s = from_problem(pr), Solver(pr)
    t = W.seeded_complex_vector(h.m, 7)
    ref = s.defl.lu.solve(t)
    got = to_n(h.esolve(to_t(t)))
    assert rel_err(got, ref) <= 1e-10
    x = W.seeded_complex_vector(h.n, 8)
    assert rel_err(to_n(h.deflate(to_t(x))), s.defl.P(x)) <= 1e-10


@pytest.mark.parametrize("p", [1, 3, 5])
def test_banded_E_with_sommerfeld_end_and_eps(p):
    """MP 1-A's E carries -i k N in its last rows; the epsilon-weighted Z."""
    pr = W.mp1a(300.0, p, 480)
    pr.eps = 0.3
    h, s = from_problem(pr), Solver(pr)
    t = W.seeded_complex_vector(h.m, 9)
    assert rel_err(to_n(h.esolve(to_t(t))), s.defl.lu.solve(t)) <= 1e-10


@pytest.mark.parametrize("p", [1, 2, 5])
@pytest.mark.parametrize("robin", [False, True])
def test_banded_exact_cslp(p, robin):
    """C_ex in 1D: z = M_beta^{-1} r by the band solver (beta_2 = 1/k, Table 2),
    several partitions; with the Sommerfeld end as well."""
    k = 600.0
    pr = W.mp1a(k, p, 960) if robin else mp1b(k, p)
    pr.precond, pr.deflation, pr.shift = "exact", False, (1.0, 1.0 / k)
    h, s = from_problem(pr), Solver(pr)
    r = W.seeded_complex_vector(h.n, 10)
    assert rel_err(to_n(h.precond(to_t(r))), s.cslp_lu.solve(r)) <= 1e-11


@pytest.mark.parametrize("p", [1, 3, 5])
def test_banded_coarsest_level(p):
    """n_el = 4102 halves once to 2051 elements: the coarsest level (2051 + p - 2
    dofs) is above the dense-inverse limit and goes to the band solver; the
    coarse solve, the FP64 V-cycle and the FP32 V-cycle against the oracle."""
    k = 0.6 * 4102
    pr = mp1b(k, p, 4102)
    h = from_problem(pr, skip_deflation=1)
    hier = mg.MGHierarchy(1, p, 4102, pr.kfield, 1.0, 0.5)
    assert h.levels == len(hier.levels) == 2 and h.level_n(1) > 2048
    b = W.seeded_complex_vector(h.level_n(1), 11)
    assert rel_err(to_n(h.coarse_solve(to_t(b))), np.linalg.solve(hier.coarse_dense, b)) <= 1e-11
    r = W.seeded_complex_vector(h.n, 12)
    assert rel_err(to_n(h.vcycle(to_t(r))), hier.apply(r, 1)) <= 1e-11
    h32 = from_problem(pr, skip_deflation=1, precision=1)
    assert rel_err(to_n(h32.vcycle(to_t(r))), hier.apply(r, 1)) <= 1e-4


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_scaling_k1e4_against_oracle(p):
    """k = 10^4 (n_el = 16000, Tables 2 and 4): DC^1_MG and D solve in the
    oracle's iteration count (within one), and the iterates after that many
    steps agree to 1e-8.  (E here is conditioned so that the device's and the
    oracle's E solves differ by ~1e-11; where the GMRES residual stalls for a
    few steps, p = 1, the intermediate least-squares iterates amplify that to
    ~1e-4 at step 4, while the iterate at the converged count is back at the
    1e-10 level.)"""
    for kw in ({}, {"n_vcycles": 0}):
        pr = mp1b(1e4, p, **kw)
        h, s = from_problem(pr), Solver(pr)
        f = s.load()
        x, it, hist, tr, st = h.solve(to_t(f), maxit=100)
        r = s.solve(f, maxit=100)
        assert st == 0 and abs(it - r.iters) <= 1, (p, kw, it, r.iters)
        xj, *_ = h.solve(to_t(f), tol=0.0, maxit=it)
        assert rel_err(to_n(xj), s.solve(f, tol=0.0, maxit=it).u) <= 1e-8
        print(f"k=1e4 p={p} {kw or 'DC1'}: GPU {it}, oracle {r.iters}")


@pytest.mark.parametrize("p", [2, 4])
def test_scaling_k1e5_true_residual(p):
    """k = 10^5 (n_el = 160 000, nine levels, E of ~80 000 unknowns): C_ex and
    DC^1_MG converge, and the recovered solution's true residual
    ||f - A u|| / ||f|| is at the tolerance's level."""
    g = json.load(open(os.path.join(GOLD, "table2_3_mp1b_iterations.json")))
    for name, kw in (("cex", dict(precond="exact", deflation=False, shift=(1.0, 1e-5))), ("dc1", {})):
        pr = mp1b(1e5, p, **kw)
        h = from_problem(pr)
        f = h.point_source(0.5)
        x, it, hist, tr, st = h.solve(f, maxit=100)
        print(f"k=1e5 p={p} {name}: {it} iterations, true residual {tr:.2e}")
        assert st == 0 and tr <= 1e-5
        if name == "cex":
            assert abs(it - g["cex"][str(p)]) <= 1
