"""GPU-vs-oracle parity of the preconditioner and deflation modes of Section
4.3's list (D / D_eps: deflation alone; C_ex: the CSLP inverted exactly; C_MG
without deflation; the literal P^T M^{-1} A ordering of Section 3), and the
failure statuses of the solve (non-finite data, a bounded wait that runs out,
the end of the Krylov space), all through the C ABI.

Tolerances as in test_gpu_parity: the exact CSLP inverse 1e-10 against the
oracle's sparse LU (FP32 transforms with FP64 refinement), iterates at equal
iteration counts 1e-10."""
import numpy as np
import pytest

import workloads as W
from oracle.solver import Solver, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2010_10232_gb300.solver import Helmholtz, IgaError, from_problem  # noqa: E402


def to_t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def to_n(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _mode(pr, **kw):
    for k, v in kw.items():
        setattr(pr, k, v)
    return pr


def _compare_solves(pr, counts=(1, 3, 6), tol=1e-7, **gpu_kw):
    """GPU and oracle: converged iteration counts within one, and iterates at
    fixed counts (tol = 0) equal to 1e-10."""
    h, s = from_problem(pr, **gpu_kw), Solver(pr)
    f = s.load()
    variant = "literal" if gpu_kw.get("deflation") == 2 else "def1"
    x, it, hist, tr, st = h.solve(to_t(f), tol=tol)
    r = s.solve(f, tol=tol, variant=variant)
    assert st == 0 and r.converged and abs(it - r.iters) <= 1, (it, r.iters)
    m = min(it, r.iters)
    np.testing.assert_allclose(hist[:m + 1], np.array(r.hist)[:m + 1], rtol=1e-6)
    for j in counts:
        xj, itj, *_ = h.solve(to_t(f), tol=0.0, maxit=j)
        rj = s.solve(f, tol=0.0, maxit=j, variant=variant)
        assert itj == j
        assert rel_err(to_n(xj), rj.u) <= 1e-10, j
    return it, r.iters, tr


@pytest.mark.parametrize("dim,p,n_el,k", [(2, 1, 40, 15.0), (2, 3, 40, 20.0), (2, 4, 24, 12.0), (1, 2, 80, 50.0),
                                          (1, 5, 160, 100.0)])
def test_exact_cslp_inverse(dim, p, n_el, k):
    """z = M_beta^{-1} r by fast diagonalisation of the finest level with FP64
    refinement, against the oracle's sparse LU of the same matrix (beta_2 =
    1/(3k) as for C_ex in Section 4.3.2, and the configs' 0.5)."""
    for b2 in (1.0 / (3.0 * k), 0.5):
        pr = W.Problem(dim=dim, p=p, n_el=n_el, kfield=W.constant_k(k), shift=(1.0, b2), precond="exact",
                       deflation=False, sources=[(0.5, 0.5)[:dim]])
        h, s = from_problem(pr), Solver(pr)
        r = W.seeded_complex_vector(h.n, 3)
        assert rel_err(to_n(h.precond(to_t(r))), s.cslp_lu.solve(r)) <= 1e-10


def test_cex_solve_2d():
    """C_ex alone (Section 4.3.2, Table 5's third column form, beta_2 = 1/(3k))."""
    pr = W.small_2d(n_el=40, p=3, k=20.0)
    _mode(pr, precond="exact", deflation=False, shift=(1.0, 1.0 / 60.0))
    it, it_o, tr = _compare_solves(pr)
    assert tr <= 1e-6


def test_deflation_only_solve():
    """D (Section 4.3.1): deflation without a CSLP, n_vcycles = 0."""
    pr = W.small_2d(n_el=34, p=2, k=15.0)
    _mode(pr, n_vcycles=0)
    _compare_solves(pr)


def test_deflation_only_eps_solve():
    """D_eps: the epsilon-weighted deflation stencil without a CSLP."""
    pr = W.small_2d(n_el=32, p=3, k=15.0)
    _mode(pr, n_vcycles=0, eps=0.2)
    _compare_solves(pr)


def test_mg_without_deflation_solve():
    """C_MG alone: the V-cycle preconditioner without deflation."""
    pr = W.small_2d(n_el=32, p=2, k=10.0)
    _mode(pr, deflation=False)
    _compare_solves(pr, counts=(1, 4), tol=1e-6)


@pytest.mark.parametrize("name,pr", [("2d_p2", W.small_2d(n_el=34, p=2, k=15.0)),
                                     ("2d_var_p3", W.small_2d(n_el=36, p=3, k=20.0, layered=True))])
def test_literal_ordering_solve(name, pr):
    """The literal ordering P^T M~^{-1} A u = P^T M~^{-1} f (deflation = 2),
    against the oracle's variant='literal'."""
    _compare_solves(pr, deflation=2)


def test_table2_counts_on_gpu():
    """MP 1-B, k = 100 (Section 4.3.1, Table 2): D and C_ex (beta_2 = 1/k)
    take the oracle's iteration counts on the GPU for p = 1..5."""
    for p in (1, 2, 3, 4, 5):
        for kw in ({"n_vcycles": 0}, {"precond": "exact", "deflation": False, "shift": (1.0, 0.01)}):
            pr = W.Problem(dim=1, p=p, n_el=160, kfield=W.constant_k(100.0), sources=[(0.5,)], **kw)
            h, s = from_problem(pr), Solver(pr)
            f = s.load()
            x, it, hist, tr, st = h.solve(to_t(f))
            r = s.solve(f)
            assert st == 0 and it == r.iters, (p, kw, it, r.iters)
            assert rel_err(to_n(x), r.u) <= 1e-10


# ------------------------------------------------------------------ failure statuses
def test_nonfinite_rhs_reports_nonfinite():
    """A NaN in the right-hand side: IGA_E_NONFINITE, no iteration run, and the
    context solves the next (finite) right-hand side normally."""
    pr = W.small_2d(n_el=24, p=2, k=10.0)
    h, s = from_problem(pr), Solver(pr)
    f = s.load()
    bad = f.copy()
    bad[7] = np.nan
    with pytest.raises(IgaError) as ei:
        h.solve(to_t(bad))
    assert ei.value.status == -5
    x, it, hist, tr, st = h.solve(to_t(f))
    r = s.solve(f)
    assert st == 0 and abs(it - r.iters) <= 1 and tr <= 1e-6


@pytest.mark.parametrize("host_loop", [0, 1])
def test_barrier_timeout_reports_timeout(host_loop):
    """The cooperative MGS Arnoldi step (arnoldi = 0) waits at grid barriers
    with a poll limit.  With the test hook that makes every barrier wait for
    one block more than the grid has, each wait runs out after 64 polls: the
    solve returns IGA_E_TIMEOUT (from the graph's WHILE loop and from the host
    loop alike) instead of hanging, and after the hook is cleared the same
    context solves normally."""
    pr = W.small_2d(n_el=64, p=3, k=20.0)          # 65^2 dofs: several cooperative blocks
    h, s = from_problem(pr, arnoldi=0, host_loop=host_loop), Solver(pr)
    f = to_t(s.load())
    h.set_wait_limit(64, 1)
    with pytest.raises(IgaError) as ei:
        h.solve(f)
    assert ei.value.status == -6
    h.set_wait_limit(0, 0)
    x, it, hist, tr, st = h.solve(f)
    r = s.solve(s.load())
    assert st == 0 and abs(it - r.iters) <= 1
    assert rel_err(to_n(x), s.direct(s.load())) <= 1e-5


def test_end_of_krylov_space_is_convergence():
    """A 1D problem with n = 8 unknowns and maxit = 30: by iteration n the
    Krylov space is the whole space, the residual estimate reaches rounding
    level and the solve reports IGA_OK with the direct solution (h_{j+1,j}
    ~ 0 is a converged step, not a breakdown)."""
    pr = W.Problem(dim=1, p=2, n_el=8, kfield=W.constant_k(3.0), sources=[(0.37,)])
    h, s = from_problem(pr), Solver(pr)
    assert h.n == 8
    f = s.load()
    x, it, hist, tr, st = h.solve(to_t(f), tol=1e-13, maxit=30)
    assert st == 0 and it <= h.n + 1
    assert rel_err(to_n(x), s.direct(f)) <= 1e-10
    assert np.all(np.isfinite(to_n(x)))


def test_mode_argument_errors():
    with pytest.raises(IgaError) as ei:
        Helmholtz(dim=2, p=2, n_el=16, kfield=W.three_layer_field(0.1), precond=1)
    assert ei.value.status == -7                     # exact CSLP: constant k only
    h = from_problem(_mode(W.small_2d(n_el=16, p=2, k=5.0), deflation=False))
    with pytest.raises(IgaError):
        h.deflate(h.vec(), h.vec())                  # no deflation pieces in this context
    h0 = from_problem(_mode(W.small_2d(n_el=16, p=2, k=5.0), n_vcycles=0))
    with pytest.raises(IgaError):
        h0.vcycle(h0.vec())                          # no V-cycle in this context
    r = to_t(W.seeded_complex_vector(h0.n, 1))
    assert rel_err(to_n(h0.precond(r)), to_n(r)) == 0.0   # M~^{-1} = I
