"""Batched solves in one CUDA-graph launch (uneven instances, several
right-hand sides each) against the single-solve path and the oracle; the
operator-tile autotuner."""
import numpy as np
import pytest

import workloads as W
from oracle.solver import Solver, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2010_10232_gb300.solver import Helmholtz, from_problem, solve_batched  # noqa: E402


def _instances():
    g = np.random.default_rng(44)
    specs = [(2, 48, 30.0, 0, 2), (3, 64, 40.0, 1, 3), (4, 32, 20.0, 1, 1), (3, 96, 60.0, 0, 2)]
    out = []
    for p, n_el, k, prec, nrhs in specs:
        pr = W.Problem(dim=2, p=p, n_el=n_el, kfield=W.constant_k(k),
                       sources=[tuple(map(float, s)) for s in g.uniform(0.1, 0.9, (nrhs, 2))])
        out.append((pr, prec))
    return out


def test_batched_matches_single_solves():
    inst = _instances()
    ctxs = [from_problem(pr, precision=prec, arnoldi=1) for pr, prec in inst]
    rhs = []
    for (pr, _), h in zip(inst, ctxs):
        rhs.append(torch.stack([h.point_source(*s) for s in pr.sources]))
    xs, its, sts, rc = solve_batched(ctxs, rhs, tol=1e-8, maxit=100)
    torch.cuda.synchronize()
    assert rc == 0
    for b, ((pr, prec), h) in enumerate(zip(inst, ctxs)):
        for r in range(len(pr.sources)):
            x1, it1, hist, tr, st = h.solve(rhs[b][r].contiguous(), tol=1e-8, maxit=100)
            assert sts[b][r] == 0 and st == 0
            assert its[b][r] == it1
            assert rel_err(xs[b][r].cpu().numpy(), x1.cpu().numpy()) <= 1e-12


def test_batched_fp64_instance_vs_oracle():
    pr = W.Problem(dim=2, p=3, n_el=40, kfield=W.constant_k(25.0), sources=[(0.5, 0.5), (0.3, 0.7)])
    h = from_problem(pr)
    s = Solver(pr)
    f = [s.load(0), s.load(1)]
    rhs = [torch.from_numpy(np.stack(f)).cuda()]
    xs, its, sts, rc = solve_batched([h], rhs, tol=1e-7, maxit=100)
    for r in range(2):
        ro = s.solve(f[r])
        assert abs(its[0][r] - ro.iters) <= 1
        if its[0][r] == ro.iters:
            assert rel_err(xs[0][r].cpu().numpy(), ro.u) <= 1e-10


def test_batched_zero_rhs_runs_no_iteration():
    h = from_problem(W.small_2d(n_el=24, p=2, k=10.0))
    rhs = [torch.zeros(2, h.n, dtype=torch.complex128, device="cuda")]
    rhs[0][1] = h.point_source(0.5, 0.5)
    xs, its, sts, rc = solve_batched([h], rhs)
    assert its[0][0] == 0 and sts[0][0] == 0
    assert float(xs[0][0].abs().max()) == 0.0
    assert its[0][1] > 0


def test_autotuner_choices():
    h = Helmholtz(dim=2, p=3, n_el=256, kfield=160.0, skip_deflation=1)
    L = h._L
    for lvl in range(h.levels):
        for prec in (0, 1):
            c = L.iga_tile_choice(h._h, lvl, prec)
            if h.level_nx(lvl) >= 8:
                assert c in ((0, 1, 2, 3, 4, 5) if prec == 0 else (0, 1, 2, 3))
            else:
                assert c == -1
    assert L.iga_tile_choice(h._h, 99, 0) == -2


@pytest.mark.parametrize("precision", [0, 1])
def test_cgs2_arnoldi_matches_mgs_and_oracle(precision):
    """The barrier-free CGS2 Arnoldi (used by the batched launch) gives the same
    iterations as modified Gram-Schmidt and the oracle's solution."""
    pr = W.small_2d(n_el=64, p=3, k=40.0)
    s = Solver(pr)
    f = s.load()
    ud = s.direct(f)
    fd = torch.from_numpy(f).cuda()
    x0, it0, *_ = from_problem(pr, precision=precision, arnoldi=0).solve(fd, tol=1e-9, maxit=120)
    x1, it1, hist, tr, st = from_problem(pr, precision=precision, arnoldi=1).solve(fd, tol=1e-9, maxit=120)
    assert st == 0 and abs(it1 - it0) <= 1
    assert rel_err(x1.cpu().numpy(), ud) <= 1e-6
    assert rel_err(x1.cpu().numpy(), x0.cpu().numpy()) <= 1e-6


def test_sharded_batched_equals_whole_batch():
    """Instances split over two ranks (run one after the other on this GPU:
    independent launches, nothing waits on another rank) give the whole
    batch's iteration counts and solutions."""
    from paper_2010_10232_gb300.sharding import solve_batched_sharded
    probs = [(pr, len(pr.sources)) for pr, _ in _instances()]
    whole, counts_whole = solve_batched_sharded(probs, 0, 1, precision=1)
    assert sorted(whole) == list(range(len(probs)))
    got = {}
    for r in range(2):
        sols, counts = solve_batched_sharded(probs, r, 2, precision=1)
        assert sorted(sols) == sorted(counts)
        for i, v in counts.items():
            assert i not in got
            got[i] = v
            assert rel_err(sols[i].cpu().numpy(), whole[i].cpu().numpy()) <= 1e-12
    assert got == counts_whole
    assert all(st == [0] * len(st) for _, st in got.values())
