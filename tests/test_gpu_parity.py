"""GPU-vs-oracle parity of every step of the hot path, called through the C ABI.

Tolerances: knots/indices bit-exact; FP64 operators 1e-13 relative (a few
ulps of rounding-order difference, times the band width); FP64 V-cycle and
deflation 1e-11 (rounding amplified by the coarse solves); full GMRES solve
1e-10 relative L2 against the oracle run with the same iteration count, as the
contract for the FP64 path states; the FP32 V-cycle 1e-4 (single-precision
storage and accumulation)."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import bspline
from oracle import assembly as asm
from oracle import multigrid as mg
from oracle import deflation as dfl
from oracle.solver import Solver, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2010_10232_gb300.solver import Helmholtz, IgaError, from_problem  # noqa: E402

CASES = {
    "1d_p2": W.config1()[0],
    "2d_p1": W.small_2d(n_el=40, p=1, k=15.0),
    "2d_p2": W.small_2d(n_el=34, p=2, k=15.0),
    "2d_p3": W.small_2d(n_el=40, p=3, k=20.0),
    "2d_p4": W.small_2d(n_el=24, p=4, k=12.0),
    "2d_p5": W.small_2d(n_el=20, p=5, k=10.0),
    "2d_var_p2": W.small_2d(n_el=32, p=2, k=20.0, layered=True),
    "2d_var_p3": W.small_2d(n_el=36, p=3, k=20.0, layered=True),
}
_cache = {}


def ctx_and_oracle(name):
    if name not in _cache:
        pr = CASES[name]
        _cache[name] = (from_problem(pr), Solver(pr), pr)
    return _cache[name]


def to_t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def to_n(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rvec(n, seed):
    return W.seeded_complex_vector(n, seed)


ALL = list(CASES)
CONST2D = [c for c in ALL if c.startswith("2d_p")]


# ------------------------------------------------------------------ setup tables
@pytest.mark.parametrize("name", ALL)
def test_knots_bitexact_and_levels(name):
    h, s, pr = ctx_and_oracle(name)
    sizes = mg.level_sizes(pr.n_el)
    assert h.levels == len(sizes)
    for l, ne in enumerate(sizes):
        assert h.level_nel(l) == ne
        assert h.level_nx(l) == ne + pr.p - 2
        k_gpu = h.knots(l)
        k_ora = bspline.open_uniform_knots(ne, pr.p)
        assert k_gpu.tobytes() == k_ora.tobytes()


@pytest.mark.parametrize("name", ["1d_p2", "2d_p1", "2d_p3", "2d_p5"])
def test_band_matrices(name):
    h, s, pr = ctx_and_oracle(name)
    for l, ne in enumerate(mg.level_sizes(pr.n_el)):
        K, M, _ = asm.assemble_1d(ne, pr.p)
        K, M = asm.interior_1d(K).toarray(), asm.interior_1d(M).toarray()
        for which, ref in ((0, K), (1, M)):
            band = h.band(l, which)
            n = ref.shape[0]
            dense = np.zeros((n, n))
            for i in range(n):
                for d in range(-pr.p, pr.p + 1):
                    if 0 <= i + d < n:
                        dense[i, i + d] = band[i, d + pr.p]
            assert np.max(np.abs(dense - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("name", ["1d_p2", "2d_p1", "2d_p2", "2d_p3", "2d_p4", "2d_p5"])
def test_knot_insertion_prolongation(name):
    h, s, pr = ctx_and_oracle(name)
    for l in range(h.levels - 1):
        ref = mg.prolongation_interior_1d(h.level_nel(l + 1), pr.p)
        np.testing.assert_allclose(h.prolongation(l), ref, rtol=0, atol=1e-14)


# ------------------------------------------------------------------ operators
@pytest.mark.parametrize("name", ALL)
def test_apply_A(name):
    h, s, pr = ctx_and_oracle(name)
    x = rvec(h.n, 11)
    y = to_n(h.apply_A(to_t(x)))
    ref = s.A @ x
    assert rel_err(y, ref) <= 1e-13


@pytest.mark.parametrize("name", ALL)
def test_apply_Mshift_every_level(name):
    h, s, pr = ctx_and_oracle(name)
    for l, lvl in enumerate(s.mg.levels):
        n = lvl.Mb.shape[0]
        x = rvec(n, 20 + l)
        y = to_n(h.apply_Mshift(l, to_t(x)))
        assert rel_err(y, lvl.Mb @ x) <= 1e-13, l


@pytest.mark.parametrize("name", ["1d_p2", "2d_p2", "2d_p3", "2d_var_p3"])
def test_jacobi_sweeps(name):
    h, s, pr = ctx_and_oracle(name)
    for l in (0, 1):
        lvl = s.mg.levels[l]
        n = lvl.Mb.shape[0]
        b, x0 = rvec(n, 30), rvec(n, 31)
        for sweeps in (1, 2, 3):
            ref = s.mg.jacobi(lvl, x0.copy(), b, sweeps)
            got = to_n(h.jacobi(l, to_t(b), to_t(x0), sweeps))
            assert rel_err(got, ref) <= 1e-13


@pytest.mark.parametrize("name", ["1d_p2", "2d_p1", "2d_p3", "2d_p5", "2d_var_p2"])
def test_restrict_prolong(name):
    h, s, pr = ctx_and_oracle(name)
    for l in range(h.levels - 1):
        P = s.mg.P[l]
        nf, nc = P.shape
        r = rvec(nf, 40 + l)
        assert rel_err(to_n(h.restrict(l, to_t(r))), P.T @ r) <= 1e-14
        c, f = rvec(nc, 50 + l), rvec(nf, 60 + l)
        got = to_n(h.prolong_add(l, to_t(c), to_t(f)))
        assert rel_err(got, f + P @ c) <= 1e-14


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_transfer_interior_stencil(p):
    """On levels large enough to have interior tiles, the tiled restriction
    takes the uniform-knot interior stencil of the knot-insertion table (edge
    tiles keep the table): restriction and prolongation in FP64 against the
    oracle's transfer matrices, and the FP64 and FP32 V-cycles against the
    oracle's V-cycle.
    The V-cycle bounds at p >= 4 are its own rounding at this size (k = 192):
    the table-only kernels gave 3.2e-11 (FP64, p = 5) and 1.17e-3 (FP32,
    p = 4, bit for bit the same as with the stencil) on the same inputs."""
    n_el = 320
    pr = W.small_2d(n_el=n_el, p=p, k=0.6 * n_el)
    h = from_problem(pr, skip_deflation=1)
    hier = mg.MGHierarchy(2, p, n_el, pr.kfield, 1.0, 0.5)
    for l in range(3):
        P = hier.P[l]
        nf, nc = P.shape
        r = rvec(nf, 140 + l)
        assert rel_err(to_n(h.restrict(l, to_t(r))), P.T @ r) <= 1e-13, l
        c, f = rvec(nc, 150 + l), rvec(nf, 160 + l)
        assert rel_err(to_n(h.prolong_add(l, to_t(c), to_t(f))), f + P @ c) <= 1e-13, l
    r = rvec(h.n, 170)
    ref = hier.apply(r, 1)
    assert rel_err(to_n(h.vcycle(to_t(r))), ref) <= (1e-11 if p <= 4 else 1e-10)
    if p <= 4:     # at p = 5 the FP32 V-cycle's own rounding reaches ~1e-2 at this size
        h32 = from_problem(pr, skip_deflation=1, precision=1)
        assert rel_err(to_n(h32.vcycle(to_t(r))), ref) <= (1e-4 if p <= 3 else 3e-3)


@pytest.mark.parametrize("name", ALL)
def test_coarse_solve(name):
    h, s, pr = ctx_and_oracle(name)
    b = rvec(s.mg.coarse_dense.shape[0], 70)
    got = to_n(h.coarse_solve(to_t(b)))
    assert rel_err(got, np.linalg.solve(s.mg.coarse_dense, b)) <= 1e-11


@pytest.mark.parametrize("name", ALL)
def test_vcycle_fp64(name):
    h, s, pr = ctx_and_oracle(name)
    r = rvec(h.n, 80)
    got = to_n(h.vcycle(to_t(r)))
    assert rel_err(got, s.mg.apply(r, 1)) <= 1e-11


@pytest.mark.parametrize("nu,cycles", [(2, 1), (3, 2), (0, 1)])
def test_vcycle_fp64_variants(nu, cycles):
    pr = W.small_2d(n_el=32, p=3, k=15.0)
    pr.nu_pre = nu
    pr.nu_post = max(nu, 1)
    pr.n_vcycles = cycles
    h = from_problem(pr)
    hier = mg.MGHierarchy(2, 3, 32, pr.kfield, 1.0, 0.5, nu_pre=pr.nu_pre, nu_post=pr.nu_post)
    r = rvec(h.n, 81)
    assert rel_err(to_n(h.vcycle(to_t(r))), hier.apply(r, cycles)) <= 1e-11


def test_twelve_vcycles_large_shift():
    """The Section 4.3.2 multigrid setting (beta_2 = 4.2, three pre- and
    post-sweeps, 12 V-cycles as a stationary iteration) at p = 2."""
    pr = W.small_2d(n_el=64, p=2, k=40.0)
    pr.nu_pre = pr.nu_post = 3
    pr.n_vcycles = 12
    pr.shift = (1.0, 4.2)
    h = from_problem(pr)
    hier = mg.MGHierarchy(2, 2, 64, pr.kfield, 1.0, 4.2, nu_pre=3, nu_post=3)
    r = rvec(h.n, 86)
    assert rel_err(to_n(h.vcycle(to_t(r))), hier.apply(r, 12)) <= 1e-11


@pytest.mark.parametrize("name", ["2d_p3", "2d_var_p3", "1d_p2"])
def test_vcycle_fp32(name):
    pr = CASES[name]
    h = from_problem(pr, precision=1)
    s = ctx_and_oracle(name)[1]
    r = rvec(h.n, 82)
    assert rel_err(to_n(h.vcycle(to_t(r))), s.mg.apply(r, 1)) <= 1e-4


# ------------------------------------------------------------------ deflation
@pytest.mark.parametrize("name", ALL)
def test_zt_z(name):
    h, s, pr = ctx_and_oracle(name)
    Z = s.Z
    x = rvec(h.n, 90)
    assert rel_err(to_n(h.zt(to_t(x))), Z.T @ x) <= 1e-14
    c = rvec(h.m, 91)
    assert rel_err(to_n(h.z(to_t(c))), Z @ c) <= 1e-14


@pytest.mark.parametrize("tile", range(6))
@pytest.mark.parametrize("name", ["2d_p1", "2d_p3", "2d_p5"])
def test_every_tile_shape(name, tile):
    """Each operator tile shape, forced on every level (FP64; the FP32 V-cycle
    with the shapes FP32 has), against the oracle: the apply, the per-level
    M_beta, Jacobi sweeps, the V-cycle, and the E solve whose refinement
    residual takes the tile of the level of nearest size."""
    pr = CASES[name]
    s = ctx_and_oracle(name)[1]
    h = from_problem(pr)
    for l in range(h.levels):
        h.set_tile(l, 0, tile)
        assert h.tile(l, 0) == tile
    x = rvec(h.n, 11)
    assert rel_err(to_n(h.apply_A(to_t(x))), s.A @ x) <= 1e-13
    for l, lvl in enumerate(s.mg.levels):
        xl = rvec(lvl.Mb.shape[0], 20 + l)
        assert rel_err(to_n(h.apply_Mshift(l, to_t(xl))), lvl.Mb @ xl) <= 1e-13, l
    for l in (0, 1):
        lvl = s.mg.levels[l]
        b, x0 = rvec(lvl.Mb.shape[0], 30), rvec(lvl.Mb.shape[0], 31)
        got = to_n(h.jacobi(l, to_t(b), to_t(x0), 2))
        assert rel_err(got, s.mg.jacobi(lvl, x0.copy(), b, 2)) <= 1e-13, l
    r = rvec(h.n, 80)
    assert rel_err(to_n(h.vcycle(to_t(r))), s.mg.apply(r, 1)) <= 1e-11
    t = rvec(h.m, 92)
    assert rel_err(to_n(h.esolve(to_t(t))), s.defl.lu.solve(t)) <= 1e-10
    if tile <= 3:
        h32 = from_problem(pr, precision=1)
        for l in range(h32.levels):
            h32.set_tile(l, 1, tile)
        assert rel_err(to_n(h32.vcycle(to_t(r))), s.mg.apply(r, 1)) <= 1e-4
    else:
        with pytest.raises(IgaError):
            h.set_tile(0, 1, tile)
    with pytest.raises(IgaError):
        h.set_tile(h.levels, 0, 0)


@pytest.mark.parametrize("name", ALL)
def test_esolve_and_deflate(name):
    h, s, pr = ctx_and_oracle(name)
    t = rvec(h.m, 92)
    ref = s.defl.lu.solve(t)
    assert rel_err(to_n(h.esolve(to_t(t))), ref) <= 1e-10
    x = rvec(h.n, 93)
    assert rel_err(to_n(h.deflate(to_t(x))), s.defl.P(x)) <= 1e-10


def test_eps_weighted_stencil():
    pr = W.small_2d(n_el=24, p=2, k=12.0)
    pr.eps = 0.37
    h = from_problem(pr)
    Z = dfl.z_matrix(2, pr.n_x, 0.37)
    x = rvec(h.n, 94)
    assert rel_err(to_n(h.zt(to_t(x))), Z.T @ x) <= 1e-14


# ------------------------------------------------------------------ load + Arnoldi
@pytest.mark.parametrize("name", ["1d_p2", "2d_p2", "2d_p3", "2d_p5"])
def test_point_source(name):
    h, s, pr = ctx_and_oracle(name)
    for pos in ((0.5, 0.5), (0.1234, 0.8765), (0.0, 1.0), (1.0, 0.25)):
        ref = asm.point_source(pr.dim, pr.p, pr.n_el, pos[:pr.dim])
        got = to_n(h.point_source(*pos))
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-15)


def test_mgs_matches_numpy():
    h, s, pr = ctx_and_oracle("2d_p3")
    n = h.n
    k = 6
    rng = np.random.default_rng(5)
    Vn = np.linalg.qr(rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k)))[0]
    w = rvec(n, 95)
    for j in (0, 2, 5):
        ww = w.copy()
        hs = []
        for i in range(j + 1):
            hi = np.vdot(Vn[:, i], ww)
            hs.append(hi)
            ww = ww - hi * Vn[:, i]
        hs.append(np.linalg.norm(ww))
        wt = to_t(w)
        hg = to_n(h.mgs(to_t(Vn.T.copy()), j, wt))
        np.testing.assert_allclose(hg, np.array(hs), rtol=1e-12, atol=1e-12)
        assert rel_err(to_n(wt), ww) <= 1e-12


# ------------------------------------------------------------------ solve
def _solve_pair(name, f, tol=1e-7, maxit=100):
    h, s, pr = ctx_and_oracle(name)
    x, it, hist, tr, st = h.solve(to_t(f), tol=tol, maxit=maxit)
    r = s.solve(f, tol=tol, maxit=maxit)
    return to_n(x), it, hist, tr, st, r


@pytest.mark.parametrize("name", ALL)
def test_solve_point_source(name):
    """Solve to 1e-7: iteration count within one of the oracle's, residual
    histories equal, the solution equal to the oracle's at 1e-10 (when the
    counts differ, both sides are re-run for the smaller count with tol = 0 and
    those iterates compared), and the reported true residual within 10x the
    tolerance and within a factor 10 of the last residual estimate."""
    h, s, pr = ctx_and_oracle(name)
    f = s.load()
    x, it, hist, tr, st, r = _solve_pair(name, f)
    assert st == 0 and r.converged
    assert abs(it - r.iters) <= 1
    m = min(it, r.iters)
    np.testing.assert_allclose(hist[:m + 1], np.array(r.hist)[:m + 1], rtol=1e-6)
    if it == r.iters:
        assert rel_err(x, r.u) <= 1e-10
    else:
        xm, itm, *_ = h.solve(to_t(f), tol=0.0, maxit=m)
        rm = s.solve(f, tol=0.0, maxit=m)
        assert itm == m and rel_err(to_n(xm), rm.u) <= 1e-10
    assert tr <= 10 * 1e-7
    assert 0.1 * hist[-1] <= tr <= 10 * hist[-1]
    true_res = np.linalg.norm(f - s.A @ x) / np.linalg.norm(f)
    assert abs(true_res - tr) <= 1e-6 * tr + 1e-15
    err_direct = rel_err(x, s.direct(f))
    print(f"{name}: iters gpu={it} oracle={r.iters} true_res={tr:.2e} err_vs_direct={err_direct:.2e}")


def test_solve_config1_seeded_rhs():
    h, s, pr = ctx_and_oracle("1d_p2")
    f = W.seeded_normal_rhs(h.n, 0).astype(np.complex128)
    x, it, hist, tr, st, r = _solve_pair("1d_p2", f)
    assert st == 0 and it == r.iters
    assert rel_err(x, r.u) <= 1e-10


@pytest.mark.parametrize("name", ["2d_p2", "2d_p3", "2d_var_p3"])
def test_iterates_at_same_count(name):
    """FP64 path vs oracle at a fixed iteration count (tol = 0)."""
    h, s, pr = ctx_and_oracle(name)
    f = s.load()
    for j in (1, 3, 6):
        x, it, hist, tr, st = h.solve(to_t(f), tol=0.0, maxit=j)
        assert st == 1 and it == j                        # IGA_NOT_CONVERGED
        r = s.solve(f, tol=0.0, maxit=j)
        assert rel_err(to_n(x), r.u) <= 1e-10


def test_flexible_fp64_matches_oracle_fgmres():
    name = "2d_p3"
    pr = CASES[name]
    s = ctx_and_oracle(name)[1]
    h = from_problem(pr, flexible=1)
    f = s.load()
    x, it, hist, tr, st = h.solve(to_t(f))
    r = s.solve(f, flexible=True)
    assert st == 0 and abs(it - r.iters) <= 1
    if it == r.iters:
        assert rel_err(to_n(x), r.u) <= 1e-10


@pytest.mark.parametrize("name", ["2d_p3", "2d_var_p3"])
def test_mixed_precision_solve(name):
    pr = CASES[name]
    s = ctx_and_oracle(name)[1]
    h = from_problem(pr, precision=1)
    f = s.load()
    x, it, hist, tr, st = h.solve(to_t(f), tol=1e-9)
    assert st == 0
    assert rel_err(to_n(x), s.direct(f)) <= 1e-6


def test_solve_host_matches_device():
    h, s, pr = ctx_and_oracle("2d_p2")
    f = s.load()
    xd, it1, *_ = h.solve(to_t(f))
    xh, it2, *_ = h.solve_host(f)
    assert it1 == it2
    assert rel_err(xh, to_n(xd)) <= 1e-14


def test_error_statuses():
    h, s, pr = ctx_and_oracle("2d_p2")
    f = to_t(s.load())
    # maxit reached -> IGA_NOT_CONVERGED with valid outputs
    x, it, hist, tr, st = h.solve(f, tol=1e-14, maxit=2)
    assert st == 1 and it == 2
    # misaligned pointer -> IGA_E_INVALID, nothing launched
    buf = torch.zeros(2 * h.n + 2, dtype=torch.float64, device="cuda")
    import ctypes
    rc = h._L.iga_apply_A(h._h, ctypes.c_void_p(buf.data_ptr() + 8), ctypes.c_void_p(f.data_ptr()))
    assert rc == -1
    with pytest.raises(IgaError):
        h.apply_A(f, f)                       # aliasing rejected


# ------------------------------------------------------------------ full size (bench configuration)
@pytest.fixture(scope="module")
def cfg2_full():
    pr = W.config2(k=200.0, p=3)
    return from_problem(pr), Solver(pr), pr


def test_full_size_apply_sampled(cfg2_full):
    """320 x 320 elements, p = 3: full A x compared row by row with the oracle's
    assembled matrix on 4096 sampled rows."""
    h, s, pr = cfg2_full
    x = rvec(h.n, 100)
    y = to_n(h.apply_A(to_t(x)))
    rows = np.random.default_rng(0).choice(h.n, 4096, replace=False)
    ref = s.A[rows] @ x
    assert rel_err(y[rows], ref) <= 1e-13


def test_full_size_solve(cfg2_full):
    """At 320 x 320, k = 200, p = 3 the coarse matrix E is nearly singular
    (min |lambda_i + lambda_j - k^2| = 0.022, cond ~ 2e7) and the GMRES iterate
    is only determined to ~1e-6 by its data: a 1e-15 relative perturbation of f
    moves the oracle's own iterate by ~2e-6.  Both sides run the oracle's
    iteration count with tol = 0 (no +-1 ambiguity) and the GPU-oracle gap must
    stay within ten times that measured self-sensitivity; the 1e-10 contract
    is checked at full size on the well-conditioned p = 1 case below."""
    h, s, pr = cfg2_full
    f = s.load()
    x, it, hist, tr, st = h.solve(to_t(f))
    r = s.solve(f)
    assert st == 0 and abs(it - r.iters) <= 1
    m = r.iters
    xm, itm, *_ = h.solve(to_t(f), tol=0.0, maxit=m)
    rm = s.solve(f, tol=0.0, maxit=m)
    f2 = f * (1 + 1e-15 * W.seeded_normal_rhs(len(f), 9))
    r2 = s.solve(f2, tol=0.0, maxit=m)
    self_sens = rel_err(r2.u, rm.u)
    gap = rel_err(to_n(xm), rm.u)
    ud = s.direct(f)
    print(f"cfg2 k=200 p=3: iters gpu={it} oracle={r.iters} true_res={tr:.2e} gap@{m}={gap:.2e} "
          f"oracle_self_sensitivity={self_sens:.2e} err_vs_direct gpu={rel_err(to_n(x), ud):.2e} "
          f"oracle={rel_err(r.u, ud):.2e}")
    assert itm == m
    assert gap <= max(1e-10, 10 * self_sens)
    assert rel_err(to_n(x), ud) <= 2 * rel_err(r.u, ud) + 1e-9


def test_full_size_solve_contract_p1():
    """Full bench size with p = 1 (320 x 320 elements, k = 200, 101 761 dofs),
    where the problem is well conditioned (a 1e-15 relative perturbation of f
    moves the oracle's result by ~5e-14): the 1e-7 solve takes the oracle's
    iteration count (+-1), and at the oracle's count (tol = 0) the GPU iterate
    equals the oracle's to 1e-10."""
    pr = W.config2(k=200.0, p=1)
    h, s = from_problem(pr), Solver(pr)
    f = s.load()
    x, it, hist, tr, st = h.solve(to_t(f))
    r = s.solve(f)
    assert st == 0 and abs(it - r.iters) <= 1
    xm, itm, *_ = h.solve(to_t(f), tol=0.0, maxit=r.iters)
    rm = s.solve(f, tol=0.0, maxit=r.iters)
    assert itm == r.iters
    gap = rel_err(to_n(xm), rm.u)
    print(f"cfg2 k=200 p=1: iters gpu={it} oracle={r.iters} gap={gap:.2e}")
    assert gap <= 1e-10


@pytest.mark.parametrize("n_el,p", [(40, 3), (46, 3), (64, 2), (96, 5), (152, 3)])
def test_esolve_fdm_sizes(n_el, p):
    """E^{-1} t by the refined FP32 fast diagonalisation against the oracle's
    sparse LU (odd m_x, m_x not a multiple of the GEMM tiles, p = 2..5)."""
    pr = W.small_2d(n_el=n_el, p=p, k=0.55 * n_el)
    h = from_problem(pr)
    s = Solver(pr)
    t = rvec(h.m, 95)
    assert rel_err(to_n(h.esolve(to_t(t))), s.defl.lu.solve(t)) <= 1e-10


@pytest.mark.parametrize("p", [2, 3])
def test_esolve_register_blocked_transforms(p):
    """m_x above 192: the fast-diagonalisation transforms of the E solve run
    on the register-blocked GEMM; E^{-1} t against the oracle's sparse LU of
    Z^T A Z, and the exact CSLP inverse of a 258^2-dof level against the
    oracle's sparse LU of M_beta."""
    n_el = 416
    pr = W.small_2d(n_el=n_el, p=p, k=0.55 * n_el)
    h, s = from_problem(pr), Solver(pr)
    assert int(round(h.m ** 0.5)) > 192
    t = rvec(h.m, 97)
    assert rel_err(to_n(h.esolve(to_t(t))), s.defl.lu.solve(t)) <= 1e-10
    pc = W.small_2d(n_el=256, p=p, k=100.0)
    pc.precond, pc.deflation, pc.shift = "exact", False, (1.0, 1.0 / 300.0)
    hc, sc = from_problem(pc), Solver(pc)
    r = rvec(hc.n, 98)
    assert rel_err(to_n(hc.precond(to_t(r))), sc.cslp_lu.solve(r)) <= 1e-10


def test_coarsest_level_too_large_is_rejected():
    """n_el = 150 halves once (75 is odd): the 76^2-dof coarsest level is refused
    by the setup with IGA_E_INVALID instead of a failing launch."""
    with pytest.raises(IgaError) as ei:
        Helmholtz(dim=2, p=3, n_el=150, kfield=50.0)
    assert "INVALID" in str(ei.value)


@pytest.mark.slow
def test_esolve_large_coarse_grid_residual():
    """m_x = 312 (four output rows per block in the two-launch pass): too large
    for the oracle's sparse LU in test time, so the device result is checked by
    its residual against the oracle's Galerkin matrix E = Z^T A Z."""
    n_el, p = 624, 3
    pr = W.small_2d(n_el=n_el, p=p, k=0.55 * n_el)
    h = from_problem(pr)
    d = asm.Discretization(2, p, n_el, pr.kfield)
    Z = dfl.z_matrix(2, d.n_x, pr.eps)
    E = (Z.T @ d.A @ Z).tocsr()
    t = rvec(h.m, 96)
    s = to_n(h.esolve(to_t(t)))
    assert np.linalg.norm(t - E @ s) <= 1e-11 * np.linalg.norm(t)


@pytest.mark.parametrize("n_el,p,cycles", [(32, 1, 1), (48, 2, 1), (40, 3, 2), (40, 4, 1), (24, 5, 1), (256, 3, 1)])
def test_vcycle_fused_levels(n_el, p, cycles):
    """The fused level kernels (residual + restriction, prolongation + post-sweep,
    pre-sweep recomputed) against the oracle's V-cycle and the per-operation
    kernels, FP64 and FP32."""
    pr = W.small_2d(n_el=n_el, p=p, k=0.6 * n_el)
    pr.n_vcycles = cycles
    hier = mg.MGHierarchy(2, p, n_el, pr.kfield, 1.0, 0.5)
    r = rvec(pr.n_x ** 2, 83)
    ref = hier.apply(r, cycles)
    for prec in (0, 1):
        hf = from_problem(pr, precision=prec, skip_deflation=1, fused_vcycle=1)
        hu = from_problem(pr, precision=prec, skip_deflation=1, fused_vcycle=0)
        ef = rel_err(to_n(hf.vcycle(to_t(r))), ref)
        eu = rel_err(to_n(hu.vcycle(to_t(r))), ref)
        if prec == 0:
            assert ef <= 1e-11 and eu <= 1e-11
        else:
            # FP32: the fused kernels are as accurate as the per-operation
            # kernels (both carry the FP32 rounding of the V-cycle, which
            # grows with p), and both stay within 1e-3 of the FP64 result
            assert ef <= max(2.0 * eu, 1e-5) and ef <= 1e-3, (ef, eu)


@pytest.fixture(scope="module")
def cfg3_full():
    pr = W.config3()
    d = asm.Discretization(2, pr.p, pr.n_el, pr.kfield)
    return pr, d


@pytest.mark.slow
def test_config3_full_size_apply_and_solves(cfg3_full):
    """Three-layer k (100/150/250), p = 3, 640 x 640 elements (410 881 dofs): the
    oracle's sparse direct solve is out of reach at this size, so the check is by
    properties the oracle can compute: sampled rows of A x against the oracle's
    assembled matrix, and the true residual ||f - A u|| / ||f|| of the FP64 and
    the FP32-V-cycle solutions of the first source, evaluated with that matrix,
    against the residual the library reports."""
    pr, d = cfg3_full
    h64 = from_problem(pr)
    x = rvec(h64.n, 101)
    y = to_n(h64.apply_A(to_t(x)))
    rows = np.random.default_rng(1).choice(h64.n, 4096, replace=False)
    assert rel_err(y[rows], d.A[rows] @ x) <= 1e-13
    f = asm.point_source(2, pr.p, pr.n_el, pr.sources[0])
    for prec in (0, 1):
        h = h64 if prec == 0 else from_problem(pr, precision=1)
        u, it, hist, tr, st = h.solve(to_t(f), tol=1e-7, maxit=100)
        assert st == 0 and 0 < it < 100
        un = to_n(u)
        true_res = np.linalg.norm(f - d.A @ un) / np.linalg.norm(f)
        assert abs(true_res - tr) <= 1e-6 * tr + 1e-14
        assert np.all(np.isfinite(un))


@pytest.mark.parametrize("n_el,p,k", [(40, 1, 15.0), (34, 2, 15.0), (256, 3, 150.0), (24, 4, 12.0), (20, 5, 10.0),
                                      (160, 5, 100.0)])
def test_fp32_register_stencil_sweep(n_el, p, k):
    """The FP32 register-stencil sweep (tile code 6: interior tiles take the
    uniform-knot stencil from registers, edge tiles their own band rows)
    forced on every level: the FP32 V-cycle stays within the FP32 tolerance
    of the oracle and within FP32 rounding of the shared-memory tile kernel."""
    pr = W.small_2d(n_el=n_el, p=p, k=k)
    hier = mg.MGHierarchy(2, p, n_el, pr.kfield, 1.0, 0.5)
    r = rvec(pr.n_x ** 2, 84)
    ref = hier.apply(r, 1)
    h6 = from_problem(pr, precision=1, skip_deflation=1)
    h0 = from_problem(pr, precision=1, skip_deflation=1)
    for l in range(h6.levels):
        h6.set_tile(l, 1, 6)
        h0.set_tile(l, 1, 0)
        assert h6.tile(l, 1) == 6
    z6 = to_n(h6.vcycle(to_t(r)))
    z0 = to_n(h0.vcycle(to_t(r)))
    e0, e6 = rel_err(z0, ref), rel_err(z6, ref)
    print(f"n_el={n_el} p={p}: FP32 V-cycle error tile 0 {e0:.2e}, tile 6 {e6:.2e}, gap {rel_err(z6, z0):.2e}")
    # both carry the FP32 rounding of the V-cycle (it grows with p); the two
    # kernels round in different orders, so they agree to that level
    assert e6 <= max(1e-4, 2.0 * e0)
    assert rel_err(z6, z0) <= max(2e-6, 2.0 * e0)


@pytest.mark.parametrize("n_el,p,k", [(40, 1, 15.0), (128, 3, 80.0), (20, 5, 10.0), (200, 5, 100.0)])
@pytest.mark.parametrize("tile", [0, 1, 2, 3, 6])
def test_fp32_operator_and_sweep_every_tile(n_el, p, k, tile):
    """FP32 M_beta x and one FP32 damped Jacobi sweep on every level, each FP32
    tile shape forced, against the oracle's FP64 level operator applied to the
    same complex64 inputs: FP32 rounding (a few ulps times the band width)."""
    pr = W.small_2d(n_el=n_el, p=p, k=k)
    hier = mg.MGHierarchy(2, p, n_el, pr.kfield, 1.0, 0.5)
    h = from_problem(pr, precision=1, skip_deflation=1)
    for l, lvl in enumerate(hier.levels):
        h.set_tile(l, 1, tile)
        n = lvl.Mb.shape[0]
        x = rvec(n, 300 + l).astype(np.complex64)
        b = rvec(n, 400 + l).astype(np.complex64)
        xt = torch.from_numpy(x).cuda()
        bt = torch.from_numpy(b).cuda()
        y = h.apply_Mshift32(l, xt)
        ref = lvl.Mb @ x.astype(np.complex128)
        assert rel_err(to_n(y).astype(np.complex128), ref) <= 2e-6, l
        xo = h.jacobi32(l, bt, xt)
        refj = hier.jacobi(lvl, x.astype(np.complex128), b.astype(np.complex128), 1)
        assert rel_err(to_n(xo).astype(np.complex128), refj) <= 2e-6, l


@pytest.mark.parametrize("n_el,p,k", [(256, 3, 150.0), (128, 2, 70.0), (40, 5, 20.0)])
def test_fp32_vcycle_folded_conversions(n_el, p, k):
    """The FP32 V-cycle with complex128 input and output folds the two
    conversions into its first and last finest-level kernels when the finest
    level runs the register-stencil sweep.  Against converting, running the
    FP32 V-cycle and converting back (the path taken when a network is
    attached; a network whose output is NaN is dropped, so it adds nothing),
    the result agrees to FP32 rounding as the V-cycle amplifies it, and both
    stay within the FP32 tolerance of the FP64 oracle."""
    from paper_2010_10232_gb300.learned import Net
    pr = W.small_2d(n_el=n_el, p=p, k=k)
    h = from_problem(pr, precision=1, skip_deflation=1)
    h.set_tile(0, 1, 6)
    r = to_t(rvec(h.n, 85))
    z_fold = to_n(h.vcycle(r))
    net = Net(seed=1)
    net.set_params(np.full(net.num_params, np.nan, dtype=np.float32))
    h.attach(net, 1.0)
    z_conv = to_n(h.vcycle(r))
    h.attach(None)
    ref = mg.MGHierarchy(2, p, n_el, pr.kfield, 1.0, 0.5).apply(rvec(h.n, 85), 1)
    e_conv = rel_err(z_conv, ref)
    print(f"n_el={n_el} p={p}: folded vs converted {rel_err(z_fold, z_conv):.2e}, converted vs oracle {e_conv:.2e}")
    assert rel_err(z_fold, z_conv) <= max(1e-5, 2.0 * e_conv)
    assert rel_err(z_fold, ref) <= max(1e-4, 3.0 * e_conv)
