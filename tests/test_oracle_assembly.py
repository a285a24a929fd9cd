"""Pins for oracle.assembly: textbook element matrices, invariants, closed-form
solutions and the paper's convergence orders (Section 4.1, Table 1)."""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import workloads as W
from oracle import assembly as asm
from oracle.solver import Solver

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_p1_textbook_matrices():
    n_el = 10
    h = 1.0 / n_el
    K, M, _ = asm.assemble_1d(n_el, 1)
    K, M = K.toarray(), M.toarray()
    # interior row: (1/h)(-1, 2, -1) and (h/6)(1, 4, 1)
    i = 5
    np.testing.assert_allclose(K[i, i - 1:i + 2], np.array([-1, 2, -1]) / h, rtol=1e-14)
    np.testing.assert_allclose(M[i, i - 1:i + 2], np.array([1, 4, 1]) * h / 6, rtol=1e-14)
    # end rows: element matrices (1/h)[1 -1; -1 1], (h/6)[2 1; 1 2]
    np.testing.assert_allclose(K[0, :2], np.array([1, -1]) / h, rtol=1e-14)
    np.testing.assert_allclose(M[0, :2], np.array([2, 1]) * h / 6, rtol=1e-14)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_1d_invariants(p):
    K, M, _ = asm.assemble_1d(9, p)
    K, M = K.toarray(), M.toarray()
    np.testing.assert_allclose(K.sum(axis=1), 0.0, atol=1e-11)   # constants in kernel
    assert abs(M.sum() - 1.0) < 1e-14                            # |Omega| = 1
    np.testing.assert_allclose(K, K.T, atol=1e-12)
    np.testing.assert_allclose(M, M.T, atol=1e-15)
    assert np.all(np.linalg.eigvalsh(M) > 0)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_2d_invariants_and_tensor_structure(p):
    kf = W.constant_k(3.0)
    n_el = 6
    S, M, Mk = asm.assemble_2d(n_el, p, kf)
    np.testing.assert_allclose(np.asarray(S.sum(axis=1)).ravel(), 0.0, atol=1e-11)
    assert abs(M.sum() - 1.0) < 1e-13
    np.testing.assert_allclose((Mk - 9.0 * M).toarray(), 0.0, atol=1e-13)
    # tensor Gauss quadrature must reproduce Kronecker products of the 1D matrices
    K1, M1, _ = asm.assemble_1d(n_el, p)
    S_kron = sp.kron(M1, K1) + sp.kron(K1, M1)
    np.testing.assert_allclose(S.toarray(), S_kron.toarray(), atol=1e-12)
    np.testing.assert_allclose(M.toarray(), sp.kron(M1, M1).toarray(), atol=1e-15)


def test_variable_k_mass_layers():
    """Piecewise-constant k: M^{k^2} = sum of k_l^2 * (mass restricted to layer l);
    with all values equal it is k^2 M; on an element wholly inside one layer the
    local matrix is k_l^2 times the plain local matrix."""
    kf = W.three_layer_field(0.1)       # 10 / 15 / 25
    n_el, p = 10, 2
    S, M, Mk = asm.assemble_2d(n_el, p, kf)
    # bounds: 100 M <= Mk <= 625 M entrywise on the diagonal
    d, dm = Mk.diagonal(), M.diagonal()
    assert np.all(d >= 100 * dm * (1 - 1e-14)) and np.all(d <= 625 * dm * (1 + 1e-14))
    same = W.KField(values=(7.0, 7.0, 7.0), lines=kf.lines)
    _, M2, Mk2 = asm.assemble_2d(n_el, p, same)
    np.testing.assert_allclose(Mk2.toarray(), 49 * M2.toarray(), rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_generalised_eigenvalues_converge(p):
    """Dirichlet eigenvalues of -u'' are j^2 pi^2 (Section 3); the IgA
    generalised eigenvalues converge at rate h^{2p}."""
    errs = []
    for n_el in (8, 16, 32):
        K, M, _ = asm.assemble_1d(n_el, p)
        K, M = asm.interior_1d(K).toarray(), asm.interior_1d(M).toarray()
        lam = sla.eigh(K, M, eigvals_only=True)[:3]
        exact = (np.arange(1, 4) * np.pi) ** 2
        errs.append(np.max(np.abs(lam - exact) / exact))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 2 * p - 0.3), rates


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_manufactured_l2_rate(p):
    """-u'' - k^2 u = f with u = sin(3 pi x): L2 error O(h^{p+1}) (Section 4.1)."""
    k = 5.0
    u = lambda x: np.sin(3 * np.pi * x)
    f = lambda x: ((3 * np.pi) ** 2 - k * k) * np.sin(3 * np.pi * x)
    errs = []
    for n_el in (8, 16, 32):
        K, M, _ = asm.assemble_1d(n_el, p)
        A = asm.interior_1d(K - k * k * M).toarray()
        b = asm.l2_load_1d(n_el, p, f)
        c = np.linalg.solve(A, b)
        errs.append(asm.l2_error_1d(n_el, p, np.concatenate([[0], c, [0]]), u))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > p + 1 - 0.25), rates


def test_mp1b_greens_function():
    """MP 1-B: the series of Section 2.1 sums to
    G(x, x') = sin(k x_<) sin(k (1 - x_>)) / (k sin k); the IgA solution
    approaches it under refinement."""
    k, x0 = 10.0, 0.5
    G = lambda x: np.where(x < x0, np.sin(k * x) * np.sin(k * (1 - x0)),
                           np.sin(k * x0) * np.sin(k * (1 - x))) / (k * np.sin(k))
    # series check of the closed form at a few points (independent of the oracle)
    xs = np.array([0.1, 0.3, 0.7])
    j = np.arange(1, 200001)
    series = 2 * np.sum(np.sin(j[None, :] * np.pi * xs[:, None]) * np.sin(j * np.pi * x0)
                        / (j ** 2 * np.pi ** 2 - k * k), axis=1)
    np.testing.assert_allclose(series, G(xs), atol=1e-5)
    for p in (1, 2, 3):
        errs = []
        for n_el in (8, 16, 32, 64):
            pr = W.Problem(dim=1, p=p, n_el=n_el, kfield=W.constant_k(k), sources=[(x0,)])
            s = Solver(pr)
            u = s.direct(s.load())
            errs.append(asm.l2_error_1d(n_el, p, np.concatenate([[0], u, [0]]), G))
        assert all(e1 < e0 for e0, e1 in zip(errs, errs[1:])), errs
        # the kink at x' limits the rate for C^{p-1} splines, but it stays >= ~1.5
        assert np.log2(errs[-2] / errs[-1]) > 1.4, errs
        gnorm = asm.l2_error_1d(64, 1, np.zeros(65), G)
        assert errs[-1] < 0.05 * gnorm, (errs, gnorm)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_mp1a_table1_rates(p):
    """MP 1-A at k = 1 (Section 4.1, Table 1): the L2 error decays as h^{p+1}.
    Only the rates are pinned: the table's absolute values use an error norm
    the paper does not define."""
    g = json.load(open(os.path.join(GOLD, "table1_mp1a_l2.json")))
    paper = np.array(g[f"p{p}"])
    ns = g["n_el"][:3] if p < 4 else [4, 8, 16]
    errs = []
    for n_el in ns:
        c = asm.mp1a_solve(n_el, p, 1.0)
        errs.append(asm.l2_error_1d(n_el, p, c, lambda x: np.exp(1j * x), nq=12))
    ours = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(ours - (p + 1)) < 0.3), ours
    if p < 4:
        theirs = np.log2(paper[:2] / paper[1:3])
        assert np.all(np.abs(theirs - (p + 1)) < 0.3), theirs


def test_dense_bruteforce_equals_sparse_lu():
    pr = W.small_2d(n_el=10, p=2, k=8.0)
    s = Solver(pr)
    f = s.load()
    u = s.direct(f)
    u2 = np.linalg.solve(s.A.toarray(), f)
    np.testing.assert_allclose(u, u2, rtol=1e-10, atol=1e-14)


def test_point_source_partition_of_unity():
    for p in (1, 2, 4):
        f = asm.point_source(2, p, 12, (0.5, 0.5))
        assert abs(f.sum() - 1.0) < 1e-14      # boundary functions vanish at the centre


def test_three_layer_k_at_hand_chosen_points():
    """The three-layer field read for MP 2-B (interfaces y = 0.30 + 0.20 x and
    y = 0.70 - 0.15 x; k = 100 below the first, 150 between, 250 above the
    second; a point on an interface belongs to the layer above it).  Expected
    values written by hand from that description, not from the KField
    coefficients: points inside each layer, exactly on each line (where the
    floating-point sums are exact), just below each line, the four corners,
    and points that tell the two slopes apart."""
    kf = W.three_layer_field()
    pts = [
        # (x, y, k): inside the layers
        (0.5, 0.10, 100.0), (0.5, 0.50, 150.0), (0.5, 0.90, 250.0),
        # exactly on a line at x = 0 (a*x = 0, so ((a x) + y) + c is exactly 0)
        (0.0, 0.30, 150.0), (0.0, 0.70, 250.0),
        # exactly on the first line at x = 1 (y = 0.5: 0.5 - 0.2 - 0.3 rounds to 0)
        (1.0, 0.50, 150.0),
        # just below each line
        (0.0, 0.30 - 1e-9, 100.0), (0.0, 0.70 - 1e-9, 150.0),
        # corners
        (0.0, 0.0, 100.0), (1.0, 0.0, 100.0), (0.0, 1.0, 250.0), (1.0, 1.0, 250.0),
        # slopes: the second line falls with x (0.685 at x = 0.1, 0.565 at x = 0.9),
        # the first rises (0.32 at x = 0.1, 0.48 at x = 0.9)
        (0.1, 0.62, 150.0), (0.9, 0.62, 250.0), (0.1, 0.40, 150.0), (0.9, 0.40, 100.0),
    ]
    x = np.array([p[0] for p in pts])
    y = np.array([p[1] for p in pts])
    want = np.array([p[2] for p in pts])
    np.testing.assert_array_equal(asm.k_of(kf, x, y), want)
    # the scaled field multiplies every layer value
    np.testing.assert_array_equal(asm.k_of(W.three_layer_field(2.0), x, y), 2.0 * want)
