"""Pins for oracle.bspline against the paper's Section 2.3.1 and Fig. 2."""
import json
import os

import numpy as np
import pytest

from oracle import bspline

GOLD = os.path.join(os.path.dirname(__file__), "golden", "fig2_bsplines.json")


def _closed_form(pieces, x):
    out = np.zeros_like(x)
    for lo, hi, expr in pieces:
        m = (x >= lo) & (x < hi)
        out[m] = eval(expr, {"x": x[m]}) if expr != "0" else 0.0
    return out


@pytest.mark.parametrize("key_knots,key_fun,p", [("xi1", "p1", 1), ("xi2", "p2", 2)])
def test_fig2_closed_forms(key_knots, key_fun, p):
    g = json.load(open(GOLD))
    t = np.array(g[key_knots], dtype=float)
    x = np.linspace(0.0, 3.0, 301)[:-1] + 0.0037          # avoid no breakpoint issue, stay < 3
    x = x[x < 3.0]
    phi = bspline.basis_all(t, p, x)
    assert phi.shape[0] == len(g[key_fun])
    for j, pieces in enumerate(g[key_fun]):
        np.testing.assert_allclose(phi[j], _closed_form(pieces, x), rtol=0, atol=1e-14)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_partition_of_unity_nonneg_interpolatory(p):
    t = bspline.open_uniform_knots(7, p)
    x = np.concatenate([np.linspace(0, 1, 513), [0.0, 1.0]])
    phi = bspline.basis_all(t, p, x)
    np.testing.assert_allclose(phi.sum(axis=0), 1.0, atol=1e-14)
    assert phi.min() >= -1e-15
    # interpolatory at both ends (Section 2.3.1)
    e0 = bspline.basis_all(t, p, [0.0])[:, 0]
    e1 = bspline.basis_all(t, p, [1.0])[:, 0]
    assert e0[0] == 1.0 and np.all(e0[1:] == 0.0)
    assert e1[-1] == 1.0 and np.all(e1[:-1] == 0.0)


@pytest.mark.parametrize("p", [1, 2, 3, 5])
def test_derivative_vs_central_difference(p):
    t = bspline.open_uniform_knots(6, p)
    x = np.linspace(0.013, 0.987, 97)
    hstep = 1e-6
    fd = (bspline.basis_all(t, p, x + hstep) - bspline.basis_all(t, p, x - hstep)) / (2 * hstep)
    d = bspline.basis_deriv_all(t, p, x)
    # skip points within hstep of a knot
    ok = np.min(np.abs(x[None, :] - t[:, None]), axis=0) > 2 * hstep
    np.testing.assert_allclose(d[:, ok], fd[:, ok], atol=5e-6 * max(1, 6 ** p))


def test_knots_are_single_divisions():
    for n_el in (5, 80, 320, 640, 1280):
        for p in (1, 3, 5):
            t = bspline.open_uniform_knots(n_el, p)
            assert len(t) == n_el + 2 * p + 1
            assert np.all(t[:p + 1] == 0.0) and np.all(t[-p - 1:] == 1.0)
            for i in range(1, n_el):
                assert t[p + i] == i / n_el
    # nested: the coarse knots are every other fine knot, bit for bit
    tf, tc = bspline.open_uniform_knots(640, 3), bspline.open_uniform_knots(320, 3)
    assert np.array_equal(tf[3:-3][::2], tc[3:-3])


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_windowed_basis_equals_global_recursion(p):
    """The per-span evaluation on knot windows (used for large meshes) gives
    bit for bit the values and derivatives of the global recursion."""
    from oracle import assembly as asm
    n_el = 300
    B, D, xq, _ = asm.local_tables(n_el, p)
    t = bspline.open_uniform_knots(n_el, p)
    pts = xq.reshape(-1)
    phi, dphi = bspline.basis_all(t, p, pts), bspline.basis_deriv_all(t, p, pts)
    nq = p + 1
    for e in range(n_el):
        cols = slice(e * nq, (e + 1) * nq)
        assert np.array_equal(B[e], phi[e:e + p + 1, cols].T)
        assert np.array_equal(D[e], dphi[e:e + p + 1, cols].T)
