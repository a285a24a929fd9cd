"""Knot vectors and B-spline evaluation (paper Section 2.3.1, "B-spline basis functions").

Test infrastructure only (see oracle/__init__.py).

Pins (tests/test_oracle_bspline.py): Fig. 2 closed forms on Xi_1 and Xi_2,
partition of unity, non-negativity, interpolation at the ends, derivative vs
central differences.
"""
from __future__ import annotations

import numpy as np


def open_uniform_knots(n_el: int, p: int) -> np.ndarray:
    """Open uniform knot vector on [0, 1] (Section 2.3.1): knot span h = 1/n_el,
    first and last knot repeated p+1 times.  Interior knots are i/n_el computed
    by one IEEE division each (never by accumulating h)."""
    interior = [float(i) / float(n_el) for i in range(1, n_el)]
    return np.array([0.0] * (p + 1) + interior + [1.0] * (p + 1), dtype=np.float64)


def n_basis(knots: np.ndarray, p: int) -> int:
    return len(knots) - p - 1


def basis_all(knots: np.ndarray, p: int, x) -> np.ndarray:
    """Values of all N = len(knots)-p-1 B-splines of degree p at points x.

    Direct use of the Cox-de Boor recursion of Section 2.3.1: degree 0 on the
    half-open span [xi_j, xi_{j+1}), then
        phi_{j,q} = (x - xi_j)/(xi_{j+q} - xi_j) phi_{j,q-1}
                  + (xi_{j+q+1} - x)/(xi_{j+q+1} - xi_{j+1}) phi_{j+1,q-1},
    with a term dropped when its denominator is zero.  The right end point
    x = xi_last is assigned to the last non-empty span (reading: the half-open
    convention would make every function vanish there).
    Returns an array of shape (N, len(x)).
    """
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    t = knots
    m = len(t) - 1
    phi = np.zeros((m, x.size))
    for j in range(m):
        phi[j] = (t[j] <= x) & (x < t[j + 1])
    # right end: last non-empty span
    last = max(j for j in range(m) if t[j] < t[j + 1])
    phi[last, x == t[-1]] = 1.0
    for q in range(1, p + 1):
        new = np.zeros((m - q, x.size))
        for j in range(m - q):
            d1 = t[j + q] - t[j]
            d2 = t[j + q + 1] - t[j + 1]
            term = np.zeros(x.size)
            if d1 != 0.0:
                term = term + (x - t[j]) / d1 * phi[j]
            if d2 != 0.0:
                term = term + (t[j + q + 1] - x) / d2 * phi[j + 1]
            new[j] = term
        phi = new
    return phi


def basis_windows(tw: np.ndarray, p: int, x: np.ndarray) -> np.ndarray:
    """basis_all for many knot windows at once: tw[e] holds 2p+2 knots and
    x[e] points inside its middle span (span p, so no point is a knot and the
    right-end rule never applies); the same recursion, term by term, as
    basis_all on each window.  Returns shape (E, p+1, len(x[e]))."""
    E, nx = x.shape
    m = tw.shape[1] - 1
    phi = np.zeros((E, m, nx))
    for j in range(m):
        phi[:, j] = (tw[:, j, None] <= x) & (x < tw[:, j + 1, None])
    with np.errstate(divide="ignore", invalid="ignore"):
        for q in range(1, p + 1):
            new = np.zeros((E, m - q, nx))
            for j in range(m - q):
                d1 = (tw[:, j + q] - tw[:, j])[:, None]
                d2 = (tw[:, j + q + 1] - tw[:, j + 1])[:, None]
                term = np.zeros((E, nx))
                term = term + np.where(d1 != 0.0, (x - tw[:, j, None]) / d1 * phi[:, j], 0.0)
                term = term + np.where(d2 != 0.0, (tw[:, j + q + 1, None] - x) / d2 * phi[:, j + 1], 0.0)
                new[:, j] = term
            phi = new
    return phi


def basis_deriv_windows(tw: np.ndarray, p: int, x: np.ndarray) -> np.ndarray:
    """basis_deriv_all for many knot windows at once (as basis_windows)."""
    E, nx = x.shape
    if p == 0:
        return np.zeros((E, 1, nx))
    low = basis_windows(tw, p - 1, x)
    d = np.zeros((E, p + 1, nx))
    with np.errstate(divide="ignore", invalid="ignore"):
        for j in range(p + 1):
            d1 = (tw[:, j + p] - tw[:, j])[:, None]
            d2 = (tw[:, j + p + 1] - tw[:, j + 1])[:, None]
            d[:, j] = d[:, j] + np.where(d1 != 0.0, p / d1 * low[:, j], 0.0)
            d[:, j] = d[:, j] - np.where(d2 != 0.0, p / d2 * low[:, j + 1], 0.0)
    return d


def basis_deriv_all(knots: np.ndarray, p: int, x) -> np.ndarray:
    """First derivatives of all degree-p B-splines at x, by differentiating the
    recursion (de Boor): phi'_{j,p} = p/(xi_{j+p}-xi_j) phi_{j,p-1}
    - p/(xi_{j+p+1}-xi_{j+1}) phi_{j+1,p-1}, zero-denominator terms dropped."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    t = knots
    if p == 0:
        return np.zeros((n_basis(t, 0), x.size))
    low = basis_all(t, p - 1, x)          # shape (len(t)-p, nx)
    nb = n_basis(t, p)
    d = np.zeros((nb, x.size))
    for j in range(nb):
        d1 = t[j + p] - t[j]
        d2 = t[j + p + 1] - t[j + 1]
        if d1 != 0.0:
            d[j] += p / d1 * low[j]
        if d2 != 0.0:
            d[j] -= p / d2 * low[j + 1]
    return d


def gauss_legendre(nq: int):
    """Gauss-Legendre nodes and weights on [-1, 1] (library routine)."""
    g, w = np.polynomial.legendre.leggauss(nq)
    return g, w


def element_quadrature(knots: np.ndarray, p: int, nq: int | None = None):
    """Per non-empty knot span e: mapped Gauss points and weights.

    A Gauss point of span [a, b] is x = a + (b - a) * ((1 + g) / 2), evaluated
    in that order in IEEE double; its weight is w * (b - a) / 2.
    Returns (xq[e, q], wq[e, q], spans[e] = (a, b))."""
    if nq is None:
        nq = p + 1
    g, w = gauss_legendre(nq)
    spans = [(knots[j], knots[j + 1]) for j in range(len(knots) - 1) if knots[j] < knots[j + 1]]
    xq = np.array([[a + (b - a) * ((1.0 + gi) / 2.0) for gi in g] for a, b in spans])
    wq = np.array([[wi * (b - a) / 2.0 for wi in w] for a, b in spans])
    return xq, wq, spans
