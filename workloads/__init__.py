"""Seeded synthetic workloads shared by the CUDA path's tests/bench and the oracle.

This module holds problem *descriptions* only (sizes, wave numbers, source
positions, layer lines, seeded random right-hand sides).  It contains none of
the method's arithmetic: no basis evaluation, no assembly, no solver step.
Both sides turn these descriptions into load vectors and operators with their
own code.

Model problems follow Section 2 of the paper (MP 1-B: 1D Dirichlet point
source; MP 2-A: 2D Dirichlet point source at the centre; MP 2-B: 2D piecewise
constant k(x, y)).  Resolution follows the kh ~ 0.625 rule of Section 4.3.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

KH = 0.625  # Section 4.3: ten points per wavelength


@dataclass(frozen=True)
class Layer:
    """A straight line a*x + b*y + c = 0.  A point with a*x + b*y + c >= 0
    lies on the 'upper' side (a point on the line belongs to the upper layer)."""
    a: float
    b: float
    c: float


@dataclass(frozen=True)
class KField:
    """Piecewise-constant wave number.  k(x, y) = values[count] where count is
    the number of lines with a*x + b*y + c >= 0, evaluated as ((a*x) + (b*y)) + c
    with no fused multiply-add.  An empty line list is the constant field
    values[0]."""
    values: tuple
    lines: tuple = ()

    @property
    def constant(self) -> bool:
        return len(self.lines) == 0

    @property
    def k_max(self) -> float:
        return max(self.values)


def constant_k(k: float) -> KField:
    return KField(values=(float(k),), lines=())


def three_layer_field(scale: float = 1.0) -> KField:
    """Stand-in for the MP 2-B step field (whose exact values live only in a
    missing figure): interfaces y = 0.30 + 0.20 x and y = 0.70 - 0.15 x,
    k = 100 / 150 / 250 from bottom to top, all multiplied by ``scale``."""
    # y - 0.20 x - 0.30 >= 0  ->  a=-0.20, b=1, c=-0.30
    l1 = Layer(-0.20, 1.0, -0.30)
    # y + 0.15 x - 0.70 >= 0  ->  a=0.15, b=1, c=-0.70
    l2 = Layer(0.15, 1.0, -0.70)
    return KField(values=(100.0 * scale, 150.0 * scale, 250.0 * scale), lines=(l1, l2))


@dataclass
class Problem:
    """One Helmholtz instance on the unit interval/square: homogeneous
    Dirichlet data everywhere, or (robin, 1D) u(0) = 1 and the Sommerfeld
    condition at x = 1."""
    dim: int
    p: int
    n_el: int
    kfield: KField
    shift: tuple = (1.0, 0.5)         # CSLP (beta1, beta2): M = S - (beta1 - i beta2) k^2 M_mass
    eps: float = 0.0                  # ADP weight epsilon (Section 3, weighted stencil)
    nu_pre: int = 1
    nu_post: int = 1
    omega: float = 0.6                # damped Jacobi (Section 3)
    n_vcycles: int = 1
    sources: list = field(default_factory=list)   # point-source positions
    name: str = ""
    precond: str = "mg"               # "mg": n_vcycles V-cycles (0 = no CSLP); "exact": CSLP inverted exactly
    deflation: bool = True            # ADP deflation on (D...) or off (C_ex alone)
    shift_uses_mass: bool = True      # CSLP shift on the mass matrix (True) or the identity (False)
    robin: bool = False               # 1D: Sommerfeld u' - i k u = 0 at x = 1 (MP 1-A); u(0) = 1 lifted

    @property
    def n_x(self) -> int:
        """Unknowns per direction: the interior functions, plus the last one
        when the end x = 1 carries the Sommerfeld condition."""
        return self.n_el + self.p - 2 + (1 if self.robin else 0)

    @property
    def ndof(self) -> int:
        return self.n_x ** self.dim


def mp1a(k: float, p: int, n_el: int) -> "Problem":
    """MP 1-A (Section 2.1): -u'' - k^2 u = 0 on [0, 1], u(0) = 1, u'(1) - i k u(1)
    = 0; exact solution exp(i k x).  The right-hand side is the lift of u(0)."""
    return Problem(dim=1, p=p, n_el=n_el, kfield=constant_k(k), robin=True, sources=[],
                   name=f"mp1a_k{k:g}_p{p}_nel{n_el}")


def n_el_for_k(k: float, multiple: int = 1) -> int:
    """Elements per direction for kh ~ 0.625, rounded to a multiple."""
    n = k / KH
    return int(multiple * round(n / multiple))


def seeded_normal_rhs(n: int, seed: int) -> np.ndarray:
    """Real N(0,1) load vector (numpy default_rng), passed to both sides."""
    return np.random.default_rng(seed).standard_normal(n)


def seeded_complex_vector(n: int, seed: int) -> np.ndarray:
    """Complex vector with N(0,1) real and imaginary parts."""
    g = np.random.default_rng(seed)
    return g.standard_normal(n) + 1j * g.standard_normal(n)


# ---------------------------------------------------------------- configs
def config1() -> list[Problem]:
    """1D, k = 50, p = 2, 80 elements; point source at 0.5 (plus a seeded
    N(0,1) right-hand side generated with seeded_normal_rhs(n, 0))."""
    return [Problem(dim=1, p=2, n_el=80, kfield=constant_k(50.0), sources=[(0.5,)],
                    name="cfg1_1d_k50_p2")]


def config2(k: float = 200.0, p: int = 3) -> Problem:
    """2D unit square, constant k, kh ~ 0.625, point source at the centre."""
    n_el = {50.0: 80, 100.0: 160, 200.0: 320, 400.0: 640}.get(float(k), n_el_for_k(k, 16))
    return Problem(dim=2, p=p, n_el=n_el, kfield=constant_k(k), sources=[(0.5, 0.5)],
                   name=f"cfg2_2d_k{int(k)}_p{p}_nel{n_el}")


def config3(n_el: int = 640, p: int = 3) -> Problem:
    """2D three-layer field, p = 3, 640 x 640 elements, four seeded sources."""
    src = np.random.default_rng(3).uniform(0.1, 0.9, (4, 2))
    return Problem(dim=2, p=p, n_el=n_el, kfield=three_layer_field(),
                   sources=[tuple(map(float, s)) for s in src], name=f"cfg3_2d_layers_p{p}_nel{n_el}")


def config4(n_instances: int = 64) -> list[tuple[Problem, int]]:
    """Batched instances: k ~ U[50, 400], p in {2,3,4}, N_el = 16*round(k/(0.625*16))
    clamped to [48, 640], 1..8 seeded point sources each."""
    g = np.random.default_rng(4)
    out = []
    for i in range(n_instances):
        k = float(g.uniform(50.0, 400.0))
        p = int(g.integers(2, 5))
        n_el = int(min(640, max(48, 16 * round(k / (KH * 16)))))
        nrhs = int(g.integers(1, 9))
        src = g.uniform(0.1, 0.9, (nrhs, 2))
        prob = Problem(dim=2, p=p, n_el=n_el, kfield=constant_k(k),
                       sources=[tuple(map(float, s)) for s in src], name=f"cfg4_inst{i}")
        out.append((prob, nrhs))
    return out


def config5(layered: bool = False) -> Problem:
    """2D, p = 3, 1280 x 1280 elements (1 640 961 dofs), centre point source:
    constant k = 800 (kh = 0.625), or the three-layer field scaled so that its
    largest value is 800 (k = 320 / 480 / 800)."""
    kf = three_layer_field(800.0 / 250.0) if layered else constant_k(800.0)
    return Problem(dim=2, p=3, n_el=1280, kfield=kf, sources=[(0.5, 0.5)],
                   name=f"cfg5_2d_{'layers' if layered else 'k800'}_p3_nel1280")


def mp1b(k: float, p: int, n_el: int | None = None) -> Problem:
    """MP 1-B (Section 2.1): 1D, Dirichlet at both ends, point source at x = 1/2;
    n_el = k / 0.625 unless given (Section 4.3.1 scales k to 10^6)."""
    n_el = n_el or int(round(k / KH))
    return Problem(dim=1, p=p, n_el=n_el, kfield=constant_k(k), sources=[(0.5,)],
                   name=f"mp1b_k{k:g}_p{p}_nel{n_el}")


def small_2d(n_el: int = 16, p: int = 2, k: float = 10.0, layered: bool = False) -> Problem:
    """Small 2D case for parity tests (spans several tiles and a ragged tail)."""
    kf = three_layer_field(k / 100.0) if layered else constant_k(k)
    return Problem(dim=2, p=p, n_el=n_el, kfield=kf, sources=[(0.5, 0.5)],
                   name=f"small2d_nel{n_el}_p{p}")


def wavelength_ok(k: float, n_el: int) -> bool:
    return k / n_el <= 0.7 + 1e-12
