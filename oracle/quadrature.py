"""Oracle velocity sets (FP64, numpy).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
module; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it.

Every set is the discrete velocity quadrature of the paper's Eq. (lbgk):
abscissae xi_alpha and weights w_alpha such that sum_alpha w_alpha p(xi_alpha)
equals the integral of p against the unit Gaussian weight omega(xi) of
Sec. 2.1 for every polynomial p up to the set's degree.

* 1-D Gauss-Hermite rules by Golub-Welsch: the symmetric tridiagonal Jacobi
  matrix of the probabilists' Hermite recurrence (zero diagonal, off-diagonal
  sqrt(k)) has the nodes as eigenvalues and the squared first eigenvector
  components as the (unit-mass) weights.  Sec. 2.1 requires a Gauss-Hermite
  rule of degree >= 2N; Sec. 3.3 uses the same rule for the DVM.
* 2-D product sets D2Q(n^2)-GH: tensor products of the 1-D rule (off-lattice).
* Table 1 on-lattice sets (D2Q9, D2Q16 with m=1,n=4, D2Q17, D2Q21, D2Q25
  with m=3,n=7), evaluated from the surds printed in Table 1.
* D2Q37: not in the paper.  Built here by moment matching over fully
  symmetric integer shells (the search idea of Sec. 2.3): for a choice of 8
  shells, the 9 even, symmetry-distinct moment equations of total degree <= 8
  are linear in the 8 shell weights and polynomial in t = 1/c^2; the left null
  vector of the shell-moment matrix gives a quartic in t whose admissible root
  fixes the lattice scale c.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class VelocitySet:
    """A 2-D discrete velocity set.

    xi: (Q, 2) abscissae in units of sqrt(R T0); w: (Q,) weights, sum 1.
    e:  (Q, 2) integer lattice vectors for on-lattice sets (xi = c * e), else None.
    c:  lattice scale for on-lattice sets, else None.
    nodes1d: the 1-D rule for product sets (nodes, weights), else None.
    """

    name: str
    xi: np.ndarray
    w: np.ndarray
    e: np.ndarray | None = None
    c: float | None = None
    nodes1d: tuple | None = None
    meta: dict = field(default_factory=dict)

    @property
    def Q(self) -> int:
        return int(self.w.shape[0])

    @property
    def on_lattice(self) -> bool:
        return self.e is not None


def gauss_hermite(n: int) -> tuple[np.ndarray, np.ndarray]:
    """n-point Gauss-Hermite rule for the unit Gaussian (Golub-Welsch).

    Returns ascending nodes and weights with sum(weights) == 1.
    """
    if n < 1:
        raise ValueError("n >= 1")
    k = np.arange(1, n, dtype=np.float64)
    J = np.diag(np.sqrt(k), 1) + np.diag(np.sqrt(k), -1)
    lam, V = np.linalg.eigh(J)
    w = V[0, :] ** 2
    # symmetrise: the exact rule is symmetric about 0
    lam = 0.5 * (lam - lam[::-1])
    w = 0.5 * (w + w[::-1])
    return lam, w / w.sum()


def product_set(n: int) -> VelocitySet:
    """D2Q(n^2) tensor-product Gauss-Hermite set, alpha = i*n + j -> (g_i, g_j)."""
    g, wg = gauss_hermite(n)
    xi = np.array([[g[i], g[j]] for i in range(n) for j in range(n)])
    w = np.array([wg[i] * wg[j] for i in range(n) for j in range(n)])
    return VelocitySet(f"D2Q{n*n}-GH", xi, w, nodes1d=(g, wg))


def _fs(a: int, b: int) -> list[tuple[int, int]]:
    """Fully symmetric orbit of (a, b) under the square's symmetry group."""
    pts = set()
    for sx in (1, -1):
        for sy in (1, -1):
            pts.add((sx * a, sy * b))
            pts.add((sx * b, sy * a))
    return sorted(pts)


def _onlattice(name, shells, weights, c) -> VelocitySet:
    e, w = [], []
    for (a, b), wt in zip(shells, weights):
        for p in _fs(a, b):
            e.append(p)
            w.append(wt)
    e = np.array(e, dtype=np.int64)
    return VelocitySet(name, c * e.astype(np.float64), np.array(w), e=e, c=float(c))


def _product_onlattice(name, ints, w1, T0) -> VelocitySet:
    """2-D product of a 1-D integer rule (values ints, weights w1), xi = e/sqrt(T0)."""
    e, w = [], []
    for i, wi in zip(ints, w1):
        for j, wj in zip(ints, w1):
            e.append((i, j))
            w.append(wi * wj)
    e = np.array(e, dtype=np.int64)
    c = 1.0 / math.sqrt(T0)
    return VelocitySet(name, c * e.astype(np.float64), np.array(w), e=e, c=c)


def d2q9() -> VelocitySet:
    """Table 1, D2Q9: xi in {0, sqrt(3) e}, weights 4/9, 1/9, 1/36."""
    return _onlattice("D2Q9", [(0, 0), (1, 0), (1, 1)], [4 / 9, 1 / 9, 1 / 36], math.sqrt(3.0))


def d2q16_int(m: int = 1, n: int = 4) -> VelocitySet:
    """Table 1, D2Q16 (m=1, n=4): product of the 1-D rule at +-m, +-n.

    W_m, W_n and the lattice temperature T0 are the printed surds.
    """
    s = math.sqrt(m**4 - 10 * n * n * m * m + n**4)
    Wm = (m * m - 5 * n * n + s) / (12 * (m * m - n * n))
    Wn = (5 * m * m - n * n - s) / (12 * (m * m - n * n))
    T0 = (m * m + n * n + s) / 6
    vs = _product_onlattice("D2Q16-int", [-n, -m, m, n], [Wn, Wm, Wm, Wn], T0)
    vs.meta["T0"] = T0
    return vs


def d2q17() -> VelocitySet:
    """Table 1, D2Q17: shells (0,0),(1,0)FS,(1,1),(2,2),(3,0)FS scaled by r."""
    s = math.sqrt(193.0)
    r = math.sqrt((125 + 5 * s) / 72)
    wts = [(575 + 193 * s) / 8100, (3355 - 91 * s) / 18000, (655 + 17 * s) / 27000,
           (685 - 49 * s) / 54000, (1445 - 101 * s) / 162000]
    return _onlattice("D2Q17", [(0, 0), (1, 0), (1, 1), (2, 2), (3, 0)], wts, r)


def d2q21() -> VelocitySet:
    """Table 1, D2Q21: shells (0,0),(1,0)FS,(1,1),(2,0)FS,(2,2),(3,0)FS, r^2 = 3/2."""
    wts = [91 / 324, 1 / 12, 2 / 27, 7 / 360, 1 / 432, 1 / 1620]
    return _onlattice("D2Q21", [(0, 0), (1, 0), (1, 1), (2, 0), (2, 2), (3, 0)], wts, math.sqrt(1.5))


def d2q25(m: int = 3, n: int = 7) -> VelocitySet:
    """Table 1, D2Q25 (m=3, n=7): product of the 1-D rule at 0, +-m, +-n."""
    D5 = math.sqrt(9 * m**4 - 42 * n * n * m * m + 9 * n**4)
    W0 = (-3 * m**4 - 3 * n**4 + 54 * m * m * n * n - (m * m + n * n) * D5) / (75 * m * m * n * n)
    Wm = (9 * m**4 - 6 * n**4 - 27 * n * n * m * m + (3 * m * m - 2 * n * n) * D5) / (300 * m * m * (m * m - n * n))
    Wn = (9 * n**4 - 6 * m**4 - 27 * n * n * m * m + (3 * n * n - 2 * m * m) * D5) / (300 * n * n * (n * n - m * m))
    T0 = (3 * m * m + 3 * n * n + D5) / 30
    vs = _product_onlattice("D2Q25", [-n, -m, 0, m, n], [Wn, Wm, W0, Wm, Wn], T0)
    vs.meta["T0"] = T0
    return vs


# --- D2Q37 by moment matching -------------------------------------------------

_EVEN_MOMENTS = [(0, 0), (2, 0), (4, 0), (2, 2), (6, 0), (4, 2), (8, 0), (6, 2), (4, 4)]
_SHELLS_LE3 = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2), (3, 0), (3, 1), (3, 2), (3, 3)]


def _dfact(k: int) -> int:
    return 1 if k <= 0 else k * _dfact(k - 2)


def _solve_shells(shells):
    """Weights and scale for 8 shells matching the 9 moment equations, or None."""
    Mm = np.array([[sum(float(ex) ** a * float(ey) ** b for ex, ey in _fs(*s)) for s in shells]
                   for (a, b) in _EVEN_MOMENTS])
    g = np.array([_dfact(a - 1) * _dfact(b - 1) for (a, b) in _EVEN_MOMENTS], dtype=np.float64)
    d = np.array([(a + b) // 2 for (a, b) in _EVEN_MOMENTS])
    U, S, Vt = np.linalg.svd(Mm)
    if S[-1] < 1e-9 * S[0]:
        return None  # shell moments degenerate
    nvec = U[:, -1]  # left null vector of the 9 x 8 matrix
    # n . (g * t^d) = 0 : polynomial in t of degree max(d)
    coef = np.zeros(d.max() + 1)
    for k in range(len(g)):
        coef[d[k]] += nvec[k] * g[k]
    roots = np.roots(coef[::-1])
    best = None
    for t in roots:
        if abs(t.imag) > 1e-9 * max(1.0, abs(t)) or t.real <= 0:
            continue
        t = t.real
        rhs = g * t ** d
        W, *_ = np.linalg.lstsq(Mm, rhs, rcond=None)
        if np.all(W > 0):
            # Newton polish of the square system  M W - g t^d = 0  in (W, t)
            for _ in range(4):
                F = Mm @ W - g * t ** d
                J = np.hstack([Mm, (-g * d * t ** np.maximum(d - 1, 0))[:, None]])
                step = np.linalg.solve(J, -F)
                W, t = W + step[:-1], t + step[-1]
            c = 1.0 / math.sqrt(t)
            if best is None or c < best[1]:
                best = (W, c)
    return best


def d2q37() -> VelocitySet:
    """On-lattice degree-9 set with 37 velocities, |e_x|,|e_y| <= 3.

    Searches 8-shell subsets of the integer shells with components <= 3 whose
    sizes add to 37, in lexicographic order of the shell list; takes the first
    with all weights positive (smallest admissible scale for that subset) and
    confirms degree 9 by direct moment evaluation.
    """
    for combo in itertools.combinations(_SHELLS_LE3, 8):
        if sum(len(_fs(*s)) for s in combo) != 37:
            continue
        sol = _solve_shells(list(combo))
        if sol is None:
            continue
        W, c = sol
        vs = _onlattice("D2Q37", list(combo), list(W), c)
        if exact_degree(vs) >= 9:
            vs.meta["shells"] = list(combo)
            return vs
    raise RuntimeError("no admissible D2Q37 shell set")


# --- registry and checks -------------------------------------------------------

_REGISTRY = {
    "D2Q16-GH": lambda: product_set(4),
    "D2Q36-GH": lambda: product_set(6),
    "D2Q64-GH": lambda: product_set(8),
    "D2Q9": d2q9,
    "D2Q16-int": d2q16_int,
    "D2Q17": d2q17,
    "D2Q21": d2q21,
    "D2Q25": d2q25,
    "D2Q37": d2q37,
}

_CACHE: dict[str, VelocitySet] = {}


def velocity_set(name: str) -> VelocitySet:
    if name not in _REGISTRY:
        raise KeyError(f"unknown velocity set {name!r}; known: {sorted(_REGISTRY)}")
    if name not in _CACHE:
        _CACHE[name] = _REGISTRY[name]()
    return _CACHE[name]


def names() -> list[str]:
    return list(_REGISTRY)


def gaussian_moment(a: int, b: int) -> float:
    """E[X^a Y^b] for independent unit Gaussians X, Y."""
    if a % 2 or b % 2:
        return 0.0
    return float(_dfact(a - 1) * _dfact(b - 1))


def exact_degree(vs: VelocitySet, max_deg: int = 20, tol: float = 1e-11) -> int:
    """Largest D such that all moments of total degree <= D are exact."""
    x, y = vs.xi[:, 0], vs.xi[:, 1]
    for D in range(0, max_deg + 1):
        for a in range(D + 1):
            b = D - a
            got = float(np.sum(vs.w * x**a * y**b))
            ref = gaussian_moment(a, b)
            if abs(got - ref) > tol * max(1.0, abs(ref)):
                return D - 1
    return max_deg
