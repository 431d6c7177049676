"""Pins of the oracle's velocity sets (Sec. 2.1 degree rule, Table 1).

P-a: the Golub-Welsch rule equals numpy's Hermite_e Gauss rule and integrates
     x^k exactly for k <= 2n - 1 (and not for k = 2n).
P-b: Table 1 weights sum to one and reach the printed-surd degrees.
D2Q37: a degree-9 integer set with positive weights.
"""
import math
import os

import numpy as np
import pytest
from numpy.polynomial import hermite_e

from oracle import quadrature as q

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1.txt")


def dfact(k):
    return 1 if k <= 0 else k * dfact(k - 2)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 8, 12, 20])
def test_gh_matches_numpy_hermegauss(n):
    x, w = q.gauss_hermite(n)
    xr, wr = hermite_e.hermegauss(n)
    np.testing.assert_allclose(x, xr, rtol=0, atol=1e-13)
    np.testing.assert_allclose(w, wr / math.sqrt(2 * math.pi), rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("n", [3, 4, 5, 6, 8])
def test_gh_exactness_degree(n):
    x, w = q.gauss_hermite(n)
    for k in range(2 * n):
        ref = 0.0 if k % 2 else float(dfact(k - 1))
        assert abs(np.sum(w * x**k) - ref) <= 1e-12 * max(1.0, ref), k
    # degree 2n is NOT exact for an n-point rule
    k = 2 * n
    assert abs(np.sum(w * x**k) - dfact(k - 1)) > 1e-6 * dfact(k - 1)


def test_gh_known_values():
    # GH-4 nodes are the roots of He_4 = x^4 - 6 x^2 + 3: x^2 = 3 +- sqrt(6)
    x, _ = q.gauss_hermite(4)
    np.testing.assert_allclose(np.sort(np.abs(x))[::2], [math.sqrt(3 - math.sqrt(6)), math.sqrt(3 + math.sqrt(6))],
                               atol=1e-14)
    # GH-8 smallest weight, squared for the 2-D product corner
    _, w = q.gauss_hermite(8)
    assert abs(w.min() ** 2 - 1.2682e-8) < 1e-11


@pytest.mark.parametrize("name,n", [("D2Q16-GH", 4), ("D2Q36-GH", 6), ("D2Q64-GH", 8)])
def test_product_sets(name, n):
    vs = q.velocity_set(name)
    assert vs.Q == n * n
    assert abs(vs.w.sum() - 1) < 1e-14
    assert q.exact_degree(vs) == 2 * n - 1


def _golden_rows():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, Q, shells, caption, deg = line.split()
            rows.append((name, int(Q), int(shells), int(caption), int(deg)))
    return rows


@pytest.mark.parametrize("row", _golden_rows(), ids=lambda r: r[0])
def test_table1_sets(row):
    name, Q, _shells, _caption, deg = row
    vs = q.velocity_set(name)
    assert vs.Q == Q
    assert abs(vs.w.sum() - 1.0) < 1e-13
    assert np.all(vs.w > 0)
    assert q.exact_degree(vs) == deg
    # integer lattice: xi = c e exactly
    np.testing.assert_allclose(vs.xi, vs.c * vs.e, atol=1e-15)


def test_table1_d2q9_weights_printed():
    vs = q.velocity_set("D2Q9")
    by_norm = {}
    for e, w in zip(vs.e, vs.w):
        by_norm.setdefault(int(e @ e), set()).add(round(w, 15))
    assert by_norm == {0: {round(4 / 9, 15)}, 1: {round(1 / 9, 15)}, 2: {round(1 / 36, 15)}}
    assert abs(vs.c - math.sqrt(3)) < 1e-15


def test_d2q37():
    vs = q.velocity_set("D2Q37")
    assert vs.Q == 37
    assert np.abs(vs.e).max() == 3
    assert np.all(vs.w > 0)
    assert q.exact_degree(vs) >= 9
    # the set is closed under the square's symmetries
    pts = {tuple(p) for p in vs.e}
    assert pts == {(-b, a) for a, b in pts}
    assert pts == {(b, a) for a, b in pts}
