"""Pins of the oracle's Hermite equilibrium (Sec. 2.1, Eq. demoeq).

P-c: the truncated equilibrium reproduces rho, rho u and the kinetic energy
     2 rho T exactly when the quadrature degree is >= N + 2; N = 2 equals the
     printed second-order form (Eq. demoeq); on a high-degree set every
     moment of order <= N equals the Maxwellian's, and order N + 1 does not.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import quadrature as q

RNG = np.random.default_rng(20090908)


def maxwell_moment_1d(a, u, T):
    """E[X^a] for X ~ Normal(u, T) from the binomial expansion."""
    tot = 0.0
    for j in range(0, a // 2 + 1):
        dfact = 1
        for k in range(2 * j - 1, 0, -2):
            dfact *= k
        tot += math.comb(a, 2 * j) * u ** (a - 2 * j) * T**j * dfact
    return tot


CASES = [(s, N) for s in ["D2Q9", "D2Q16-int"] for N in (2, 3)] + \
        [(s, N) for s in ["D2Q17", "D2Q21", "D2Q25", "D2Q37", "D2Q16-GH", "D2Q36-GH", "D2Q64-GH"] for N in (2, 3, 4)]


@pytest.mark.parametrize("name,N", CASES)
def test_conserved_moments(oracle_mod, name, N):
    P = oracle.Problem(name, N, 4, 1, 0.1)
    xi = P.vs.xi
    for _ in range(5):
        rho = RNG.uniform(0.8, 1.2)
        ux, uy = RNG.uniform(-0.3, 0.3, 2)
        T = RNG.uniform(0.85, 1.15)
        f = P.feq(rho, ux, uy, T)
        assert abs(f.sum() - rho) < 1e-13 * rho
        assert abs(f @ xi[:, 0] - rho * ux) < 2e-13
        assert abs(f @ xi[:, 1] - rho * uy) < 2e-13
        c2 = (xi[:, 0] - ux) ** 2 + (xi[:, 1] - uy) ** 2
        assert abs(f @ c2 - 2 * rho * T) < 1e-13


@pytest.mark.parametrize("name", ["D2Q9", "D2Q17", "D2Q37", "D2Q16-GH", "D2Q36-GH"])
def test_second_order_matches_printed_form(oracle_mod, name):
    P = oracle.Problem(name, 2, 4, 1, 0.1)
    xi, w = P.vs.xi, P.vs.w
    for _ in range(5):
        rho = RNG.uniform(0.8, 1.2)
        u = RNG.uniform(-0.3, 0.3, 2)
        T = RNG.uniform(0.85, 1.15)
        xu = xi @ u
        printed = w * rho * (1 + xu + 0.5 * (xu**2 - u @ u + (T - 1) * (np.sum(xi**2, 1) - 2)))
        np.testing.assert_allclose(P.feq(rho, u[0], u[1], T), printed, rtol=1e-12, atol=1e-16)


@pytest.mark.parametrize("N", [2, 3, 4])
def test_moments_up_to_order_N_are_maxwellian(oracle_mod, N):
    P = oracle.Problem("D2Q64-GH", N, 4, 1, 0.1)  # degree 15 >= N + (N + 1)
    x, y = P.vs.xi[:, 0], P.vs.xi[:, 1]
    rho, ux, uy, T = 1.1, 0.25, -0.2, 1.12
    f = P.feq(rho, ux, uy, T)
    for a in range(N + 2):
        for b in range(N + 2 - a):
            got = f @ (x**a * y**b)
            ref = rho * maxwell_moment_1d(a, ux, T) * maxwell_moment_1d(b, uy, T)
            if a + b <= N:
                assert abs(got - ref) < 1e-12 * max(1, abs(ref)), (a, b)
    # the order-(N+1) moments are not all Maxwellian: the expansion is truncated at N
    diffs = [abs(f @ (x**a * y**(N + 1 - a)) - rho * maxwell_moment_1d(a, ux, T) *
                 maxwell_moment_1d(N + 1 - a, uy, T)) for a in range(N + 2)]
    assert max(diffs) > 1e-4


def test_isothermal_flag_fixes_T(oracle_mod):
    P = oracle.Problem("D2Q36-GH", 3, 4, 1, 0.1, isothermal=True)
    f1 = P.feq(1.0, 0.1, 0.05, 1.3)
    f2 = P.feq(1.0, 0.1, 0.05, 1.0)
    np.testing.assert_array_equal(f1, f2)


def test_rest_state_is_weights(oracle_mod):
    for name in q.names():
        P = oracle.Problem(name, 3, 4, 1, 0.1)
        np.testing.assert_allclose(P.feq(1.0, 0.0, 0.0, 1.0), P.vs.w, rtol=1e-13, atol=1e-17)
