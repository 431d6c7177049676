"""Linear-mode analysis used to pin the oracle (numpy, complex128).

TEST INFRASTRUCTURE ONLY.

Two independent descriptions of the small-amplitude shear wave u_y ~ sin(k x):

* ``lb_mode_matrix``: one step of the scheme of Eq. 2order, linearised about
  rest (rho = 1, u = 0, T = 1) and written for one Fourier mode k.  The
  equilibrium linearises to f^eq_a = w_a [1 + drho + xi_a.du + (T - 1)(|xi_a|^2 - 2)/2]
  (the expansion of Sec. 2.1 keeps only these first-order terms), with
  drho = sum df, du = sum xi df and dT = sum |xi|^2 df / 2 - drho, so
  P_ab = w_a [1 + xi_a.xi_b + (|xi_a|^2/2 - 1)(|xi_b|^2/2 - 1)].
  One step is M(k) = diag(S_a(k)) [(1 - omega) I + omega P], S_a the Fourier
  symbol of the streaming: exp(-i k e_ax dx) for the exact shift and
  1 - i C sin(theta) - C^2 (1 - cos(theta)), C = xi_ax dt/dx, theta = k dx, for
  Lax-Wendroff.
* ``dvm_dispersion_roots``: the continuous reduced linearised BGK equation of
  Sec. 3.3, dG/dt + xi dG/dx = (u - G)/tau with u = sum_k w_k G_k, for the
  mode exp(i k x + s t): 1 = sum_k w_k / (1 + tau s + i tau k xi_k).
"""
from __future__ import annotations

import numpy as np


def lb_mode_matrix(xi, w, omega, dx, dt, k=1.0, e=None, isothermal=False):
    xi = np.asarray(xi, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    Q = w.size
    xx = np.einsum("ai,bi->ab", xi, xi)
    P = np.ones((Q, Q)) + xx
    if not isothermal:
        s2 = 0.5 * np.sum(xi * xi, axis=1) - 1.0
        P += np.outer(s2, s2)
    P = w[:, None] * P
    theta = k * dx
    if e is not None:
        S = np.exp(-1j * k * np.asarray(e)[:, 0] * dx)
    else:
        C = xi[:, 0] * dt / dx
        S = 1.0 - 1j * C * np.sin(theta) - C * C * (1.0 - np.cos(theta))
    return S[:, None] * ((1.0 - omega) * np.eye(Q) + omega * P)


def lb_linear_history(xi, w, omega, dx, dt, u0, nsteps, e=None, isothermal=False):
    """A(n) and S(n), n = 0..nsteps, of the linearised scheme from u_y = u0 sin x."""
    xi = np.asarray(xi, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    M = lb_mode_matrix(xi, w, omega, dx, dt, 1.0, e, isothermal)
    # e^{ix} coefficient of the initial equilibrium deviation w_a xi_ay u0 sin x
    f = w * xi[:, 1] * (u0 / 2j)
    Q = w.size
    xx = np.einsum("ai,bi->ab", xi, xi)
    Pm = np.ones((Q, Q)) + xx
    if not isothermal:
        s2 = 0.5 * np.sum(xi * xi, axis=1) - 1.0
        Pm += np.outer(s2, s2)
    Pm = w[:, None] * Pm
    kxy = xi[:, 0] * xi[:, 1]
    A = np.empty(nsteps + 1)
    S = np.empty(nsteps + 1)
    for n in range(nsteps + 1):
        c = np.sum(xi[:, 1] * f)
        s = (1.0 - 0.5 * omega) * np.sum(kxy * (f - Pm @ f))
        A[n] = -2.0 * c.imag
        S[n] = 2.0 * s.real
        f = M @ f
    return A, S


def lb_decay_rate(xi, w, omega, dx, dt, e=None, isothermal=False):
    """-ln|lambda|/dt of the least-damped eigenvalue carrying shear (u_y) content."""
    xi = np.asarray(xi, dtype=np.float64)
    M = lb_mode_matrix(xi, w, omega, dx, dt, 1.0, e, isothermal)
    lam, V = np.linalg.eig(M)
    shear = np.abs(xi[:, 1] @ V)
    ok = shear > 1e-8 * shear.max()
    i = np.argmax(np.where(ok, np.abs(lam), -1.0))
    return -np.log(np.abs(lam[i])) / dt


def dvm_dispersion_roots(xi1d, w1d, tau, k=1.0):
    """All roots s of 1 = sum_k w_k / (1 + tau s + i tau k xi_k)."""
    xi1d = np.asarray(xi1d, dtype=np.float64)
    w1d = np.asarray(w1d, dtype=np.float64)
    # polynomial in sigma = 1 + tau s : prod_k (sigma + i tau k xi_k) - sum_k w_k prod_{j!=k}(...)
    lin = [np.array([1.0, 1j * tau * k * x]) for x in xi1d]  # highest power first
    full = np.array([1.0 + 0j])
    for p in lin:
        full = np.convolve(full, p)
    rest = np.zeros(len(xi1d), dtype=complex)
    for kk in range(len(xi1d)):
        pk = np.array([1.0 + 0j])
        for j, p in enumerate(lin):
            if j != kk:
                pk = np.convolve(pk, p)
        rest += w1d[kk] * pk
    poly = full.copy()
    poly[1:] -= rest
    sig = np.roots(poly)
    return (sig - 1.0) / tau


def dvm_decay_rate(xi1d, w1d, tau, k=1.0):
    """Decay rate (-Re s) of the least-damped root of the dispersion relation."""
    s = dvm_dispersion_roots(xi1d, w1d, tau, k)
    return float(-np.max(s.real))
