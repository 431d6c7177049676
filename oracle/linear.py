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

The driven wave (body force g = (0, g_y), g_y = A_f sin x cos(phi t)) adds, to
first order in A_f, two terms to one step: the equilibrium is taken at
u = sum xi f~ + g dt/2 (Sec. 2.2), which adds omega w_a xi_ay g dt/2, and the
force term of Sec. 2.1 is w_a xi_ay g, relaxed with the weight omega tau of
Eq. 2order.  Since omega (tau + dt/2) = dt the step gains
b_a = dt w_a xi_ay g before streaming; the measured velocity is
u_y = sum xi_y f~ + g dt/2.  Hydrodynamic limits of the driven response
u_y = Re(U e^{i phi t}) sin x: Navier-Stokes U = A_f / (i phi + nu), nu = tau
(T = 1), and the R13 closed form printed in Sec. 4 (Kn there is tau).
"""
from __future__ import annotations

import numpy as np


def stream_symbol(xi, dx, dt, k=1.0, e=None, streaming="lax_wendroff"):
    """Fourier symbol S_a(k) of one streaming step for the mode exp(i k x): the exact
    shift, Lax-Wendroff, or second-order upwind (Beam-Warming: with c = |C| and
    z = exp(-i s theta), s = sign(C), S = 1 - c/2 (3 - 4 z + z^2) + c^2/2 (1 - z)^2)."""
    xi = np.asarray(xi, dtype=np.float64)
    theta = k * dx
    if e is not None:
        return np.exp(-1j * k * np.asarray(e)[:, 0] * dx)
    C = xi[:, 0] * dt / dx
    if streaming == "upwind2":
        c = np.abs(C)
        z = np.exp(-1j * np.where(C >= 0, 1.0, -1.0) * theta)
        return 1.0 - 0.5 * c * (3.0 - 4.0 * z + z * z) + 0.5 * c * c * (1.0 - z) ** 2
    return 1.0 - 1j * C * np.sin(theta) - C * C * (1.0 - np.cos(theta))


def lb_mode_matrix(xi, w, omega, dx, dt, k=1.0, e=None, isothermal=False, streaming="lax_wendroff"):
    xi = np.asarray(xi, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    Q = w.size
    xx = np.einsum("ai,bi->ab", xi, xi)
    P = np.ones((Q, Q)) + xx
    if not isothermal:
        s2 = 0.5 * np.sum(xi * xi, axis=1) - 1.0
        P += np.outer(s2, s2)
    P = w[:, None] * P
    S = stream_symbol(xi, dx, dt, k, e, streaming)
    return S[:, None] * ((1.0 - omega) * np.eye(Q) + omega * P)


def lb_linear_history(xi, w, omega, dx, dt, u0, nsteps, e=None, isothermal=False, scheme="second_order",
                      streaming="lax_wendroff"):
    """A(n) and S(n), n = 0..nsteps, of the linearised scheme from u_y = u0 sin x.
    scheme "first_order" (Eq. slb) reads sigma_xy without the factor 1 - omega/2."""
    xi = np.asarray(xi, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    M = lb_mode_matrix(xi, w, omega, dx, dt, 1.0, e, isothermal, streaming)
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
        s = (1.0 - 0.5 * omega if scheme == "second_order" else 1.0) * np.sum(kxy * (f - Pm @ f))
        A[n] = -2.0 * c.imag
        S[n] = 2.0 * s.real
        f = M @ f
    return A, S


def lb_decay_rate(xi, w, omega, dx, dt, e=None, isothermal=False, streaming="lax_wendroff"):
    """-ln|lambda|/dt of the least-damped eigenvalue carrying shear (u_y) content."""
    xi = np.asarray(xi, dtype=np.float64)
    M = lb_mode_matrix(xi, w, omega, dx, dt, 1.0, e, isothermal, streaming)
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


def dvm_forced_response(xi1d, w1d, tau, phi, k=1.0):
    """Periodic response H of the continuous reduced DVM (Sec. 3.3, Eq. gb with
    G_a = 0) to g = Re(e^{i phi t}) sin(k x): u -> Re(H e^{i phi t}) sin(k x).
    For the mode, G_k (i phi + i k xi_k + 1/tau) = u / tau + 1, so with
    S1 = sum_k w_k / (i phi + i k xi_k + 1/tau), H = S1 / (1 - S1 / tau)."""
    xi1d = np.asarray(xi1d, dtype=np.float64)
    w1d = np.asarray(w1d, dtype=np.float64)
    s1 = np.sum(w1d / (1j * phi + 1j * k * xi1d + 1.0 / tau))
    return complex(s1 / (1.0 - s1 / tau))


def _projection(xi, w, isothermal):
    Q = w.size
    Pm = np.ones((Q, Q)) + np.einsum("ai,bi->ab", xi, xi)
    if not isothermal:
        s2 = 0.5 * np.sum(xi * xi, axis=1) - 1.0
        Pm += np.outer(s2, s2)
    return w[:, None] * Pm


def lb_linear_forced_history(xi, w, omega, dx, dt, force_amp, phi, nsteps, e=None, isothermal=False,
                             scheme="second_order"):
    """A(n), n = 0..nsteps, of the linearised scheme started at rest and driven by
    g_y = force_amp sin(x_i) cos(phi t).  For the first-order scheme of Eq. slb the
    source is dt w_a xi_ay g as well (omega tau = dt) and u_y = sum xi_y f."""
    xi = np.asarray(xi, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    M = lb_mode_matrix(xi, w, omega, dx, dt, 1.0, e, isothermal)
    theta = dx
    if e is not None:
        S = np.exp(-1j * np.asarray(e)[:, 0] * dx)
    else:
        C = xi[:, 0] * dt / dx
        S = 1.0 - 1j * C * np.sin(theta) - C * C * (1.0 - np.cos(theta))
    f = np.zeros(w.size, dtype=complex)
    A = np.empty(nsteps + 1)
    for n in range(nsteps + 1):
        g = force_amp * np.cos(phi * n * dt) / 2j  # e^{ix} coefficient of g_y
        shift = 0.5 * dt * g if scheme == "second_order" else 0.0
        A[n] = -2.0 * (np.sum(xi[:, 1] * f) + shift).imag
        f = M @ f + S * (dt * w * xi[:, 1] * g)
    return A


def lb_linear_forced_response(xi, w, omega, dx, dt, phi, e=None, isothermal=False):
    """Periodic response H of the linearised scheme: u_y -> Re(H A_f e^{i phi t}) sin x
    for g_y = Re(A_f e^{i phi t}) sin x."""
    xi = np.asarray(xi, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    M = lb_mode_matrix(xi, w, omega, dx, dt, 1.0, e, isothermal)
    if e is not None:
        S = np.exp(-1j * np.asarray(e)[:, 0] * dx)
    else:
        C = xi[:, 0] * dt / dx
        S = 1.0 - 1j * C * np.sin(dx) - C * C * (1.0 - np.cos(dx))
    z = np.exp(1j * phi * dt)
    # unit drive sin(x) e^{i phi t}: its e^{ix} coefficient is e^{i phi t} / (2i)
    X = np.linalg.solve(z * np.eye(w.size) - M, S * (dt * w * xi[:, 1] / 2j))
    u_coef = np.sum(xi[:, 1] * X) + 0.5 * dt / 2j
    return complex(2j * u_coef)


def ns_response(nu, phi):
    """Navier-Stokes response U / A_f = 1 / (i phi + nu) of the driven wave (k = 1)."""
    return 1.0 / (1j * phi + nu)


def r13_response(kn, phi):
    """R13 response U / A_f of the driven standing shear wave, Sec. 4 (kn = tau)."""
    i = 1j
    num = 288 * kn**4 * i - 510 * phi * kn**3 + (520 * i - 225 * phi**2 * i) * kn**2 - 375 * phi * kn + 150 * i
    den = (288 * phi * kn**4 + (510 * phi**2 * i - 270 * i) * kn**3 + (745 * phi - 225 * phi**3) * kn**2
           + (375 * phi**2 * i - 150 * i) * kn + 150 * phi)
    return complex(-num / den)
