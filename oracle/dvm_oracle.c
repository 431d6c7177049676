/*
 * Oracle: discrete velocity method for the linearised BGK equation of the
 * standing shear wave, in the reduced form of Sec. 3.3 (Eqs. LBGK, ga, gb).
 *
 * TEST INFRASTRUCTURE ONLY (loaded by tests/ and bench.py's CPU leg only).
 *
 * The wave here varies along x and the flow is along y, so the reduced
 * unknown is G(x, xi_k, t) = (1/sqrt(2 pi)) int xi_y psi exp(-xi_y^2/2) dxi_y
 * at the nodes xi_k of a 1-D Gauss-Hermite rule in xi_x:
 *     dG/dt + xi_k dG/dx = (u - G) / tau,     u(x) = sum_k w_k G(x, xi_k)
 * (the velocity moment over the unit Gaussian, which is how the paper's
 * u = (1/sqrt(2 pi)) int G dxi reads once the Gaussian factor of the moment is
 * restored).  The other reduced function G_a of Eq. ga obeys a homogeneous
 * equation, starts at zero and stays zero, so the force term g (G_a + 1) of
 * Eq. gb is the body force g(x, t) = A_f sin(x_i) cos(phi t) itself:
 *     dG/dt + xi_k dG/dx = (u - G) / tau + g.
 * Space-time discretisation, independent of the lattice: Strang splitting of
 * the relaxation and force (integrated exactly: u gains int g dt, since
 * sum w_k = 1, and G - u decays by exp(-h / tau)) around one Lax-Wendroff
 * advection step, dt = cfl * dx / max|xi_k|.
 * Observables: A = 2/nx sum u sin(x_i), S = 2/nx sum sigma cos(x_i),
 * sigma = sum_k w_k xi_k G (the xy pressure-tensor moment).
 */
#include <math.h>
#include <stdlib.h>

/* Test builds only (tests/test_oracle_planted.py): ORACLE_PLANT = 8 drives with -g. */
#ifndef ORACLE_PLANT
#define ORACLE_PLANT 0
#endif

/* int_{t0}^{t0 + h} cos(phi t) dt */
static double cos_integral(double phi, double t0, double h)
{
    if (phi == 0.0) return h;
    return (sin(phi * (t0 + h)) - sin(phi * t0)) / phi;
}

/* relaxation and force over [t0, t0 + h], exactly: u += A_f sin(x) int cos,
 * G = u + (G - u) exp(-h / tau) */
static void relax_force(double *G, double *u, int nx, int nv, double dx, double decay, double force_amp,
                        double force_freq, double t0, double h)
{
    double c = (ORACLE_PLANT == 8 ? -force_amp : force_amp) * cos_integral(force_freq, t0, h);
    for (int i = 0; i < nx; ++i) {
        double un = u[i] + c * sin(i * dx);
        for (int k = 0; k < nv; ++k) {
            double *g = &G[(size_t)k * nx + i];
            *g = un + (*g - u[i]) * decay;
        }
        u[i] = un;
    }
}

int oracle_dvm_run_forced(int nx, int nv, const double *xi, const double *w, double tau, double cfl,
                          double u0, double force_amp, double force_freq, int nsteps, double *t_out,
                          double *A_out, double *S_out)
{
    if (nx < 3 || nv < 1 || nsteps < 0 || cfl <= 0.0 || cfl > 1.0) return -1;
    const double pi = 3.14159265358979323846;
    double dx = 2.0 * pi / nx, vmax = 0.0;
    for (int k = 0; k < nv; ++k) vmax = fabs(xi[k]) > vmax ? fabs(xi[k]) : vmax;
    double dt = cfl * dx / vmax;
    double *G = malloc(sizeof(double) * (size_t)nx * nv);
    double *Gn = malloc(sizeof(double) * (size_t)nx);
    double *u = malloc(sizeof(double) * (size_t)nx);
    if (!G || !Gn || !u) {
        free(G);
        free(Gn);
        free(u);
        return -1;
    }
    /* equilibrium start: psi = xi_y u_y, so G = u_y at every node */
    for (int k = 0; k < nv; ++k)
        for (int i = 0; i < nx; ++i) G[(size_t)k * nx + i] = u0 * sin(i * dx);
    double decay_half = exp(-0.5 * dt / tau);
    for (int s = 0; s <= nsteps; ++s) {
        double A = 0, S = 0;
        for (int i = 0; i < nx; ++i) {
            double ui = 0, si = 0;
            for (int k = 0; k < nv; ++k) {
                ui += w[k] * G[(size_t)k * nx + i];
                si += w[k] * xi[k] * G[(size_t)k * nx + i];
            }
            u[i] = ui;
            A += ui * sin(i * dx);
            S += si * cos(i * dx);
        }
        if (t_out) t_out[s] = s * dt;
        if (A_out) A_out[s] = 2.0 * A / nx;
        if (S_out) S_out[s] = 2.0 * S / nx;
        if (s == nsteps) break;
        /* half relaxation (with the force), advection, half relaxation (with the force) */
        relax_force(G, u, nx, nv, dx, decay_half, force_amp, force_freq, s * dt, 0.5 * dt);
        for (int k = 0; k < nv; ++k) {
            double C = xi[k] * dt / dx;
            double *g = &G[(size_t)k * nx];
            for (int i = 0; i < nx; ++i) {
                double fm = g[(i - 1 + nx) % nx], f0 = g[i], fp = g[(i + 1) % nx];
                Gn[i] = f0 - 0.5 * C * (fp - fm) + 0.5 * C * C * (fp - 2.0 * f0 + fm);
            }
            for (int i = 0; i < nx; ++i) g[i] = Gn[i];
        }
        for (int i = 0; i < nx; ++i) {
            double ui = 0;
            for (int k = 0; k < nv; ++k) ui += w[k] * G[(size_t)k * nx + i];
            u[i] = ui;
        }
        relax_force(G, u, nx, nv, dx, decay_half, force_amp, force_freq, (s + 0.5) * dt, 0.5 * dt);
    }
    free(G);
    free(Gn);
    free(u);
    return 0;
}

int oracle_dvm_run(int nx, int nv, const double *xi, const double *w, double tau, double cfl,
                   double u0, int nsteps, double *t_out, double *A_out, double *S_out)
{
    return oracle_dvm_run_forced(nx, nv, xi, w, tau, cfl, u0, 0.0, 0.0, nsteps, t_out, A_out, S_out);
}

/* time step used by oracle_dvm_run for the same arguments */
double oracle_dvm_dt(int nx, int nv, const double *xi, double cfl)
{
    const double pi = 3.14159265358979323846;
    double vmax = 0.0;
    for (int k = 0; k < nv; ++k) vmax = fabs(xi[k]) > vmax ? fabs(xi[k]) : vmax;
    return cfl * (2.0 * pi / nx) / vmax;
}
