/*
 * Oracle: plain FP64 lattice Boltzmann stepper for the standing shear wave.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liboracle.so, which
 * only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg load.
 * It shares no code, header or table with the CUDA library.
 *
 * What it computes, step by step, in the paper's order (Sec. 2.1-2.2):
 *   state       f~_alpha(r, t)                      (the variable of Eq. 2order)
 *   force       g = (0, g_y), g_y(x_i, t) = A_f sin(x_i) cos(phi t) (the standing-wave
 *               drive of Sec. 4, Eq. force, turned so that the flow is along y and
 *               varies along x), or a uniform g_y = A_f cos(phi t); A_f = 0: unforced
 *   moments     rho = sum f~,  rho u = sum xi f~ + rho g dt / 2   (Sec. 2.2)
 *               D rho T = sum |xi - u|^2 f, D = 2, of the distribution f behind
 *               f~ (kinetic temperature; with a force T = T(f~) + dt^2 g^2 / 8)
 *   equilibrium f^eq_alpha = w_alpha sum_{n<=N} (1/n!) a_eq^(n) : chi^(n)(xi_alpha)
 *               with a_eq^(n) = int f^eq chi^(n) dxi   (Eqs. approxf, an, Sec. 2.1),
 *               the tensor contraction taken over every index tuple in {x,y}^n
 *               and each a_eq component integrated against the Maxwellian by an
 *               inner Gauss-Hermite rule (exact for these polynomial degrees).
 *   force term  g_alpha = w_alpha sum_{n=1..N} 1/(n-1)! g a_eq^(n-1) : chi^(n)(xi_alpha)
 *               (Sec. 2.1), the contraction over every index tuple whose first
 *               index carries g; it is the source -g . grad_xi f^eq of Eq. bgk moved
 *               to the right-hand side (its N = 2 form is printed in Sec. 2.1)
 *   collide     f* = f~ - omega (f~ - f^eq) + omega tau g_alpha,
 *               omega = dt / (tau + dt/2)                                  (Eq. 2order)
 *   stream      on-lattice: f~_alpha(r + xi_alpha dt) = f*_alpha(r), an exact
 *               periodic shift by e_alpha (Sec. 2.3); off-lattice: Lax-Wendroff
 *               along x then along y (the scheme named in Sec. 3.3 and the
 *               caption of the D2Q400 figure), periodic; or (streaming = 1) the
 *               second-order upwind (Beam-Warming) scheme along x then y, which
 *               uses the two upstream neighbours:
 *               out_i = f_i - C/2 (3 f_i - 4 f_{i-s} + f_{i-2s})
 *                             + C^2/2 (f_i - 2 f_{i-s} + f_{i-2s}),  s = sign(C),
 *               with |C| in place of C.
 * First-order scheme (scheme = 1, the standard LB of Eq. slb, Sec. 2.2): the state is
 * f itself and one step is f(r + xi dt, t + dt) = f - (dt/tau)(f - f^eq) + dt g_alpha,
 * i.e. the collide line above with omega = dt / tau (so omega tau = dt), moments
 * rho u = sum xi f with no dt/2 term, T of f with no correction, and
 * sigma_xy = sum xi_x xi_y (f - f^eq); streaming as above.
 * Hermite order N = 1 (Sec. 3.3, Eq. lbm1) is the n <= 1 part of the same sums.
 * Observables at each time level n are taken from f~(n), before collision:
 *   mass = sum rho, mom = sum rho u, A = 2/(nx ny) sum u_y sin(x_i),
 *   S = 2/(nx ny) sum sigma_xy cos(x_i),
 *   sigma_xy = (1 - omega/2) sum xi_x xi_y (f~ - f^eq + dt/2 g_alpha)  (f - f^eq of f~),
 *   H = sum (f~ - w rho0)^2 / w, x_i = i * dx.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Test builds only: ORACLE_PLANT = k compiles mistake k into the stepper, so that the
 * tests can check that the pins catch it (tests/test_oracle_planted.py).  0: none. */
#ifndef ORACLE_PLANT
#define ORACLE_PLANT 0
#endif
#define PLANTED(k) (ORACLE_PLANT == (k))
/* planted 7: the first-order scheme relaxes with the second-order omega */
/* planted 9: second-order upwind streaming from the downstream side */

#define ORACLE_MAXQ 128
#define ORACLE_MAXN 4
#define ORACLE_MAXINNER 32

typedef struct {
    int nx, ny;          /* periodic grid */
    int Q;               /* number of discrete velocities */
    int N;               /* Hermite order of the equilibrium */
    const double *xi;    /* Q x 2 abscissae */
    const double *w;     /* Q weights */
    const int *e;        /* Q x 2 integer lattice vectors (on-lattice), or NULL (Lax-Wendroff) */
    double dx, dt, tau;  /* cell size, time step, collision time in Eq. bgk units */
    double rho0;         /* reference density of the H norm */
    int isothermal;      /* 1: T = 1 in the equilibrium */
    int ninner;          /* inner Gauss-Hermite rule for a_eq integrals */
    const double *zin, *win;
    double force_amp;    /* A_f of g_y = A_f s(x_i) cos(phi t); 0: unforced */
    double force_freq;   /* phi */
    int force_uniform;   /* 1: s(x) = 1, 0: s(x) = sin(x_i) */
    int scheme;          /* 0: Eq. 2order, 1: Eq. slb (first order) */
    int streaming;       /* off-lattice: 0 Lax-Wendroff, 1 second-order upwind */
} oracle_lb_params;

/* relaxation rate of the scheme */
static double scheme_omega(const oracle_lb_params *p)
{
    if (p->scheme == 1) return PLANTED(7) ? p->dt / (p->tau + 0.5 * p->dt) : p->dt / p->tau;
    return p->dt / (p->tau + 0.5 * p->dt);
}

/* probabilists' Hermite polynomial He_k(x) by its three-term recurrence */
static double hermite_he(int k, double x)
{
    double h0 = 1.0, h1 = x;
    if (k == 0) return h0;
    for (int j = 1; j < k; ++j) {
        double h2 = x * h1 - j * h0;
        h0 = h1;
        h1 = h2;
    }
    return h1;
}

static double factorial(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

/* a_eq component for an index tuple with kx x-indices and ky y-indices:
 * int f^eq He_kx(xi_x) He_ky(xi_y) dxi, f^eq the Maxwellian (rho, u, T). */
static double a_eq_component(const oracle_lb_params *p, double rho, double ux, double uy,
                             double T, int kx, int ky)
{
    double s = sqrt(T), acc = 0.0;
    for (int i = 0; i < p->ninner; ++i) {
        double hx = hermite_he(kx, ux + s * p->zin[i]);
        for (int j = 0; j < p->ninner; ++j)
            acc += p->win[i] * p->win[j] * hx * hermite_he(ky, uy + s * p->zin[j]);
    }
    return rho * acc;
}

void oracle_feq(const oracle_lb_params *p, double rho, double ux, double uy, double T, double *feq)
{
    double Teq = p->isothermal ? 1.0 : T;
    for (int a = 0; a < p->Q; ++a) feq[a] = 0.0;
    for (int n = 0; n <= p->N; ++n) {
        double inv_nfact = 1.0 / factorial(n);
        if (PLANTED(5) && n == p->N) break; /* planted: highest Hermite order dropped */
        for (int t = 0; t < (1 << n); ++t) { /* index tuple: bit b set -> index b is y */
            int ky = __builtin_popcount((unsigned)t), kx = n - ky;
            double an = a_eq_component(p, rho, ux, uy, Teq, kx, ky);
            for (int a = 0; a < p->Q; ++a) {
                double chi = hermite_he(kx, p->xi[2 * a]) * hermite_he(ky, p->xi[2 * a + 1]);
                feq[a] += inv_nfact * an * chi;
            }
        }
    }
    for (int a = 0; a < p->Q; ++a) feq[a] *= p->w[a];
}

/* Hermite force term g_alpha for g = (0, gy) at the Maxwellian (rho, u, T):
 * F_alpha = w_alpha sum_{n=1..N} 1/(n-1)! sum over index tuples (i1..in) with
 * i1 = y of gy a_eq^(n-1)_(i2..in) chi^(n)_(i1..in)(xi_alpha). */
void oracle_force(const oracle_lb_params *p, double rho, double ux, double uy, double T, double gy,
                  double *F)
{
    double Teq = p->isothermal ? 1.0 : T;
    for (int a = 0; a < p->Q; ++a) F[a] = 0.0;
    for (int n = 1; n <= p->N; ++n) {
        double inv = 1.0 / factorial(n - 1);
        for (int t = 0; t < (1 << n); ++t) { /* bit b set -> index b is y; bit 0 is i1 */
            if (!(t & 1)) continue;           /* g has no x component */
            int ky = __builtin_popcount((unsigned)t), kx = n - ky;
            double am1 = a_eq_component(p, rho, ux, uy, Teq, kx, ky - 1); /* a^(n-1) over i2..in */
            for (int a = 0; a < p->Q; ++a) {
                double chi = hermite_he(kx, p->xi[2 * a]) * hermite_he(ky, p->xi[2 * a + 1]);
                F[a] += (PLANTED(1) ? -inv : inv) * gy * am1 * chi; /* planted 1: sign */
            }
        }
    }
    for (int a = 0; a < p->Q; ++a) F[a] *= p->w[a];
}

/* g_y at column x and time t */
static double force_at(const oracle_lb_params *p, int x, double t)
{
    if (p->force_amp == 0.0) return 0.0;
    const double pi = 3.14159265358979323846;
    double s = p->force_uniform ? 1.0 : sin(2.0 * pi * (double)x / (double)p->nx);
    return p->force_amp * s * cos(p->force_freq * t);
}

/* macroscopic moments of one cell's populations f[a * stride] */
static void cell_moments(const oracle_lb_params *p, const double *f, size_t stride,
                         double *rho, double *ux, double *uy, double *T)
{
    double r = 0, jx = 0, jy = 0;
    for (int a = 0; a < p->Q; ++a) {
        double fa = f[(size_t)a * stride];
        r += fa;
        jx += p->xi[2 * a] * fa;
        jy += p->xi[2 * a + 1] * fa;
    }
    double vx = jx / r, vy = jy / r, e = 0;
    for (int a = 0; a < p->Q; ++a) {
        double cx = p->xi[2 * a] - vx, cy = p->xi[2 * a + 1] - vy;
        e += (cx * cx + cy * cy) * f[(size_t)a * stride];
    }
    *rho = r;
    *ux = vx;
    *uy = vy;
    *T = e / (2.0 * r);
}

/* Observables of f~ and the collision into fstar (if not NULL). rec: 8 doubles. */
static void collide_and_observe(const oracle_lb_params *p, const double *f, double *fstar,
                                double omega, double t, double *rec,
                                double *orho, double *oux, double *ouy, double *oT, double *osxy)
{
    const int nx = p->nx, ny = p->ny, Q = p->Q;
    const size_t plane = (size_t)nx * ny;
    const double pi = 3.14159265358979323846;
    double mass = 0, mx = 0, my = 0, A = 0, S = 0, H = 0;
    double feq[ORACLE_MAXQ], F[ORACLE_MAXQ];
    const double tau = p->tau;
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            size_t c = (size_t)y * nx + x;
            double rho, ux, uy, T;
            cell_moments(p, f + c, plane, &rho, &ux, &uy, &T);
            double gy = force_at(p, x, t);
            if (gy != 0.0) {
                /* Eq. 2order: rho u = sum xi f~ + rho g dt/2; T of f: T(f~) + dt^2 g^2 / 8 */
                if (p->scheme == 0) {
                    if (!PLANTED(2)) uy += 0.5 * p->dt * gy; /* planted 2: no dt/2 correction */
                    T += p->dt * p->dt * gy * gy / 8.0;
                }
                oracle_force(p, rho, ux, uy, T, gy, F);
            } else {
                for (int a = 0; a < Q; ++a) F[a] = 0.0;
            }
            oracle_feq(p, rho, ux, uy, T, feq);
            double sxy = 0, h = 0;
            for (int a = 0; a < Q; ++a) {
                double fa = f[(size_t)a * plane + c];
                double fneq = fa - feq[a] + (p->scheme == 0 ? 0.5 * p->dt * F[a] : 0.0);
                sxy += p->xi[2 * a] * p->xi[2 * a + 1] * fneq;
                double d = fa - p->w[a] * p->rho0;
                h += d * d / p->w[a];
                if (fstar)
                    fstar[(size_t)a * plane + c] =
                        fa - omega * (fa - feq[a]) + omega * (PLANTED(3) ? 1.0 : tau) * F[a]; /* planted 3 */
            }
            if (p->scheme == 0 && !PLANTED(6)) sxy *= (1.0 - 0.5 * omega); /* planted 6: no (1 - omega/2) */
            double xi_pos = 2.0 * pi * (double)x / (double)nx; /* x_i = i dx, dx = 2 pi / nx */
            mass += rho;
            mx += rho * ux;
            my += rho * uy;
            A += uy * sin(xi_pos);
            S += sxy * cos(xi_pos);
            H += h;
            if (orho) orho[c] = rho;
            if (oux) oux[c] = ux;
            if (ouy) ouy[c] = uy;
            if (oT) oT[c] = T;
            if (osxy) osxy[c] = sxy;
        }
    }
    if (rec) {
        double norm = 2.0 / ((double)nx * ny);
        rec[1] = mass;
        rec[2] = mx;
        rec[3] = my;
        rec[4] = A * norm;
        rec[5] = S * norm;
        rec[6] = H;
        rec[7] = 0.0;
    }
}

/* Lax-Wendroff update of one periodic line: out_i = f_i - C/2 (f_{i+1} - f_{i-1})
 * + C^2/2 (f_{i+1} - 2 f_i + f_{i-1}), read with stride s, length n. */
static void lax_wendroff_line(const double *in, double *out, int n, size_t s, double C)
{
    for (int i = 0; i < n; ++i) {
        double fm = in[(size_t)((i - 1 + n) % n) * s];
        double f0 = in[(size_t)i * s];
        double fp = in[(size_t)((i + 1) % n) * s];
        double Cs = PLANTED(4) ? -C : C; /* planted 4: streaming against xi */
        out[(size_t)i * s] = f0 - 0.5 * Cs * (fp - fm) + 0.5 * Cs * Cs * (fp - 2.0 * f0 + fm);
    }
}

/* Second-order upwind (Beam-Warming) update of one periodic line, read with stride s:
 * the two neighbours on the upstream side of the Courant number C. */
static void upwind2_line(const double *in, double *out, int n, size_t s, double C)
{
    int up = C >= 0.0 ? -1 : 1; /* direction of the upstream neighbours */
    if (PLANTED(9)) up = -up;   /* planted 9: the downstream neighbours */
    double c = fabs(C);
    for (int i = 0; i < n; ++i) {
        double f0 = in[(size_t)i * s];
        double f1 = in[(size_t)(((i + up) % n + n) % n) * s];
        double f2 = in[(size_t)(((i + 2 * up) % n + n) % n) * s];
        out[(size_t)i * s] = f0 - 0.5 * c * (3.0 * f0 - 4.0 * f1 + f2) + 0.5 * c * c * (f0 - 2.0 * f1 + f2);
    }
}

static void stream(const oracle_lb_params *p, const double *fstar, double *fnew, double *tmp)
{
    const int nx = p->nx, ny = p->ny;
    const size_t plane = (size_t)nx * ny;
    for (int a = 0; a < p->Q; ++a) {
        const double *src = fstar + (size_t)a * plane;
        double *dst = fnew + (size_t)a * plane;
        if (p->e) {
            int ex = p->e[2 * a], ey = p->e[2 * a + 1];
            for (int y = 0; y < ny; ++y) {
                int ys = ((y - ey) % ny + ny) % ny;
                for (int x = 0; x < nx; ++x) {
                    int xs = ((x - ex) % nx + nx) % nx;
                    dst[(size_t)y * nx + x] = src[(size_t)ys * nx + xs];
                }
            }
        } else {
            double Cx = p->xi[2 * a] * p->dt / p->dx;
            double Cy = p->xi[2 * a + 1] * p->dt / p->dx; /* dy = dx */
            void (*line)(const double *, double *, int, size_t, double) =
                p->streaming == 1 ? upwind2_line : lax_wendroff_line;
            for (int y = 0; y < ny; ++y)
                line(src + (size_t)y * nx, tmp + (size_t)y * nx, nx, 1, Cx);
            for (int x = 0; x < nx; ++x)
                line(tmp + x, dst + x, ny, (size_t)nx, Cy);
        }
    }
}

/* Shear-wave initial state f~(0) = f^eq(rho = 1, u, T = 1) with
 * u_x = 0, u_y = u0 sin(x_i) + u1 sin(2 pi j / ny) sin(x_i). */
void oracle_lb_init_shear(const oracle_lb_params *p, double u0, double u1, double *f)
{
    const int nx = p->nx, ny = p->ny;
    const size_t plane = (size_t)nx * ny;
    const double pi = 3.14159265358979323846;
    double feq[ORACLE_MAXQ];
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double sx = sin(2.0 * pi * x / nx), sy = sin(2.0 * pi * y / ny);
            oracle_feq(p, 1.0, 0.0, u0 * sx + u1 * sy * sx, 1.0, feq);
            for (int a = 0; a < p->Q; ++a) f[(size_t)a * plane + (size_t)y * nx + x] = feq[a];
        }
}

/* Advance f~ (Q x ny x nx, in/out) from time level n0 by nsteps.  diag: (nsteps + 1)
 * x 8 records (t, mass, mom_x, mom_y, A, S, H, 0) for levels n0..n0+nsteps, or NULL.
 * Returns 0, or -1 on bad arguments. */
int oracle_lb_run_from(const oracle_lb_params *p, double *f, int n0, int nsteps, double *diag)
{
    if (!p || !f || p->Q <= 0 || p->Q > ORACLE_MAXQ || p->N < 0 || p->N > ORACLE_MAXN ||
        p->nx <= 0 || p->ny <= 0 || p->ninner > ORACLE_MAXINNER || nsteps < 0)
        return -1;
    const size_t n = (size_t)p->Q * p->nx * p->ny;
    double *fstar = malloc(n * sizeof(double));
    double *tmp = malloc((size_t)p->nx * p->ny * sizeof(double));
    if (!fstar || !tmp) {
        free(fstar);
        free(tmp);
        return -1;
    }
    double omega = scheme_omega(p);
    for (int s = 0; s < nsteps; ++s) {
        double *rec = diag ? diag + (size_t)s * 8 : NULL;
        double t = (double)(n0 + s) * p->dt;
        collide_and_observe(p, f, fstar, omega, t, rec, NULL, NULL, NULL, NULL, NULL);
        if (rec) rec[0] = t;
        stream(p, fstar, f, tmp);
    }
    if (diag) {
        double *rec = diag + (size_t)nsteps * 8;
        double t = (double)(n0 + nsteps) * p->dt;
        collide_and_observe(p, f, NULL, omega, t, rec, NULL, NULL, NULL, NULL, NULL);
        rec[0] = t;
    }
    free(fstar);
    free(tmp);
    return 0;
}

int oracle_lb_run(const oracle_lb_params *p, double *f, int nsteps, double *diag)
{
    return oracle_lb_run_from(p, f, 0, nsteps, diag);
}

/* Per-cell moments of f~ at time level n (any output may be NULL). */
int oracle_lb_moments(const oracle_lb_params *p, const double *f, int n, double *rho, double *ux,
                      double *uy, double *T, double *sxy)
{
    if (!p || !f) return -1;
    double omega = scheme_omega(p);
    collide_and_observe(p, f, NULL, omega, (double)n * p->dt, NULL, rho, ux, uy, T, sxy);
    return 0;
}
