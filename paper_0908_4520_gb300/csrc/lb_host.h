// Host-side builder declarations (quadrature, step constants).
#pragma once

#include <cmath>
#include <string>
#include <type_traits>
#include <vector>

#include "lb.h"
#include "lb_device.h"

namespace lbh {

struct VelocitySetInfo {
    lb_quadrature quad = LB_D2Q16_GH;
    int q = 0, na = 0, halo = 0, degree = 0;
    bool on_lattice = false;
    bool product_weights = false;   // w_a = W[ix] W[iy] (the collision's per-axis factorisation)
    double c = 0.0;                 // lattice scale (on-lattice)
    std::vector<double> axis;       // distinct component values a_i
    std::vector<double> axis_w;     // 1-D Gauss-Hermite weights (product sets)
    std::vector<int> axis_int;      // integer component values (on-lattice)
    std::vector<int> ix, iy;        // per velocity: axis-node indices
    std::vector<int> ex, ey;        // per velocity: integer lattice vector (on-lattice)
    std::vector<double> w;          // weights
    std::vector<double> xi;         // 2q abscissae
};

void gauss_hermite(int n, std::vector<double>& x, std::vector<double>& w);
int exact_degree(const VelocitySetInfo& vs, double tol);
bool build_velocity_set(lb_quadrature quad, VelocitySetInfo* out, std::string* err);

double hermite_he(int k, double x);

// Message returned by lb_last_error(NULL) on this thread.
void set_last_error(const std::string& m);

// Power of two nearest v > 0 (16-bit storage scales: exact inverses in FP32).
inline double pow2_near(double v) { return std::exp2(std::nearbyint(std::log2(v))); }

// FP32 constants that must sum to exactly one with their complement (the relaxation
// weight omega and 1 - omega, the three Lax-Wendroff weights) are rounded to a
// multiple of 2^-24 (2^-23 at or above 1): then 1 - v is exact in FP32 and no step
// scales the conserved moments by a fixed rounding bias.  The change of v is below
// 6e-8, far inside the FP32 error of the step.
inline double snap_unit(double v) {
    const double q = std::fabs(v) >= 1.0 ? 8388608.0 : 16777216.0;
    return std::nearbyint(v * q) / q;
}

// The FP32 relaxation tables of one omega with the small second terms that make the
// discrete conservation identities exact (fp32_identities.cpp).
void fp32_relax_identities(const VelocitySetInfo& vs, float omega, lbk::Tab<float>& t);

// Kernel tables of a velocity set (FP64 on the host, rounded once to R):
// axis nodes, He_k(a_i)/k!, Lax-Wendroff weights for Courant numbers a_i dt/dx,
// weights and their inverses, xi_x xi_y, |xi|^2, 16-bit storage scales w S.
template <class R>
void build_tab(const VelocitySetInfo& vs, double dt, double dx, double scale, lbk::Tab<R>& t) {
    t = lbk::Tab<R>{};
    // 1-D marginal weights: W_i = sum of w_a over the velocities with ix = i
    std::vector<double> wm(vs.na, 0.0);
    for (int a = 0; a < vs.q; ++a) wm[vs.ix[a]] += vs.w[a];
    for (int i = 0; i < vs.na; ++i) {
        t.a[i] = (R)vs.axis[i];
        t.a2[i] = (R)(vs.axis[i] * vs.axis[i]);
        t.wm[i] = (R)wm[i];
        t.wminv[i] = (R)(1.0 / wm[i]);
        double fact = 1.0;
        for (int k = 0; k <= lbk::kMaxN; ++k) {
            if (k > 1) fact *= k;
            t.hn[i][k] = (R)(hermite_he(k, vs.axis[i]) / fact);
            t.whn[i][k] = (R)(wm[i] * hermite_he(k, vs.axis[i]) / fact);
        }
        const double C = vs.on_lattice ? 0.0 : vs.axis[i] * dt / dx;
        double l0 = 0.5 * C * (1.0 + C), l2 = -0.5 * C * (1.0 - C);
        if (std::is_same<R, float>::value) {  // weights summing to one exactly in FP32
            l0 = snap_unit(l0);
            l2 = snap_unit(l2);
        }
        t.lw[i][0] = (R)l0;
        t.lw[i][1] = (R)(1.0 - l0 - l2);
        t.lw[i][2] = (R)l2;
        // second-order upwind (Beam-Warming), c = |C|: the two upstream neighbours and the cell
        const double c = std::fabs(C);
        double u0 = 0.5 * c * (c - 1.0), u1 = c * (2.0 - c);
        if (std::is_same<R, float>::value) {
            u0 = snap_unit(u0);
            u1 = snap_unit(u1);
        }
        t.uw[i][0] = (R)u0;
        t.uw[i][1] = (R)u1;
        t.uw[i][2] = (R)(1.0 - u0 - u1);
    }
    for (int a = 0; a < vs.q; ++a) {
        t.w[a] = (R)vs.w[a];
        t.winv[a] = (R)(1.0 / vs.w[a]);
        t.xixy[a] = (R)(vs.xi[2 * a] * vs.xi[2 * a + 1]);
        t.xi2[a] = (R)(vs.xi[2 * a] * vs.xi[2 * a] + vs.xi[2 * a + 1] * vs.xi[2 * a + 1]);
        // 16-bit storage scale of velocity a: the power of two nearest w_a S, so that
        // stored = deviation * scinv and deviation = stored * sc are exact inverses (a
        // product sc * scinv != 1 would scale every population by a fixed bias per step)
        const double p2 = pow2_near(vs.w[a] * scale);
        t.sc[a] = (R)p2;
        t.scinv[a] = (R)(1.0 / p2);
    }
}

// The relaxation tables of one omega (the value the kernels receive): omega W_i, omega w_a
// and, in FP32, the small second terms that make the conservation identities exact.
template <class R>
void build_relax(const VelocitySetInfo& vs, R omega, lbk::Tab<R>& t) {
    if constexpr (std::is_same<R, float>::value) {
        fp32_relax_identities(vs, omega, t);
    } else {
        for (int i = 0; i < vs.na; ++i) {
            t.ow[i] = omega * t.wm[i];
            t.owlo[i] = t.hn1lo[i] = t.whn1lo[i] = R(0);
        }
        for (int a = 0; a < vs.q; ++a) t.oww[a] = omega * t.w[a];
        t.mass_lo = R(0);
    }
}

}  // namespace lbh
