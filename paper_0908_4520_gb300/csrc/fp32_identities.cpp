// Exact conservation identities of the FP32 collision.
//
// The FP32 collision forms the moments of the streamed populations with the axis
// nodes a_i and rebuilds the equilibrium from weight tables (Sec. 2.1).  In exact
// arithmetic the discrete identities
//     (sum_i omega W_i)(sum_j W_j) = omega                    (mass)
//     (sum_i omega W_i)(sum_j a_j W_j He_1(a_j)) = omega       (y momentum)
//     (sum_i a_i omega W_i He_1(a_i))(sum_j W_j) = omega       (x momentum)
// (and their analogues over the velocities for sets without product weights) make one
// relaxation step conserve mass and momentum (Eq. 2order).  With the factors rounded to
// FP32 they hold only to about 1e-8, and that residual is a fixed relative bias of the
// conserved moments in every collision: at small Kn, where the physical decay per step is
// small, it accumulates into a visible decay-rate error (1e-4 relative after 2000 steps at
// Kn = 0.01 on a 256^2 grid).
//
// The tables keep their round-to-nearest values (moving any weight or node would change
// the higher moments - the pressure, the sound speed - by more than it gains); instead each
// identity gets a small second FP32 term `lo` = eps x (its factor), eps ~ 1e-8 the identity's
// relative residual, which the collision adds in one more FMA per axis node (on-lattice
// sets: the mass residual goes to the rest velocity, which carries no momentum or
// pressure).  The sums are evaluated exactly: every FP32 value is an integer times a power
// of two, so a product of up to three of them is an integer multiple of 2^-110 that fits
// in 128 bits (terms of the lo entries, ~1e-8 of the rest, in long double); the residuals
// are formed from these sums in long double.
#include <cmath>

#include "lb_host.h"

namespace lbh {
namespace {

using i128 = __int128;
constexpr int kScale = 110;

void split(float v, long long* m, int* e) {
    int ex = 0;
    const float fr = std::frexp(v, &ex);
    *m = (long long)std::ldexp(fr, 24);  // v = m 2^(ex - 24), |m| < 2^24
    *e = ex - 24;
}

// exact product of the FP32 values times 2^kScale (false if not representable)
bool exact(std::initializer_list<float> fs, i128* out) {
    i128 m = 1;
    int e = 0;
    for (float f : fs) {
        if (f == 0.0f) {
            *out = 0;
            return true;
        }
        long long mi;
        int ei;
        split(f, &mi, &ei);
        m *= (i128)mi;
        e += ei;
    }
    const int sh = e + kScale;
    int bits = 0;
    for (i128 v = m < 0 ? -m : m; v != 0; v >>= 1) ++bits;
    if (sh < 0 || bits + sh > 120) return false;
    *out = m << sh;
    return true;
}

long double value(i128 v) { return std::ldexp((long double)v, -kScale); }

}  // namespace

void fp32_relax_identities(const VelocitySetInfo& vs, float omega, lbk::Tab<float>& t) {
    const int na = vs.na;
    for (int i = 0; i < lbk::kMaxNA; ++i) t.owlo[i] = t.hn1lo[i] = t.whn1lo[i] = 0.0f;
    t.mass_lo = 0.0f;
    const long double om = omega;
    i128 v;
    if (vs.product_weights) {
        for (int i = 0; i < na; ++i) t.ow[i] = omega * t.wm[i];
        i128 s_ow = 0, s_w = 0, s_awa = 0;
        for (int i = 0; i < na; ++i) {
            if (!exact({t.ow[i]}, &v)) return;
            s_ow += v;
            if (!exact({t.wm[i]}, &v)) return;
            s_w += v;
            if (!exact({t.a[i], t.whn[i][1]}, &v)) return;
            s_awa += v;
        }
        // mass: (omega W_i + lo_i) scales the density term, lo_i = eps omega W_i
        const long double em = om / (value(s_ow) * value(s_w)) - 1.0L;
        for (int i = 0; i < na; ++i) t.owlo[i] = (float)((long double)t.ow[i] * em);
        // y momentum: the first-order y factor W_j He_1(a_j) + lo_j (it multiplies omega W_i,
        // rounded, in the collision)
        const long double ey = om / (value(s_ow) * value(s_awa)) - 1.0L;
        for (int j = 0; j < na; ++j) t.whn1lo[j] = (float)((long double)t.whn[j][1] * ey);
        // x momentum: He_1(a_i) + lo_i inside the density term (omega W_i + lo_i); the terms
        // of the tiny lo_i (~1e-8 of the others) are summed in long double
        i128 s_x = 0;
        long double s_xlo = 0.0L;
        for (int i = 0; i < na; ++i) {
            if (!exact({t.a[i], t.ow[i], t.hn[i][1]}, &v)) return;
            s_x += v;
            s_xlo += (long double)t.a[i] * (long double)t.owlo[i] * (long double)t.hn[i][1];
        }
        const long double ex = om / ((value(s_x) + s_xlo) * value(s_w)) - 1.0L;
        for (int i = 0; i < na; ++i) t.hn1lo[i] = (float)((long double)t.hn[i][1] * ex);
    } else {
        for (int a = 0; a < vs.q; ++a) t.oww[a] = omega * t.w[a];
        i128 s_m = 0, s_x = 0;
        for (int a = 0; a < vs.q; ++a) {
            if (!exact({t.oww[a]}, &v)) return;
            s_m += v;
            if (!exact({t.a[vs.ix[a]], t.oww[a], t.hn[vs.ix[a]][1]}, &v)) return;
            s_x += v;
        }
        // mass: the residual omega - sum omega w_a relaxes with the rest velocity
        t.mass_lo = (float)(om - value(s_m));
        // momentum: He_1(a_i) + lo_i (the y sum is the same by the x <-> y symmetry of the set)
        const long double ex = om / value(s_x) - 1.0L;
        for (int i = 0; i < na; ++i) t.hn1lo[i] = (float)((long double)t.hn[i][1] * ex);
    }
}

}  // namespace lbh
