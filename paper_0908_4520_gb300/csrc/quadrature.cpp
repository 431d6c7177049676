// Host-side velocity-set builder (FP64): nodes, weights and per-axis tables
// for the compile-time sets of velocity_sets.h.
//
//  * Gauss-Hermite rules (Sec. 2.1: quadrature of degree >= 2N for the
//    Hermite coefficients): the Jacobi matrix of the probabilists' Hermite
//    recurrence (zero diagonal, off-diagonal sqrt(k)) is diagonalised by
//    cyclic Jacobi rotations; its eigenvalues are the nodes and the squared
//    first eigenvector components the weights (Golub-Welsch).  Nodes are then
//    Newton-polished on He_n and the weights recomputed as
//    (n-1)! / (n He_{n-1}(x)^2), which is exact for the unit-mass rule.
//  * Table 1 sets from the surds printed there.
//  * D2Q37 by moment matching over fully symmetric integer shells with
//    components <= 3 (the search idea of Sec. 2.3): for 8 shells of total size
//    37 the 9 symmetry-distinct even moment equations of degree <= 8 are
//    linear in the shell weights W and polynomial in t = 1/c^2; consistency,
//    det[M | g t^d] = 0, is a quartic in t whose admissible root (all W > 0,
//    smallest c) fixes the set.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "lb_host.h"
#include "velocity_sets.h"

namespace lbh {

// probabilists' Hermite polynomial He_k(x) by its three-term recurrence
double hermite_he(int k, double x) {
    double h0 = 1.0, h1 = x;
    if (k == 0) return 1.0;
    for (int j = 1; j < k; ++j) {
        const double h2 = x * h1 - j * h0;
        h0 = h1;
        h1 = h2;
    }
    return h1;
}

namespace {

double he(int k, double x) { return hermite_he(k, x); }

// eigenvalues / vectors of a small dense symmetric matrix (cyclic Jacobi)
void jacobi_eigen(int n, std::vector<double>& a, std::vector<double>& v) {
    v.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) v[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += a[(size_t)p * n + q] * a[(size_t)p * n + q];
        if (off < 1e-300) break;
        for (int p = 0; p < n; ++p) {
            for (int q = p + 1; q < n; ++q) {
                const double apq = a[(size_t)p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                const double theta = (a[(size_t)q * n + q] - a[(size_t)p * n + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {  // columns p, q
                    const double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
                    a[(size_t)k * n + p] = c * akp - s * akq;
                    a[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // rows p, q
                    const double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
                    a[(size_t)p * n + k] = c * apk - s * aqk;
                    a[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = v[(size_t)k * n + p], vkq = v[(size_t)k * n + q];
                    v[(size_t)k * n + p] = c * vkp - s * vkq;
                    v[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
        }
    }
}

long long dfact(int k) { return k <= 0 ? 1 : k * dfact(k - 2); }

double gaussian_moment(int a, int b) {
    if ((a & 1) || (b & 1)) return 0.0;
    return (double)(dfact(a - 1) * dfact(b - 1));
}

// fully symmetric orbit of (a, b)
std::vector<std::pair<int, int>> orbit(int a, int b) {
    std::vector<std::pair<int, int>> pts;
    for (int sx : {1, -1})
        for (int sy : {1, -1}) {
            pts.push_back({sx * a, sy * b});
            pts.push_back({sx * b, sy * a});
        }
    std::sort(pts.begin(), pts.end());
    pts.erase(std::unique(pts.begin(), pts.end()), pts.end());
    return pts;
}

// Gaussian elimination with partial pivoting; returns false if singular.
bool solve_dense(int n, std::vector<long double> m, std::vector<long double> rhs, std::vector<long double>& x) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs((double)m[(size_t)r * n + c]) > std::fabs((double)m[(size_t)piv * n + c])) piv = r;
        if (std::fabs((double)m[(size_t)piv * n + c]) < 1e-300) return false;
        if (piv != c) {
            for (int k = 0; k < n; ++k) std::swap(m[(size_t)c * n + k], m[(size_t)piv * n + k]);
            std::swap(rhs[c], rhs[piv]);
        }
        for (int r = c + 1; r < n; ++r) {
            const long double f = m[(size_t)r * n + c] / m[(size_t)c * n + c];
            for (int k = c; k < n; ++k) m[(size_t)r * n + k] -= f * m[(size_t)c * n + k];
            rhs[r] -= f * rhs[c];
        }
    }
    x.assign(n, 0.0L);
    for (int r = n - 1; r >= 0; --r) {
        long double s = rhs[r];
        for (int k = r + 1; k < n; ++k) s -= m[(size_t)r * n + k] * x[k];
        x[r] = s / m[(size_t)r * n + r];
    }
    return true;
}

long double det_dense(int n, std::vector<long double> m) {
    long double det = 1.0L;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs((double)m[(size_t)r * n + c]) > std::fabs((double)m[(size_t)piv * n + c])) piv = r;
        if (m[(size_t)piv * n + c] == 0.0L) return 0.0L;
        if (piv != c) {
            for (int k = 0; k < n; ++k) std::swap(m[(size_t)c * n + k], m[(size_t)piv * n + k]);
            det = -det;
        }
        det *= m[(size_t)c * n + c];
        for (int r = c + 1; r < n; ++r) {
            const long double f = m[(size_t)r * n + c] / m[(size_t)c * n + c];
            for (int k = c; k < n; ++k) m[(size_t)r * n + k] -= f * m[(size_t)c * n + k];
        }
    }
    return det;
}

const int kMoments[9][2] = {{0, 0}, {2, 0}, {4, 0}, {2, 2}, {6, 0}, {4, 2}, {8, 0}, {6, 2}, {4, 4}};

// Solve one 8-shell candidate.  On success fills W (per shell) and c.
bool solve_shells(const std::vector<std::pair<int, int>>& shells, std::vector<double>& W, double& c) {
    const int ns = 8;
    std::vector<long double> M(9 * ns);
    std::vector<long double> g(9);
    int d[9];
    for (int r = 0; r < 9; ++r) {
        const int a = kMoments[r][0], b = kMoments[r][1];
        for (int s = 0; s < ns; ++s) {
            long double acc = 0;
            for (auto& p : orbit(shells[s].first, shells[s].second))
                acc += std::pow((long double)p.first, a) * std::pow((long double)p.second, b);
            M[(size_t)r * ns + s] = acc;
        }
        g[r] = gaussian_moment(a, b);
        d[r] = (a + b) / 2;
    }
    // quartic coefficients: det [M | g t^d] = sum_r (-1)^(r+ns) g_r minor_r t^d_r
    long double poly[5] = {0, 0, 0, 0, 0};
    for (int r = 0; r < 9; ++r) {
        std::vector<long double> minor;
        for (int rr = 0; rr < 9; ++rr)
            if (rr != r)
                for (int s = 0; s < ns; ++s) minor.push_back(M[(size_t)rr * ns + s]);
        const long double sign = ((r + ns) % 2 == 0) ? 1.0L : -1.0L;
        poly[d[r]] += sign * g[r] * det_dense(ns, minor);
    }
    auto P = [&](long double t) {
        long double v = 0;
        for (int k = 4; k >= 0; --k) v = v * t + poly[k];
        return v;
    };
    bool found = false;
    double best_c = 0;
    std::vector<double> bestW;
    // positive real roots by a log-spaced scan and bisection
    const int nscan = 4000;
    long double tprev = 1e-3L, pprev = P(tprev);
    for (int i = 1; i <= nscan; ++i) {
        const long double t = 1e-3L * std::pow(1e5L, (long double)i / nscan);
        const long double pv = P(t);
        if ((pprev < 0) != (pv < 0)) {
            long double lo = tprev, hi = t, plo = pprev;
            for (int it = 0; it < 200; ++it) {
                const long double mid = 0.5L * (lo + hi);
                const long double pm = P(mid);
                if ((pm < 0) == (plo < 0)) {
                    lo = mid;
                    plo = pm;
                } else {
                    hi = mid;
                }
            }
            long double troot = 0.5L * (lo + hi);
            // weights by least squares over the 9 equations (normal equations),
            // then Newton on the square 9x9 system in (W, t)
            std::vector<long double> nrm(ns * ns, 0.0L), rhs(ns, 0.0L), w;
            for (int i = 0; i < ns; ++i) {
                for (int j = 0; j < ns; ++j)
                    for (int r = 0; r < 9; ++r) nrm[(size_t)i * ns + j] += M[(size_t)r * ns + i] * M[(size_t)r * ns + j];
                for (int r = 0; r < 9; ++r) rhs[i] += M[(size_t)r * ns + i] * g[r] * std::pow(troot, d[r]);
            }
            if (solve_dense(ns, nrm, rhs, w)) {
                std::vector<long double> x(w);
                x.push_back(troot);
                for (int it = 0; it < 6; ++it) {
                    std::vector<long double> J(81), F(9), dx;
                    for (int r = 0; r < 9; ++r) {
                        long double fr = -g[r] * std::pow(x[8], d[r]);
                        for (int s = 0; s < ns; ++s) {
                            fr += M[(size_t)r * ns + s] * x[s];
                            J[(size_t)r * 9 + s] = M[(size_t)r * ns + s];
                        }
                        J[(size_t)r * 9 + 8] = d[r] > 0 ? -g[r] * d[r] * std::pow(x[8], d[r] - 1) : 0.0L;
                        F[r] = -fr;
                    }
                    if (!solve_dense(9, J, F, dx)) break;
                    for (int k = 0; k < 9; ++k) x[k] += dx[k];
                }
                bool pos = x[8] > 0;
                for (int s = 0; s < ns; ++s) pos = pos && x[s] > 0;
                if (pos) {
                    const double cc = 1.0 / std::sqrt((double)x[8]);
                    if (!found || cc < best_c) {
                        found = true;
                        best_c = cc;
                        bestW.assign(ns, 0.0);
                        for (int s = 0; s < ns; ++s) bestW[s] = (double)x[s];
                    }
                }
            }
        }
        tprev = t;
        pprev = pv;
    }
    if (found) {
        W = bestW;
        c = best_c;
    }
    return found;
}

void product_axis(VelocitySetInfo& vs, int n) {
    gauss_hermite(n, vs.axis, vs.axis_w);
}

template <class VS>
void fill_indices(VelocitySetInfo& vs) {
    vs.q = VS::Q;
    vs.na = VS::NA;
    vs.halo = VS::kHalo;
    vs.on_lattice = VS::kOnLattice;
    vs.product_weights = VS::kProductWeights;
    vs.ix.resize(VS::Q);
    vs.iy.resize(VS::Q);
    vs.ex.resize(VS::Q);
    vs.ey.resize(VS::Q);
    for (int a = 0; a < VS::Q; ++a) {
        vs.ix[a] = VS::ix(a);
        vs.iy[a] = VS::iy(a);
        vs.ex[a] = VS::ex(a);
        vs.ey[a] = VS::ey(a);
    }
    if (VS::kOnLattice) {
        vs.axis_int.resize(VS::NA);
        for (int i = 0; i < VS::NA; ++i) vs.axis_int[i] = VS::axis_int(i);
    }
}

// weight of an on-lattice velocity from its shell (|ex|, |ey|) unordered
double shell_weight(const std::vector<std::pair<int, int>>& shells, const std::vector<double>& W, int ex, int ey) {
    int a = std::abs(ex), b = std::abs(ey);
    if (a < b) std::swap(a, b);
    for (size_t s = 0; s < shells.size(); ++s)
        if (shells[s].first == a && shells[s].second == b) return W[s];
    return -1.0;
}

}  // namespace

void gauss_hermite(int n, std::vector<double>& x, std::vector<double>& w) {
    std::vector<double> J((size_t)n * n, 0.0), V;
    for (int k = 1; k < n; ++k) J[(size_t)(k - 1) * n + k] = J[(size_t)k * n + k - 1] = std::sqrt((double)k);
    jacobi_eigen(n, J, V);
    x.resize(n);
    for (int i = 0; i < n; ++i) x[i] = J[(size_t)i * n + i];
    std::sort(x.begin(), x.end());
    double nm1_fact = 1.0;
    for (int k = 2; k < n; ++k) nm1_fact *= k;
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        double xi = x[i];
        for (int it = 0; it < 8; ++it) {  // Newton on He_n, He_n' = n He_{n-1}
            const double step = he(n, xi) / (n * he(n - 1, xi));
            xi -= step;
            if (std::fabs(step) < 1e-17 * std::max(1.0, std::fabs(xi))) break;
        }
        x[i] = xi;
    }
    for (int i = 0; i < n / 2; ++i) {  // exact symmetry about 0
        const double s = 0.5 * (x[n - 1 - i] - x[i]);
        x[i] = -s;
        x[n - 1 - i] = s;
    }
    if (n % 2) x[n / 2] = 0.0;
    double sum = 0.0;
    for (int i = 0; i < n; ++i) {
        const double h = he(n - 1, x[i]);
        w[i] = nm1_fact / (n * h * h);
        sum += w[i];
    }
    for (int i = 0; i < n; ++i) w[i] /= sum;
}

int exact_degree(const VelocitySetInfo& vs, double tol) {
    for (int D = 0; D <= 20; ++D) {
        for (int a = 0; a <= D; ++a) {
            const int b = D - a;
            double s = 0.0;
            for (int q = 0; q < vs.q; ++q) s += vs.w[q] * std::pow(vs.xi[2 * q], a) * std::pow(vs.xi[2 * q + 1], b);
            const double ref = gaussian_moment(a, b);
            if (std::fabs(s - ref) > tol * std::max(1.0, std::fabs(ref))) return D - 1;
        }
    }
    return 20;
}

bool build_velocity_set(lb_quadrature quad, VelocitySetInfo* out, std::string* err) {
    VelocitySetInfo vs;
    vs.quad = quad;
    std::vector<std::pair<int, int>> shells;
    std::vector<double> W;
    auto onlattice_from_1d = [&](const std::vector<int>& ints, const std::vector<double>& w1, double T0) {
        vs.c = 1.0 / std::sqrt(T0);
        vs.w.resize(vs.q);
        for (int a = 0; a < vs.q; ++a) {
            double wx = -1, wy = -1;
            for (size_t k = 0; k < ints.size(); ++k) {
                if (ints[k] == vs.ex[a]) wx = w1[k];
                if (ints[k] == vs.ey[a]) wy = w1[k];
            }
            vs.w[a] = wx * wy;
        }
    };
    switch (quad) {
        case LB_D2Q16_GH: fill_indices<lbvs::GH4>(vs); product_axis(vs, 4); break;
        case LB_D2Q36_GH: fill_indices<lbvs::GH6>(vs); product_axis(vs, 6); break;
        case LB_D2Q64_GH: fill_indices<lbvs::GH8>(vs); product_axis(vs, 8); break;
        case LB_D2Q9:
            fill_indices<lbvs::D2Q9>(vs);
            shells = {{0, 0}, {1, 0}, {1, 1}};
            W = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0};
            vs.c = std::sqrt(3.0);
            break;
        case LB_D2Q16_INT: {
            fill_indices<lbvs::D2Q16I>(vs);
            const double m = 1, n = 4, s = std::sqrt(m * m * m * m - 10 * n * n * m * m + n * n * n * n);
            const double Wm = (m * m - 5 * n * n + s) / (12 * (m * m - n * n));
            const double Wn = (5 * m * m - n * n - s) / (12 * (m * m - n * n));
            const double T0 = (m * m + n * n + s) / 6;
            onlattice_from_1d({-4, -1, 1, 4}, {Wn, Wm, Wm, Wn}, T0);
            break;
        }
        case LB_D2Q25: {
            fill_indices<lbvs::D2Q25>(vs);
            const double m = 3, n = 7, m2 = m * m, n2 = n * n;
            const double D5 = std::sqrt(9 * m2 * m2 - 42 * n2 * m2 + 9 * n2 * n2);
            const double W0 = (-3 * m2 * m2 - 3 * n2 * n2 + 54 * m2 * n2 - (m2 + n2) * D5) / (75 * m2 * n2);
            const double Wm = (9 * m2 * m2 - 6 * n2 * n2 - 27 * n2 * m2 + (3 * m2 - 2 * n2) * D5) / (300 * m2 * (m2 - n2));
            const double Wn = (9 * n2 * n2 - 6 * m2 * m2 - 27 * n2 * m2 + (3 * n2 - 2 * m2) * D5) / (300 * n2 * (n2 - m2));
            const double T0 = (3 * m2 + 3 * n2 + D5) / 30;
            onlattice_from_1d({-7, -3, 0, 3, 7}, {Wn, Wm, W0, Wm, Wn}, T0);
            break;
        }
        case LB_D2Q17: {
            fill_indices<lbvs::D2Q17>(vs);
            const double s = std::sqrt(193.0);
            shells = {{0, 0}, {1, 0}, {1, 1}, {2, 2}, {3, 0}};
            W = {(575 + 193 * s) / 8100, (3355 - 91 * s) / 18000, (655 + 17 * s) / 27000,
                 (685 - 49 * s) / 54000, (1445 - 101 * s) / 162000};
            vs.c = std::sqrt((125 + 5 * s) / 72);
            break;
        }
        case LB_D2Q21:
            fill_indices<lbvs::D2Q21>(vs);
            shells = {{0, 0}, {1, 0}, {1, 1}, {2, 0}, {2, 2}, {3, 0}};
            W = {91.0 / 324, 1.0 / 12, 2.0 / 27, 7.0 / 360, 1.0 / 432, 1.0 / 1620};
            vs.c = std::sqrt(1.5);
            break;
        case LB_D2Q37: {
            fill_indices<lbvs::D2Q37>(vs);
            const std::vector<std::pair<int, int>> cand = {{0, 0}, {1, 0}, {1, 1}, {2, 0}, {2, 1},
                                                           {2, 2}, {3, 0}, {3, 1}, {3, 2}, {3, 3}};
            bool ok = false;
            // 8-shell subsets in lexicographic order of the candidate list
            std::vector<int> idx(8);
            for (int i = 0; i < 8; ++i) idx[i] = i;
            while (!ok) {
                std::vector<std::pair<int, int>> sub;
                int npts = 0;
                for (int i : idx) {
                    sub.push_back(cand[i]);
                    npts += (int)orbit(cand[i].first, cand[i].second).size();
                }
                if (npts == 37) {
                    double c = 0;
                    std::vector<double> Ws;
                    if (solve_shells(sub, Ws, c)) {
                        shells = sub;
                        W = Ws;
                        vs.c = c;
                        // verify below; accept the first subset whose set is exact to degree 9
                        VelocitySetInfo probe = vs;
                        probe.w.resize(probe.q);
                        probe.xi.resize(2 * probe.q);
                        bool match = true;
                        for (int a = 0; a < probe.q; ++a) {
                            probe.w[a] = shell_weight(shells, W, probe.ex[a], probe.ey[a]);
                            if (probe.w[a] < 0) match = false;
                            probe.xi[2 * a] = c * probe.ex[a];
                            probe.xi[2 * a + 1] = c * probe.ey[a];
                        }
                        if (match && exact_degree(probe, 1e-10) >= 9) ok = true;
                    }
                }
                if (ok) break;
                // next combination of 8 out of 10
                int i = 7;
                while (i >= 0 && idx[i] == 10 - 8 + i) --i;
                if (i < 0) break;
                ++idx[i];
                for (int j = i + 1; j < 8; ++j) idx[j] = idx[j - 1] + 1;
            }
            if (!ok) {
                if (err) *err = "D2Q37: no admissible shell set matches the compiled velocity list";
                return false;
            }
            break;
        }
        default:
            if (err) *err = "unknown quadrature";
            return false;
    }
    if (vs.on_lattice) {
        vs.axis.resize(vs.na);
        for (int i = 0; i < vs.na; ++i) vs.axis[i] = vs.c * vs.axis_int[i];
        if (!shells.empty()) {
            vs.w.resize(vs.q);
            for (int a = 0; a < vs.q; ++a) {
                vs.w[a] = shell_weight(shells, W, vs.ex[a], vs.ey[a]);
                if (vs.w[a] <= 0) {
                    if (err) *err = "velocity outside the set's shells";
                    return false;
                }
            }
        }
    } else {
        vs.c = 0.0;
        vs.w.resize(vs.q);
        for (int a = 0; a < vs.q; ++a) vs.w[a] = vs.axis_w[vs.ix[a]] * vs.axis_w[vs.iy[a]];
    }
    vs.xi.resize(2 * vs.q);
    for (int a = 0; a < vs.q; ++a) {
        vs.xi[2 * a] = vs.axis[vs.ix[a]];
        vs.xi[2 * a + 1] = vs.axis[vs.iy[a]];
    }
    vs.degree = exact_degree(vs, 1e-10);
    *out = vs;
    return true;
}

}  // namespace lbh
