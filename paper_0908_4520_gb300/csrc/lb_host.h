// Host-side builder declarations (quadrature, step constants).
#pragma once

#include <string>
#include <vector>

#include "lb.h"

namespace lbh {

struct VelocitySetInfo {
    lb_quadrature quad = LB_D2Q16_GH;
    int q = 0, na = 0, halo = 0, degree = 0;
    bool on_lattice = false;
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

}  // namespace lbh
