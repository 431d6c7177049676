// Compile-time velocity sets of the fused kernels.
//
// Every set is described on an "axis-node" grid: each velocity alpha has
// components xi_alpha = (a[ix(alpha)], a[iy(alpha)]) where a[0..NA) are the
// distinct component values.  The Hermite equilibrium of Sec. 2.1 then
// factorises per axis (He_kx(xi_x) He_ky(xi_y)), which the kernels exploit.
//
//  * Gauss-Hermite product sets (off-lattice, Lax-Wendroff streaming):
//    a = the n-point Gauss-Hermite nodes, alpha = ix * n + iy.
//  * On-lattice sets (exact shift): a = c * ai, ai the integer values listed
//    here; e_alpha = (ai[ix], ai[iy]).  D2Q9, D2Q16 (m=1, n=4), D2Q17, D2Q21
//    and D2Q25 (m=3, n=7) are the sets of Table 1; D2Q37 is the degree-9
//    integer set found by moment matching (its weights and c come from the
//    host builder, which checks that its search lands on these shells).
// The order of the velocities here is THE order of the populations in
// memory and of every per-velocity table the host builds.  kProductWeights
// marks sets whose weights factorise, w_a = W[ix] W[iy] (the Gauss-Hermite
// products, and D2Q9, D2Q16, D2Q25 of Table 1), which the equilibrium exploits.
#pragma once

#ifdef __CUDACC__
#define LB_HD __host__ __device__
#else
#define LB_HD
#endif

namespace lbvs {

constexpr int kMaxQ = 64;
constexpr int kMaxNA = 8;

template <int NQ1>
struct GaussHermiteProduct {
    static constexpr int NA = NQ1;
    static constexpr int Q = NQ1 * NQ1;
    static constexpr bool kOnLattice = false;
    static constexpr bool kProductWeights = true;
    static constexpr int kHalo = 1;
    LB_HD static constexpr int ix(int a) { return a / NQ1; }
    LB_HD static constexpr int iy(int a) { return a % NQ1; }
    // sign of axis node i (the nodes are in ascending order and symmetric; NQ1 even)
    LB_HD static constexpr int axis_sign(int i) { return i < NQ1 / 2 ? -1 : 1; }
    LB_HD static constexpr int axis_int(int) { return 0; }
    LB_HD static constexpr int ex(int) { return 0; }
    LB_HD static constexpr int ey(int) { return 0; }
};

using GH4 = GaussHermiteProduct<4>;
using GH6 = GaussHermiteProduct<6>;
using GH8 = GaussHermiteProduct<8>;

#define LB_ONLATTICE_SET(NAME, QQ, NAA, HALO, PRODW, AXIS, EX, EY)                  \
    struct NAME {                                                                   \
        static constexpr int Q = QQ;                                                \
        static constexpr int NA = NAA;                                              \
        static constexpr bool kOnLattice = true;                                    \
        static constexpr bool kProductWeights = PRODW;                              \
        static constexpr int kHalo = HALO;                                          \
        LB_HD static constexpr int axis_int(int i) {                                \
            constexpr int v[NAA] = AXIS;                                            \
            return v[i];                                                            \
        }                                                                           \
        LB_HD static constexpr int ex(int a) {                                      \
            constexpr int v[QQ] = EX;                                               \
            return v[a];                                                            \
        }                                                                           \
        LB_HD static constexpr int ey(int a) {                                      \
            constexpr int v[QQ] = EY;                                               \
            return v[a];                                                            \
        }                                                                           \
        LB_HD static constexpr int find(int v) {                                    \
            int k = 0;                                                              \
            for (int i = 0; i < NAA; ++i)                                           \
                if (axis_int(i) == v) k = i;                                        \
            return k;                                                               \
        }                                                                           \
        LB_HD static constexpr int ix(int a) { return find(ex(a)); }                \
        LB_HD static constexpr int iy(int a) { return find(ey(a)); }                \
    }

#define LB_LIST(...) {__VA_ARGS__}

LB_ONLATTICE_SET(D2Q9, 9, 3, 1, true, LB_LIST(-1, 0, 1),
                 LB_LIST(-1, 0, 1, -1, 0, 1, -1, 0, 1),
                 LB_LIST(-1, -1, -1, 0, 0, 0, 1, 1, 1));

LB_ONLATTICE_SET(D2Q16I, 16, 4, 4, true, LB_LIST(-4, -1, 1, 4),
                 LB_LIST(-4, -1, 1, 4, -4, -1, 1, 4, -4, -1, 1, 4, -4, -1, 1, 4),
                 LB_LIST(-4, -4, -4, -4, -1, -1, -1, -1, 1, 1, 1, 1, 4, 4, 4, 4));

LB_ONLATTICE_SET(D2Q25, 25, 5, 7, true, LB_LIST(-7, -3, 0, 3, 7),
                 LB_LIST(-7, -3, 0, 3, 7, -7, -3, 0, 3, 7, -7, -3, 0, 3, 7, -7, -3, 0, 3, 7, -7, -3, 0, 3, 7),
                 LB_LIST(-7, -7, -7, -7, -7, -3, -3, -3, -3, -3, 0, 0, 0, 0, 0, 3, 3, 3, 3, 3, 7, 7, 7, 7, 7));

LB_ONLATTICE_SET(D2Q17, 17, 7, 3, false, LB_LIST(-3, -2, -1, 0, 1, 2, 3),
                 LB_LIST(0, -2, 2, -1, 0, 1, -3, -1, 0, 1, 3, -1, 0, 1, -2, 2, 0),
                 LB_LIST(-3, -2, -2, -1, -1, -1, 0, 0, 0, 0, 0, 1, 1, 1, 2, 2, 3));

LB_ONLATTICE_SET(D2Q21, 21, 7, 3, false, LB_LIST(-3, -2, -1, 0, 1, 2, 3),
                 LB_LIST(0, -2, 0, 2, -1, 0, 1, -3, -2, -1, 0, 1, 2, 3, -1, 0, 1, -2, 0, 2, 0),
                 LB_LIST(-3, -2, -2, -2, -1, -1, -1, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 2, 2, 2, 3));

LB_ONLATTICE_SET(D2Q37, 37, 7, 3, false, LB_LIST(-3, -2, -1, 0, 1, 2, 3),
                 LB_LIST(-1, 0, 1, -2, -1, 0, 1, 2, -3, -2, -1, 0, 1, 2, 3, -3, -2, -1, 0, 1, 2, 3,
                         -3, -2, -1, 0, 1, 2, 3, -2, -1, 0, 1, 2, -1, 0, 1),
                 LB_LIST(-3, -3, -3, -2, -2, -2, -2, -2, -1, -1, -1, -1, -1, -1, -1, 0, 0, 0, 0, 0, 0, 0,
                         1, 1, 1, 1, 1, 1, 1, 2, 2, 2, 2, 2, 3, 3, 3));

#undef LB_LIST
#undef LB_ONLATTICE_SET

}  // namespace lbvs
