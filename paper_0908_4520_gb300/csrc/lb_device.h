// Shared host/device declarations of the fused lattice Boltzmann kernels.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda.h>
#include <cuda_runtime.h>

#include "lb.h"
#include "velocity_sets.h"

namespace lbk {

constexpr int kMaxQ = lbvs::kMaxQ;
constexpr int kMaxNA = lbvs::kMaxNA;
constexpr int kMaxN = 4;
constexpr int kDiagSlots = 8;  // doubles per partial / record
constexpr int kGhostX = 8;     // ghost columns kept on each side of a population row

// Per-handle constant tables, passed by value in the kernel parameter space
// (constant bank): per-velocity entries are read with compile-time indices.
template <class R>
struct Tab {
    R a[kMaxNA];              // axis node values (xi components)
    R a2[kMaxNA];             // a_i^2
    R wm[kMaxNA];             // 1-D marginal weights W_i (product-weight sets: w_a = W[ix] W[iy])
    R wminv[kMaxNA];          // 1 / W_i
    R hn[kMaxNA][kMaxN + 1];  // He_k(a_i) / k!
    R whn[kMaxNA][kMaxN + 1]; // W_i He_k(a_i) / k!
    R lw[kMaxNA][3];          // Lax-Wendroff weights of f*(x-1), f*(x), f*(x+1)
    R uw[kMaxNA][3];          // second-order upwind weights of f*(x-2s), f*(x-s), f*(x), s = sign(a_i)
    R w[kMaxQ];               // quadrature weights
    R winv[kMaxQ];            // 1 / w
    R xixy[kMaxQ];            // xi_x xi_y
    R xi2[kMaxQ];             // |xi|^2
    // relaxation tables of one omega; the `lo` entries (FP32 only, else 0) are the small second
    // terms that make the FP32 conservation identities exact (fp32_identities.cpp)
    R ow[kMaxNA];             // omega W_i (the relaxation weight of the per-axis factors)
    R owlo[kMaxNA];           // second term of omega W_i in the density term (mass)
    R hn1lo[kMaxNA];          // second term of He_1(a_i) in the x moment
    R whn1lo[kMaxNA];         // second term of W_i He_1(a_i) in the y moment
    R oww[kMaxQ];             // omega w_a (sets without product weights)
    R mass_lo;                // sets without product weights: mass residual, relaxed with the rest velocity
    R sc[kMaxQ];              // 16-bit storage: deviation = stored * w S
    R scinv[kMaxQ];           // 16-bit storage: stored = deviation / (w S)
};

enum Kind : int {
    kStep = 0, kMoments = 1, kInit = 2, kStepTma = 3, kStepForced = 4, kMomentsTma = 5, kStepTmaStore = 6,
    kQueryShape = -1
};

// Population layout: plane a, row y, column x at
//   a * plane + origin + y * pitch + x,   origin = gy * pitch + kGhostX,
// for -kGhostX <= x < nx + kGhostX and -gy <= y < ny + gy: the rim holds the
// periodic images of the grid, rewritten by every launch that writes the
// populations, so streaming never wraps an index.
template <class R>
struct Args {
    CUtensorMap tmap;         // TMA view of src (step kernel with TMA staging only)
    CUtensorMap tmap_st;      // TMA view of the cells of dst, nx x ny x q (store-staged kernel only)
    const void* src;          // populations read (storage type), q planes
    void* dst;                // populations written
    long long plane;          // elements per population plane ((ny + 2 gy) * pitch)
    long long origin;         // offset of cell (0, 0) in a plane
    int nx, ny, pitch, gy;
    int ntiles_x, ntiles;     // tile grid (tile = rows x 32*V columns)
    int x0_last;              // first column of the last tile of a row (nx - 32V when nx >= 32V)
    int raw;                  // 1: src holds f~ itself (no streaming)
    int isothermal;
    int diag_every;           // record diagnostics when level % diag_every == 0
    int withhold_stage;       // test of the bounded waits (lb_params.test_withhold_stage)
    R omega, rho0;
    R sigma_fac;              // 1 - omega / 2 (Eq. 2order), 1 (Eq. slb)
    R tau;                    // collision time of Eq. bgk
    R hdt;                    // dt / 2 of the force corrections of the moments (Eq. 2order), 0 (Eq. slb)
    double dt;
    double force_amp;         // body force g_y = force_amp sin(x_i) cos(force_freq t); 0: none
    double force_freq;
    const R* sinx;            // sin(x_i), nx entries
    const R* cosx;            // cos(x_i)
    double* partials;         // gridDim.x * kDiagSlots
    unsigned int* ticket;     // last-block election counter (returns to 0)
    long long* level;         // device time level, advanced by every step launch
    lb_diag* ring;            // diagnostics ring
    int ring_cap;
    int* status;              // bit 0: non-finite state
    // moments kind
    double *o_rho, *o_ux, *o_uy, *o_T, *o_sxy;
    double* o_pop;            // full f~ as FP64, q * ny * nx (may be null)
    // init kind
    double u0, u1;            // shear wave amplitudes (fields == null)
    const double *i_rho, *i_ux, *i_uy, *i_T; // initial fields (may be null)
    Tab<R> tab;
};

// Launch geometry of a compiled (set, storage) unit.
struct Shape {
    int V;          // cells per thread along x (tile width 32 V), register kernels
    int rows;       // warps per block = lattice rows per tile
    int threads;    // 32 * rows
    int occupancy;  // resident blocks per SM of the step kernel
    // TMA-staged step kernel (0 = not built for this unit)
    int tma;
    int tma_V, tma_rows, tma_threads, tma_smem, tma_occupancy;
    int tma_tw;     // cells a tile row produces (32 V, or 30 with halo lanes)
    int box_w, box_h, box_d;  // tensor-map box (x, y, velocities)
    // store-staged TMA kernel (0 = not built for this unit): tile of st_rows x st_tw cells,
    // load box st_box_w x st_box_h x box_d, one store box st_tw x st_rows x q per tile
    int st, st_tw, st_rows, st_threads, st_smem, st_occupancy, st_box_w, st_box_h;
    int st_auto;    // 1: the automatic choice prefers the store-staged kernel on large grids
};

struct Launch {
    int kind;                 // Kind
    int n_eq;                 // 1..4
    int upwind;               // 1: second-order upwind streaming (off-lattice sets, 32/64-bit storage)
    int grid;                 // blocks (persistent grid-stride over tiles)
    cudaStream_t stream;
    const void* args;         // Args<float>/Args<double> matching the unit, or Shape* for kQueryShape
};

using LaunchFn = cudaError_t (*)(const Launch&);

// Every generated (set, storage) unit registers its entry point at load time.
bool register_launcher(int quadrature, int precision, LaunchFn fn);
LaunchFn find_launcher(int quadrature, int precision);

}  // namespace lbk
