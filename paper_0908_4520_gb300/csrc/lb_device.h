// Shared host/device declarations of the fused lattice Boltzmann kernels.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "lb.h"
#include "velocity_sets.h"

namespace lbk {

constexpr int kMaxQ = lbvs::kMaxQ;
constexpr int kMaxNA = lbvs::kMaxNA;
constexpr int kMaxN = 4;
constexpr int kRows = 8;             // warps per block = lattice rows per tile
constexpr int kThreads = 32 * kRows; // threads per block
constexpr int kDiagSlots = 8;        // doubles per partial / record

// Per-handle constant tables, passed by value in the kernel parameter space
// (constant bank): per-velocity entries are read with compile-time indices.
template <class R>
struct Tab {
    R a[kMaxNA];              // axis node values (xi components)
    R hn[kMaxNA][kMaxN + 1];  // He_k(a_i) / k!
    R lw[kMaxNA][3];          // Lax-Wendroff weights of f*(x-1), f*(x), f*(x+1)
    R w[kMaxQ];               // quadrature weights
    R winv[kMaxQ];            // 1 / w
    R xixy[kMaxQ];            // xi_x xi_y
    R xi2[kMaxQ];             // |xi|^2
    R sc[kMaxQ];              // 16-bit storage: deviation = stored * w S
    R scinv[kMaxQ];           // 16-bit storage: stored = deviation / (w S)
};

enum Kind : int { kStep = 0, kMoments = 1, kInit = 2 };

template <class R>
struct Args {
    const void* src;          // populations read (storage type), q planes
    void* dst;                // populations written
    long long plane;          // elements per population plane (ny * pitch)
    int nx, ny, pitch;
    int ntiles_x, ntiles;     // tile grid (tile = kRows rows x 32*V columns)
    int raw;                  // 1: src holds f~ itself (no streaming)
    int isothermal;
    int diag_every;           // record diagnostics when level % diag_every == 0
    R omega, rho0;
    R sigma_fac;              // 1 - omega / 2
    double dt;
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

struct Launch {
    int kind;                 // Kind
    int n_eq;                 // 2..4
    lb_precision prec;
    int grid;                 // blocks (persistent grid-stride over tiles)
    cudaStream_t stream;
    const void* args;         // Args<float> or Args<double> matching prec
};

// Cells per thread along x for a set (the tile width is 32 * V).
constexpr int cells_per_thread(int q) { return q > 40 ? 1 : 2; }

}  // namespace lbk
