/*
 * lb.h - C-ABI of the GB300 high-order lattice Boltzmann library (liblb.so).
 *
 * One handle = one periodic nx x ny lattice advanced by the fused BGK
 * collide-stream update of the paper (Meng & Zhang, "Accuracy analysis of
 * high-order lattice Boltzmann models for rarefied gas flows"):
 *   moments    rho = sum f~, rho u = sum xi f~, 2 rho T = sum |xi - u|^2 f~  (Sec. 2.2)
 *   equilibrium Hermite expansion of the Maxwellian truncated at order N     (Sec. 2.1,
 *              Eqs. approxf, an, demoeq; N = 1: Sec. 3.3, Eq. lbm1)
 *   collision  f* = f~ - omega (f~ - f^eq), omega = dt / (tau + dt/2)         (Eq. 2order;
 *              the first-order scheme of Eq. slb as an option)
 *   streaming  exact shift along integer e_alpha for on-lattice sets (Table 1),
 *              Lax-Wendroff for off-lattice Gauss-Hermite product sets
 *              (Sec. 2.3; Sec. 3.3; caption of the D2Q400 figure), second-order
 *              upwind as an option
 * plus the body force of the driven standing shear wave (Secs. 2.1, 2.2, 4), batches
 * of many small lattices, a request loop, and the reduced discrete velocity method of
 * Sec. 3.3 (free and driven).
 *
 * Conventions (every function):
 *  - Returns lb_status; nothing is thrown across the ABI.  Out-pointers are
 *    written only on LB_OK.  lb_last_error(h) holds a human-readable message
 *    for the handle's last failure.
 *  - The library owns all device memory of a handle (optionally through the
 *    caller's allocator callbacks in lb_params).  The caller owns host arrays.
 *  - Work is enqueued on the handle's CUDA stream.  lb_step returns after
 *    enqueueing; device-side errors (non-finite state) surface at the next
 *    synchronising call (lb_moments, lb_diagnostics, lb_synchronize).
 *  - A handle is not thread-safe; different handles may be used from
 *    different threads and run concurrently on different streams.
 *
 * Units (Eq. nondime): lengths in 1/theta, velocities in sqrt(R T0), so the
 * grid spacing is dx = dy = 2 pi / nx and rho0 = T0 = 1.
 */
#ifndef LB_H
#define LB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_handle lb_handle;

typedef enum {
    LB_OK = 0,
    LB_ERR_ARG = -1,          /* invalid argument (sizes, NULL handle, omega out of (0,2), ...) */
    LB_ERR_UNSUPPORTED = -2,  /* valid request this build does not provide */
    LB_ERR_NOMEM = -3,        /* device or host allocation failed */
    LB_ERR_CUDA = -4,         /* CUDA runtime error (message in lb_last_error) */
    LB_ERR_UNSTABLE = -5,     /* the state became non-finite */
    LB_ERR_TIMEOUT = -6,      /* a bounded device wait ran out (the kernel stopped early) */
    LB_ERR_BUDGET = -7,       /* request exceeds the configured device-memory budget */
    LB_ERR_STATE = -8         /* call out of order (e.g. lb_step before an init) */
} lb_status;

/* Velocity sets.  *_GH: tensor products of the n-point Gauss-Hermite rule
 * (off-lattice, Lax-Wendroff streaming).  The others are on-lattice
 * (xi = c e, e integer, exact shift): D2Q9, D2Q16 (m=1,n=4), D2Q17, D2Q21
 * and D2Q25 (m=3,n=7) from Table 1; D2Q37 (degree 9, |e| <= 3) is built by
 * moment matching over integer shells (the search of Sec. 2.3). */
typedef enum {
    LB_D2Q16_GH = 0,
    LB_D2Q36_GH = 1,
    LB_D2Q64_GH = 2,
    LB_D2Q37 = 3,
    LB_D2Q9 = 4,
    LB_D2Q16_INT = 5,
    LB_D2Q17 = 6,
    LB_D2Q21 = 7,
    LB_D2Q25 = 8
} lb_quadrature;

/* Storage of the populations.  F32/F64 store the deviation f~ - w rho0;
 * BF16/F16 store (f~ - w rho0) / s_a, s_a the power of two nearest w_a S for a
 * per-handle scale S (so that the load and store scales are exact inverses),
 * rounded stochastically.  The arithmetic is FP32 for F32/BF16/F16 and FP64 for F64. */
typedef enum { LB_F32 = 0, LB_F64 = 1, LB_BF16 = 2, LB_F16 = 3 } lb_precision;

/* How kn maps to the collision time tau of Eq. bgk.
 * LAMBDA: kn is lambda/L with lambda = mu/p sqrt(pi R T/2), tau = kn sqrt(2/pi).
 * PAPER:  kn is Eq. KN, tau = kn. */
typedef enum { LB_KN_LAMBDA = 0, LB_KN_PAPER = 1 } lb_kn_convention;

/* Time discretisation of the collision (Sec. 2.2).
 * SECOND_ORDER (default): Eq. 2order; the state is f~, omega = dt / (tau + dt/2),
 *   rho u = sum xi f~ + rho g dt/2 and sigma_xy carries the factor (1 - omega/2).
 * FIRST_ORDER: the standard LB of Eq. slb (first-order upwind along the
 *   characteristic); the state is f itself, omega = dt / tau (the relaxation time
 *   tau/dt without the -1/2 correction), the force enters as dt g_alpha, and
 *   rho u = sum xi f, sigma_xy = sum xi_x xi_y (f - f^eq).  It is linearly unstable
 *   for omega >= 2, so lb_create_ex rejects tau <= dt/2 (LB_ERR_ARG).  Streaming is
 *   the velocity set's own in both (exact shift, or Lax-Wendroff off-lattice). */
typedef enum { LB_SCHEME_SECOND_ORDER = 0, LB_SCHEME_FIRST_ORDER = 1 } lb_scheme;

/* Streaming of the off-lattice (Gauss-Hermite product) sets.
 * LAX_WENDROFF (default): 1-D Lax-Wendroff along x then y (the scheme named in
 *   Sec. 3.3); on-lattice sets always stream by the exact shift.
 * UPWIND2: 1-D second-order upwind (Beam-Warming) along x then y, from the cell and
 *   its two upstream neighbours: out_i = f_i - c/2 (3 f_i - 4 f_{i-s} + f_{i-2s})
 *   + c^2/2 (f_i - 2 f_{i-s} + f_{i-2s}), c = |C|, s = sign(C), C = xi dt/dx
 *   (exact shift at c = 1).  Off-lattice sets with F32/F64 storage only
 *   (LB_ERR_UNSUPPORTED otherwise); the rim holds two ghost rows.  F32 steps run the
 *   TMA-staged kernel (28-cell tile rows), F64 the plain-load kernel; same bits. */
typedef enum { LB_STREAM_LAX_WENDROFF = 0, LB_STREAM_UPWIND2 = 1 } lb_streaming;

typedef struct {
    lb_quadrature quadrature;
    int n_eq;                  /* Hermite order N of the equilibrium, 1..4.  N = 1 is the
                                  first-order expansion f^eq = w rho (1 + xi.u) of Sec. 3.3
                                  (Eq. lbm1, the isothermal linearised BGK form): T does not
                                  enter it and is reported only */
    int nx, ny;                /* periodic grid; nx even, >= 2; ny >= 1 */
    double kn;                 /* Knudsen number (> 0), see kn_convention */
    lb_precision precision;    /* default LB_F32 */
    lb_kn_convention kn_convention; /* default LB_KN_LAMBDA */
    double cfl;                /* off-lattice only: dt = cfl dx / max|xi_x|, 0 < cfl <= 1 (default 1) */
    int isothermal;            /* 1: T = 1 in the equilibrium (default 0: kinetic T) */
    int diag_capacity;         /* records kept in the device ring (default 65536) */
    double storage_scale;      /* 16-bit scale S (rounded to a power of two); 0 = 2 x the initial amplitude */
    int step_kernel;           /* 0: automatic; 1: plain-load step kernel; 2: TMA-staged step kernel;
                                  3: TMA-staged with TMA tensor stores of each tile
                                  (Lax-Wendroff sets: FP32 up to 36 velocities, 16-bit all; nx
                                  a multiple of 4 for FP32, of 8 for 16-bit)
                                  (LB_ERR_UNSUPPORTED if not built for the set or storage).  All
                                  give bitwise-identical populations. */
    void *stream;              /* cudaStream_t to run on; NULL = a stream the handle creates */
    /* optional device allocator (e.g. PyTorch's caching allocator); both or neither */
    void *(*alloc)(void *ctx, size_t bytes, void *stream);
    void (*free)(void *ctx, void *ptr, size_t bytes, void *stream);
    void *alloc_ctx;
    /* body force driving the standing shear wave (Sec. 4, Eq. force, turned so that the
     * flow is along y): g = (0, g_y), g_y(x_i, t) = force_amp sin(x_i) cos(force_freq t).
     * It enters the moments (rho u_y = sum xi_y f~ + rho g_y dt/2, Sec. 2.2) and the
     * collision through the Hermite force term of Sec. 2.1 (Eq. 2order).  Reported
     * u_y, momentum and sigma_xy are those of the forced scheme.  Forced steps run the
     * plain-load kernel (step_kernel 2 is LB_ERR_UNSUPPORTED).  0 (default): free wave. */
    double force_amp;
    double force_freq;
    /* Test facility for the failure detection of the TMA-staged step kernel: 1 = its
     * producer in block 0 withholds the first stage of its first tile, so that block's
     * bounded waits run out (about a second each) and the next synchronising call returns
     * LB_ERR_TIMEOUT; the context stays usable.  0 (default) in normal use. */
    int test_withhold_stage;
    lb_scheme scheme;          /* default LB_SCHEME_SECOND_ORDER */
    lb_streaming streaming;    /* default LB_STREAM_LAX_WENDROFF */
} lb_params;

/* One diagnostics record per time level n (t = n dt), FP64 sums over the grid:
 * mass = sum rho, mom_x/mom_y = sum rho u, amp = 2/(nx ny) sum u_y sin(x_i),
 * shear = 2/(nx ny) sum sigma_xy cos(x_i) with sigma_xy = (1 - omega/2)
 * sum xi_x xi_y (f~ - f^eq) (pressure-tensor sign; factor 1 for LB_SCHEME_FIRST_ORDER),
 * hnorm = sum (f~ - w rho0)^2 / w,
 * x_i = i dx.  flags != 0 marks a non-finite sum. */
typedef struct {
    double t, mass, mom_x, mom_y, amp, shear, hnorm, flags;
} lb_diag;

typedef struct {
    int q;              /* number of velocities */
    int degree;         /* exact polynomial degree of the quadrature */
    int on_lattice;     /* 1: exact shift streaming, 0: Lax-Wendroff */
    int halo;           /* max |e| (on-lattice) or 1 (Lax-Wendroff) */
    double dx, dt, tau, omega;
    double c_lattice;   /* xi = c e for on-lattice sets, else 0 */
    long long time_level;   /* n: the state is f~(n dt) */
    int tma_staged;         /* 1: steps run the TMA-staged kernel, 2: its store-staged variant */
    long long records;      /* diagnostics records produced so far (n + 1 after init) */
    size_t bytes_per_cell_update; /* algorithmic HBM bytes: 2 q sizeof(storage) */
    size_t device_bytes;    /* device memory held by the handle */
    double storage_scale;   /* 16-bit scale S (1 for F32/F64) */
} lb_info_t;

/* Fill *p with defaults (F32, LAMBDA, cfl 1, kinetic T, own stream). */
void lb_params_default(lb_params *p);

/* Create a handle with default parameters.  Host work + device allocation; no launch. */
lb_status lb_create(lb_quadrature q, int n_eq, int nx, int ny, double kn, lb_handle **out);
lb_status lb_create_ex(const lb_params *p, lb_handle **out);

/* Standing shear wave at rest density and temperature (Sec. 4):
 * rho = 1, T = 1, u_x = 0, u_y = u0 sin(x_i) + u1 sin(2 pi j / ny) sin(x_i),
 * f~(0) = f^eq.  Resets time to 0 and records level 0. */
lb_status lb_init_shear_wave(lb_handle *h, double u0, double u1);

/* f~(0) = f^eq(rho, u, T) from caller host arrays of nx*ny doubles, row-major
 * (index j*nx + i); T may be NULL (T = 1).  Resets time to 0. */
lb_status lb_init_fields(lb_handle *h, const double *rho, const double *ux, const double *uy,
                         const double *T);

/* Advance n >= 0 time levels (asynchronous; CUDA-graph replay). */
lb_status lb_step(lb_handle *h, int n);

/* Moments of f~ at the current time level into caller host arrays of nx*ny
 * doubles (any may be NULL).  Synchronises the handle's stream. */
lb_status lb_moments(lb_handle *h, double *rho, double *ux, double *uy, double *T, double *sxy);

/* Same, into caller DEVICE arrays of nx*ny doubles, asynchronous on the stream. */
lb_status lb_moments_device(lb_handle *h, double *rho, double *ux, double *uy, double *T,
                            double *sxy);

/* f~ at the current level as FP64 (full f, not the deviation), q*ny*nx doubles,
 * index (alpha*ny + j)*nx + i, into a caller host array.  Synchronises. */
lb_status lb_populations(lb_handle *h, double *f);

/* Copy the most recent min(records, capacity, max_records) diagnostics records,
 * oldest first, into out; *n_out receives the count.  Synchronises. */
lb_status lb_diagnostics(lb_handle *h, lb_diag *out, int max_records, int *n_out);

/* The record of one time level, without waiting for the levels enqueued after it: waits
 * only until the launch that produced `level` has completed (later levels keep running on
 * the handle's stream), then copies its record into *out (caller host memory) on a stream
 * of the handle's own.  So a loop that enqueues level n + 1 before reading level n keeps
 * the GPU busy.  level in [max(0, current - diag_capacity + 1), current].
 * Errors: LB_ERR_ARG (level outside the ring), LB_ERR_STATE (no init yet), LB_ERR_CUDA,
 * LB_ERR_UNSTABLE (the record's sums are non-finite; *out is written). */
lb_status lb_diagnostics_at(lb_handle *h, long long level, lb_diag *out);

/* Decay rate of the shear-wave amplitude (FP64, host): minus the least-squares
 * slope of ln|A(n)| against t over the diagnostics records with t >= t_start,
 * up to the first record whose |A| falls below floor_rel * |A(0)|.  Needs the
 * records to be still in the ring (capacity).  *rate and *npoints on LB_OK;
 * LB_ERR_ARG when fewer than 3 records qualify.  Also returns, if not NULL,
 * the fitted sigma_xy amplitude ratio: max|S(n)| / |A(0)| over the window. */
lb_status lb_fit_decay(lb_handle *h, double t_start, double floor_rel, double *rate, int *npoints,
                       double *shear_ratio);

/* Wait for the handle's work; reports device-side errors. */
lb_status lb_synchronize(lb_handle *h);

/* Slab decomposition of one periodic grid over several lattices (one per GPU, or several
 * on one GPU): each lattice holds a band of rows of the grid, and its streaming (Sec. 2.3:
 * exact shift by e_a, or the Lax-Wendroff stencil) reads gy rows beyond its own on either
 * side (gy = info.halo rows: 1 for Lax-Wendroff, max|e_y| for the exact shift, 2 for
 * second-order upwind).  Between two levels the caller fills those ghost rows with the
 * neighbours' boundary rows: pack side 0 (rows 0..gy-1) and side 1 (rows ny-gy..ny-1) of
 * this lattice's state into device buffers, move them to the lower and upper neighbour,
 * and unpack what arrives into side 0 (ghost rows -gy..-1) and side 1 (ghost rows
 * ny..ny+gy-1).  The library's own kernels fill the ghost rows with the lattice's own
 * periodic images; an exchange after init and after every lb_step(h, 1) overwrites them,
 * so a lattice stepped one level at a time between exchanges advances its band of the
 * whole grid.  Both calls act on the state the next lb_step reads, are enqueued on the
 * handle's stream (asynchronous; order other streams with events), and copy whole padded
 * rows of every velocity plane, as stored: with 16-bit storage every band must use the same
 * lb_params.storage_scale (the automatic scale follows each band's own initial amplitude).
 * dst / src: device buffers of lb_halo_bytes bytes, owned by
 * the caller.  LB_ERR_STATE before init; LB_ERR_ARG for a side other than 0, 1 or a NULL
 * buffer.  The paper has no slab decomposition; this is the data-parallel split of its
 * grid. */
lb_status lb_halo_bytes(const lb_handle *h, size_t *bytes);
lb_status lb_halo_pack(lb_handle *h, int side, void *dst);
lb_status lb_halo_unpack(lb_handle *h, int side, const void *src);

lb_status lb_get_info(const lb_handle *h, lb_info_t *out);

/* Number of kernels the handle has launched (graph replays count each node). */
long long lb_kernel_launches(const lb_handle *h);

/* NULL-safe. */
lb_status lb_destroy(lb_handle *h);

const char *lb_status_string(lb_status s);
const char *lb_last_error(const lb_handle *h);

/* Host-only: the velocity set the library builds (no device needed).
 * xi: 2q doubles (xi_x, xi_y per velocity), w: q doubles, e: 2q ints or NULL
 * (on-lattice only); pass NULL arrays to query *q and *degree only. */
lb_status lb_quadrature_info(lb_quadrature quad, int *q, int *degree, double *xi, double *w,
                             int *e);

/* ---------------------------------------------------------------------------
 * Batches: many small, uneven shear-wave instances advanced together by one
 * persistent kernel launch per lb_batch_run (CUDA-graph replay).  Slots can be
 * added and removed between runs (continuous batching); admission is by the
 * device-memory budget of the batch arena.  Lax-Wendroff product sets only.
 * Each instance starts from the shear wave u_y = u0 sin(x_i) (rho = T = 1) and
 * records A(n), S(n) (as in lb_diag, summed in FP32) for every level it
 * processes.  The per-cell arithmetic is the single-lattice one (the same
 * collision function): an instance's results are bitwise the same alone or in
 * any mix, and agree with an lb_handle run of the same problem to FP32 rounding.
 * ------------------------------------------------------------------------- */
typedef struct lb_batch lb_batch;

typedef struct {
    lb_quadrature quadrature; /* LB_D2Q16_GH, LB_D2Q36_GH or LB_D2Q64_GH */
    int n_eq;                 /* 2..4 (degree >= N + 2) */
    int nx, ny;               /* nx >= 2, ny >= 1 */
    double kn;                /* Knudsen number, the batch's kn_convention */
    double u0;                /* shear-wave amplitude */
    int max_steps;            /* last time level to process (levels 0..max_steps) */
    double stop_ratio;        /* stop at the first level n > 0 with sqrt(H(n)/H(0)) <= stop_ratio (0: never) */
} lb_instance_desc;

typedef struct {
    lb_precision precision;   /* LB_F32 (default), LB_F16 or LB_BF16 deviation storage */
    lb_kn_convention kn_convention;
    size_t budget_bytes;      /* device arena for populations, histories, tables (default 1 GiB) */
    int max_slots;            /* default 4096 */
    int threads;              /* threads per CTA (64..256, multiple of 32); 0 = 256 */
    int smem_bytes;           /* on-chip instance budget per CTA (bytes); -1 = 96 KiB */
    void *stream;             /* cudaStream_t; NULL = own stream */
    int warp_cells;           /* instances of at most this many cells are each advanced by one
                                 warp (a CTA then advances threads/32 of them at once, each with
                                 its share of the on-chip budget); larger ones by a whole CTA.
                                 0 = every instance by a CTA; -1 (default) = 512 */
} lb_batch_params;

typedef struct {
    int level;                /* levels processed: records 0..level-1 exist */
    int done;                 /* 1: finished (stop rule, max_steps or non-finite) */
    int status;               /* bit 0: non-finite state */
    int q;
    double dt, omega, tau;
    size_t bytes;             /* arena bytes held by the slot */
} lb_instance_state;

void lb_batch_params_default(lb_batch_params *p);
lb_status lb_batch_create(const lb_batch_params *p, lb_batch **out);
/* Admit one instance; *slot receives its id.  LB_ERR_BUDGET if the arena has no room. */
lb_status lb_batch_add(lb_batch *b, const lb_instance_desc *d, int *slot);
/* Release a slot (its arena memory is reusable by the next add). */
lb_status lb_batch_remove(lb_batch *b, int slot);
/* One launch: every live, unfinished slot advances by up to `chunk` levels
 * (0 = until it finishes).  Asynchronous on the batch stream. */
lb_status lb_batch_run(lb_batch *b, int chunk);
/* Wait for the batch stream and refresh the host view of every slot. */
lb_status lb_batch_sync(lb_batch *b);
lb_status lb_batch_state(lb_batch *b, int slot, lb_instance_state *out);
/* A(n), S(n) of levels 0..min(level, max)-1 into caller host arrays (either may be NULL). */
lb_status lb_batch_history(lb_batch *b, int slot, double *amp, double *shear, int max, int *n_out);
/* FP64 decay-rate fit of a slot's history (same rule as lb_fit_decay). */
lb_status lb_batch_fit(lb_batch *b, int slot, double t_start, double floor_rel, double *rate, int *npoints);
size_t lb_batch_bytes_in_use(const lb_batch *b);
long long lb_batch_kernel_launches(const lb_batch *b);
/* Timing of the last completed batch launch (waits for it): *span_s, the time from the first
 * CTA's start to the last CTA's end; *tail_s, the time the last CTA ran after every other CTA
 * had finished (the launch's tail: one instance that no other CTA can share); *ctas, the CTAs
 * that ran.  Any pointer may be NULL.  LB_ERR_STATE before the first launch.  The paper has
 * no batching; this measures the persistent multi-instance launch. */
lb_status lb_batch_run_profile(lb_batch *b, double *span_s, double *tail_s, int *ctas);
lb_status lb_batch_destroy(lb_batch *b);
const char *lb_batch_last_error(const lb_batch *b);

/* ---------------------------------------------------------------------------
 * Discrete velocity method of Sec. 3.3: the reduced linearised BGK equation of the
 * free standing shear wave (Eqs. LBGK, ga, gb, force zero),
 *   dG/dt + xi_k dG/dx = (u - G)/tau,  u = sum_k w_k G_k,
 * at the nodes xi_k of the n_nodes-point Gauss-Hermite rule, started from G = u0 sin x.
 * Strang splitting of the exact relaxation around one Lax-Wendroff step,
 * dt = cfl dx / max|xi_k|, dx = 2 pi / nx, FP64 on the GPU, one CTA per collision
 * time.  For the same-quadrature cross-check of the lattice runs (Sec. 3.2).
 *   tau          n_inst collision times (host array)
 *   amp, shear   caller host arrays of n_inst x (nsteps + 1) doubles: A(n) and S(n)
 *                (as in lb_diag, sigma = sum_k w_k xi_k G) of instance i at [i*(nsteps+1) + n]
 *   stream       cudaStream_t (NULL = default); returns after the run.
 * Errors: LB_ERR_ARG; LB_ERR_UNSUPPORTED if n_nodes x nx does not fit one CTA's shared
 * memory (8 (n_nodes + 2) nx bytes); LB_ERR_NOMEM; LB_ERR_CUDA (lb_last_error(NULL)).
 * ------------------------------------------------------------------------- */
lb_status lb_dvm_run(int n_inst, const double *tau, int n_nodes, int nx, double cfl, double u0,
                     int nsteps, double *amp, double *shear, void *stream);

/* The same DVM driven by the body force of the standing shear wave (Sec. 4, Eq. force,
 * turned so that the flow is along y): g(x, t) = force_amp sin(x_i) cos(force_freq t).
 * The reduced function of Eq. ga stays zero, so the force term of Eq. gb is g:
 *   dG/dt + xi_k dG/dx = (u - G)/tau + g.
 * The relaxation half steps integrate relaxation and force exactly (u gains the time
 * integral of g, G - u decays by exp(-dt / (2 tau))).  Arguments, results and errors as
 * lb_dvm_run (LB_ERR_ARG also for a non-finite force_amp or force_freq); force_amp = 0
 * is lb_dvm_run. */
lb_status lb_dvm_run_forced(int n_inst, const double *tau, int n_nodes, int nx, double cfl, double u0,
                            double force_amp, double force_freq, int nsteps, double *amp, double *shear,
                            void *stream);

/* ---------------------------------------------------------------------------
 * Allocation-free solve of one small shear wave.  The paper has no
 * counterpart: this is an engineering entry point for callers that cannot
 * allocate device memory, e.g. a process whose free device memory is already
 * claimed by another allocator (a framework's caching allocator, a fixed
 * per-process budget), so that cudaMalloc would fail, or a latency-critical
 * loop that must not call cudaMalloc/cudaFree because they can synchronise the
 * device.  It allocates nothing (no cudaMalloc, cudaFree or allocating library
 * routine): all device state of the solve (instance descriptor, work-queue
 * counter, sin/cos table, history, both population buffers) lives in one
 * fixed __device__ array of LB_STATIC_SCRATCH_BYTES per device.  CUDA loads
 * device code lazily by default, so the array is reserved by the first call
 * on a device: make that call early (at start-up, while the memory is free).
 *
 * The instance is the lb_batch one (same desc, same kernel, same constants):
 * it runs from level 0 until the stop rule or max_steps, and its history is
 * that of the same desc run in an lb_batch with default launch shape.
 *   desc        Gauss-Hermite product set, n_eq 2..4, grid, kn, u0, max_steps, stop_ratio
 *   precision   LB_F32, LB_F16 or LB_BF16 deviation storage (FP32 arithmetic)
 *   history     caller host array of 2 max_records floats, or NULL if max_records = 0:
 *               (A(n), S(n)) interleaved for levels 0..min(level, max_records)-1
 *   state       optional; level, done, status, q, dt, omega, tau, and in `bytes`
 *               the scratch bytes the solve used
 *   stream      cudaStream_t to run on (NULL = the default stream); the call
 *               returns after the solve has finished.
 * Needs: 512 + 8 nx + 8 (max_steps + 1) + 2 q nx ny sizeof(storage) bytes
 * (each term rounded up to 256); a larger solve returns LB_ERR_BUDGET with the
 * sizes in lb_last_error(NULL), before any device work.  Errors: LB_ERR_ARG,
 * LB_ERR_UNSUPPORTED, LB_ERR_CUDA, LB_ERR_UNSTABLE (non-finite state; history
 * and state are not written); messages in lb_last_error(NULL).
 *
 * First call on each device: one-time set-up with that device current (the
 * scratch's device address via cudaGetSymbolAddress, the velocity-set tables,
 * the kernel's shared-memory attribute).  Make that first call before any
 * stream capture begins on the device.
 *
 * The scratch is one array per device shared by every call on that device:
 * calls that overlap in time (from several host threads, on any streams)
 * race on it and return wrong results.  Serialise them.
 * ------------------------------------------------------------------------- */
#define LB_STATIC_SCRATCH_BYTES (8u << 20)

lb_status lb_solve_static(const lb_instance_desc *desc, lb_precision precision,
                          lb_kn_convention kn_convention, float *history, int max_records,
                          lb_instance_state *state, void *stream);

/* ---------------------------------------------------------------------------
 * Serving: a request loop over batches.  Requests (shear-wave solves) are
 * queued as they arrive; each lb_server_step admits queued requests while the
 * device-memory budget allows, advances every admitted request by one chunk of
 * levels (small requests as slots of one continuously batched persistent
 * launch, large ones as lattices of their own on a second stream, so the two
 * kinds overlap on the device), and retires the finished ones with their FP64
 * decay-rate fit.  Finished requests are collected with lb_server_poll.
 * ------------------------------------------------------------------------- */
typedef struct lb_server lb_server;

typedef struct {
    lb_batch_params batch;     /* small requests (precision applies to both lanes) */
    int chunk;                 /* levels per step (default 200) */
    long long large_cells;     /* requests with nx*ny >= large_cells run as lattices (default 65536) */
    size_t budget_bytes;       /* device bytes for large requests (default 8 GiB) */
    int max_large;             /* concurrent large requests (default 4) */
} lb_server_params;

typedef struct {
    long long id;
    double arrival;            /* caller's clock, seconds */
    lb_instance_desc desc;
} lb_request;

typedef struct {
    long long id;
    double arrival, admitted, finished; /* caller's clock at submit, at admission, at retirement */
    int levels;                /* levels processed */
    int status;                /* lb_status of the solve */
    double decay_rate;         /* FP64 fit of ln|A(n)| (0 if the window had < 3 points) */
    int fit_points;
    double shear_amp;          /* max |S(n)| / |A(0)| over the history */
} lb_response;

void lb_server_params_default(lb_server_params *p);
lb_status lb_server_create(const lb_server_params *p, lb_server **out);
/* Queue a request; `now` is the caller's clock (seconds). */
lb_status lb_server_submit(lb_server *s, const lb_request *r);
/* One scheduling iteration at caller time `now`: admit, advance one chunk, retire.
 * *active receives the number of admitted requests still running, *queued the
 * number waiting. */
lb_status lb_server_step(lb_server *s, double now, int *active, int *queued);
/* Move up to max finished responses to out; *n_out receives the count. */
lb_status lb_server_poll(lb_server *s, lb_response *out, int max, int *n_out);
/* A(n), S(n) of a finished request into caller host arrays (either may be NULL);
 * the server keeps a history until it is fetched once. */
lb_status lb_server_history(lb_server *s, long long id, double *amp, double *shear, int max, int *n_out);
lb_status lb_server_destroy(lb_server *s);
const char *lb_server_last_error(const lb_server *s);

#ifdef __cplusplus
}
#endif

#endif /* LB_H */
