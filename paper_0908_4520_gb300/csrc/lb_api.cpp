// C-ABI of liblb.so: handles, device memory, step constants, CUDA-graph
// stepping, moments and diagnostics read-back.  Every compute step runs in
// the kernels of lb_kernels.cuh; this file only marshals.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "lb.h"
#include "lb_device.h"
#include "lb_host.h"

namespace lbk {

namespace {
struct Registry {
    std::mutex mu;
    LaunchFn fn[16][4] = {};
};
Registry& registry() {
    static Registry r;
    return r;
}
}  // namespace

bool register_launcher(int quadrature, int precision, LaunchFn fn) {
    if (quadrature < 0 || quadrature >= 16 || precision < 0 || precision >= 4) return false;
    Registry& r = registry();
    std::lock_guard<std::mutex> g(r.mu);
    r.fn[quadrature][precision] = fn;
    return true;
}

LaunchFn find_launcher(int quadrature, int precision) {
    if (quadrature < 0 || quadrature >= 16 || precision < 0 || precision >= 4) return nullptr;
    Registry& r = registry();
    std::lock_guard<std::mutex> g(r.mu);
    return r.fn[quadrature][precision];
}

}  // namespace lbk

// extra elements per row (a multiple of 16 keeps every row 64-byte aligned); tuning knob
#ifndef LB_PITCH_PAD
#define LB_PITCH_PAD 32  // measured: +3 % for the exact-shift sets at 4096^2, neutral elsewhere
#endif

namespace {

using LaunchFn = lbk::LaunchFn;

thread_local std::string g_create_error;

size_t storage_bytes(lb_precision p) {
    switch (p) {
        case LB_F64: return 8;
        case LB_BF16:
        case LB_F16: return 2;
        default: return 4;
    }
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda)
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(ptr);
    });
    return fn;
}

int sm_count() {
    static int n = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            n = 0;
    });
    return n;
}

}  // namespace

struct lb_handle {
    lb_params p{};
    lbh::VelocitySetInfo vs;
    LaunchFn launch = nullptr;
    lbk::Shape shape{};
    int pitch = 0, gy = 0, ntiles_x = 0, ntiles = 0, x0_last = 0, grid = 0, grid_init = 0;
    bool use_tma = false;
    int tma_ntiles_x = 0, tma_ntiles = 0, tma_x0_last = 0, tma_grid = 0;
    CUtensorMap tmap[2];
    // store-staged TMA step kernel: its tiles, load maps (its box) and store maps (the cells of
    // each buffer as a destination)
    bool use_st = false;
    int st_ntiles_x = 0, st_ntiles = 0, st_grid = 0;
    CUtensorMap tmap_stl[2], tmap_out[2];
    long long plane = 0, origin = 0, ncell = 0;
    size_t pop_bytes = 0, device_bytes = 0;
    double dx = 0, dt = 0, tau = 0, omega = 0, scale = 1.0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void* buf[2] = {nullptr, nullptr};
    int cur = 0;
    bool raw_prev = true, initialized = false;
    long long level = 0, launches = 0;
    void* sin_d = nullptr;
    void* cos_d = nullptr;
    double* partials = nullptr;
    unsigned int* ticket = nullptr;
    long long* level_d = nullptr;
    lb_diag* ring = nullptr;
    int* status = nullptr;
    double* mom = nullptr;   // 5 * ncell scratch for lb_moments
    double* pop = nullptr;   // q * ncell scratch for lb_populations
    cudaGraphExec_t chunk[2] = {nullptr, nullptr};
    cudaGraphExec_t pair[2] = {nullptr, nullptr};
    cudaGraphExec_t single[2] = {nullptr, nullptr};  // one level (parameters uploaded once)
    // completion markers of the enqueued levels: ev[i] follows the launch that produced
    // level ev_level[i] (lb_diagnostics_at waits on the first marker at or past a level)
    static constexpr int kMarks = 8;
    cudaEvent_t ev[kMarks] = {};
    long long ev_level[kMarks] = {-1, -1, -1, -1, -1, -1, -1, -1};
    int ev_next = 0;
    cudaStream_t copy_stream = nullptr;  // record read-back beside the running levels
    std::vector<std::pair<void*, size_t>> allocs;
    std::string err;

    lb_status mark_level() {
        if (!ev[ev_next]) {
            const cudaError_t e = cudaEventCreateWithFlags(&ev[ev_next], cudaEventDisableTiming);
            if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
        }
        const cudaError_t e = cudaEventRecord(ev[ev_next], stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        ev_level[ev_next] = level;
        ev_next = (ev_next + 1) % kMarks;
        return LB_OK;
    }

    lb_status fail(lb_status s, const std::string& m) {
        err = m;
        return s;
    }
    lb_status cuda_fail(cudaError_t e, const char* where) {
        err = std::string(where) + ": " + cudaGetErrorString(e);
        return LB_ERR_CUDA;
    }
    void* dalloc(size_t bytes) {
        void* ptr = nullptr;
        if (p.alloc) {
            ptr = p.alloc(p.alloc_ctx, bytes, stream);
        } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
            ptr = nullptr;
        }
        if (ptr) {
            allocs.push_back({ptr, bytes});
            device_bytes += bytes;
        }
        return ptr;
    }
    void release() {
        for (int i = 0; i < kMarks; ++i) {
            if (ev[i]) cudaEventDestroy(ev[i]);
            ev[i] = nullptr;
            ev_level[i] = -1;
        }
        if (copy_stream) cudaStreamDestroy(copy_stream);
        copy_stream = nullptr;
        for (int i = 0; i < 2; ++i) {
            if (chunk[i]) cudaGraphExecDestroy(chunk[i]);
            if (pair[i]) cudaGraphExecDestroy(pair[i]);
            if (single[i]) cudaGraphExecDestroy(single[i]);
            chunk[i] = pair[i] = single[i] = nullptr;
        }
        if (stream) cudaStreamSynchronize(stream);
        for (auto& a : allocs) {
            if (p.free) p.free(p.alloc_ctx, a.first, a.second, stream);
            else cudaFree(a.first);
        }
        allocs.clear();
        if (own_stream && stream) cudaStreamDestroy(stream);
        stream = nullptr;
    }

    // tiling: 0 the plain-load kernel's, 1 the TMA-staged kernel's, 2 the store-staged kernel's
    template <class R>
    void fill_args(lbk::Args<R>& A, int tiling) const {
        std::memset(&A, 0, sizeof(A));
        A.plane = plane;
        A.origin = origin;
        A.nx = p.nx;
        A.ny = p.ny;
        A.pitch = pitch;
        A.gy = gy;
        A.ntiles_x = tiling == 2 ? st_ntiles_x : tiling == 1 ? tma_ntiles_x : ntiles_x;
        A.ntiles = tiling == 2 ? st_ntiles : tiling == 1 ? tma_ntiles : ntiles;
        A.x0_last = tiling == 2 ? 0 : tiling == 1 ? tma_x0_last : x0_last;
        A.isothermal = p.isothermal;
        A.diag_every = 1;
        const double om = std::is_same<R, float>::value ? lbh::snap_unit(omega) : omega;
        A.omega = (R)om;
        A.rho0 = (R)1.0;
        const bool first = p.scheme == LB_SCHEME_FIRST_ORDER;
        A.sigma_fac = (R)(first ? 1.0 : 1.0 - 0.5 * om);
        A.tau = (R)tau;
        A.hdt = (R)(first ? 0.0 : 0.5 * dt);
        A.dt = dt;
        A.force_amp = p.force_amp;
        A.force_freq = p.force_freq;
        A.withhold_stage = p.test_withhold_stage;
        A.sinx = static_cast<const R*>(sin_d);
        A.cosx = static_cast<const R*>(cos_d);
        A.partials = partials;
        A.ticket = ticket;
        A.level = level_d;
        A.ring = ring;
        A.ring_cap = p.diag_capacity;
        A.status = status;
        // the kernel tables (and the relaxation tables of this omega), built once per storage scale
        if (tab_scale != scale) {
            lbh::build_tab<float>(vs, dt, dx, scale, tab_f);
            lbh::build_relax<float>(vs, (float)lbh::snap_unit(omega), tab_f);
            lbh::build_tab<double>(vs, dt, dx, scale, tab_d);
            lbh::build_relax<double>(vs, omega, tab_d);
            tab_scale = scale;
        }
        if constexpr (std::is_same<R, float>::value) {
            A.tab = tab_f;
        } else {
            A.tab = tab_d;
        }
    }
    mutable lbk::Tab<float> tab_f;
    mutable lbk::Tab<double> tab_d;
    mutable double tab_scale = -1.0;

};

namespace {

template <class R>
lb_status launch_with(lb_handle* h, int kind, const void* src, void* dst, int raw, int grid,
                      double* o_rho, double* o_ux, double* o_uy, double* o_T, double* o_sxy, double* o_pop,
                      double u0, double u1, const double* i_rho, const double* i_ux, const double* i_uy,
                      const double* i_T) {
    lbk::Args<R> A;
    const bool tma = (kind == lbk::kStepTma || kind == lbk::kMomentsTma);
    const bool st = kind == lbk::kStepTmaStore;
    h->fill_args(A, st ? 2 : tma ? 1 : 0);
    if (tma) A.tmap = h->tmap[src == h->buf[0] ? 0 : 1];
    if (st) {
        A.tmap = h->tmap_stl[src == h->buf[0] ? 0 : 1];
        A.tmap_st = h->tmap_out[dst == h->buf[0] ? 0 : 1];
    }
    A.src = src;
    A.dst = dst;
    A.raw = raw;
    A.o_rho = o_rho;
    A.o_ux = o_ux;
    A.o_uy = o_uy;
    A.o_T = o_T;
    A.o_sxy = o_sxy;
    A.o_pop = o_pop;
    A.u0 = u0;
    A.u1 = u1;
    A.i_rho = i_rho;
    A.i_ux = i_ux;
    A.i_uy = i_uy;
    A.i_T = i_T;
    lbk::Launch L;
    L.kind = kind;
    L.n_eq = h->p.n_eq;
    L.upwind = h->p.streaming == LB_STREAM_UPWIND2;
    L.grid = grid;
    L.stream = h->stream;
    L.args = &A;
    const cudaError_t e = h->launch(L);
    if (e != cudaSuccess) return h->cuda_fail(e, "kernel launch");
    ++h->launches;
    return LB_OK;
}

lb_status launch_any(lb_handle* h, int kind, const void* src, void* dst, int raw, int grid,
                     double* o_rho = nullptr, double* o_ux = nullptr, double* o_uy = nullptr,
                     double* o_T = nullptr, double* o_sxy = nullptr, double* o_pop = nullptr,
                     double u0 = 0, double u1 = 0, const double* i_rho = nullptr,
                     const double* i_ux = nullptr, const double* i_uy = nullptr,
                     const double* i_T = nullptr) {
    if (h->p.precision == LB_F64)
        return launch_with<double>(h, kind, src, dst, raw, grid, o_rho, o_ux, o_uy, o_T, o_sxy, o_pop, u0, u1,
                                   i_rho, i_ux, i_uy, i_T);
    return launch_with<float>(h, kind, src, dst, raw, grid, o_rho, o_ux, o_uy, o_T, o_sxy, o_pop, u0, u1, i_rho,
                              i_ux, i_uy, i_T);
}

// One step launch: level n -> n+1 (src = buf[cur] holds f*(n-1), dst gets f*(n)).
lb_status step_once(lb_handle* h, int from) {
    if (h->p.force_amp != 0.0)  // the forced step runs the plain-load kernel
        return launch_any(h, lbk::kStepForced, h->buf[from], h->buf[1 - from], 0, h->grid);
    if (h->use_st) return launch_any(h, lbk::kStepTmaStore, h->buf[from], h->buf[1 - from], 0, h->st_grid);
    if (h->use_tma) return launch_any(h, lbk::kStepTma, h->buf[from], h->buf[1 - from], 0, h->tma_grid);
    return launch_any(h, lbk::kStep, h->buf[from], h->buf[1 - from], 0, h->grid);
}

lb_status encode_maps(lb_handle* h) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return h->fail(LB_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    CUtensorMapDataType dt;
    switch (h->p.precision) {
        case LB_F32: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; break;
        case LB_BF16: dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; break;
        case LB_F16: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT16; break;
        default: return h->fail(LB_ERR_UNSUPPORTED, "TMA staging is built for 32- and 16-bit storage");
    }
    const size_t b = storage_bytes(h->p.precision);
    const cuuint64_t dims[3] = {(cuuint64_t)h->pitch, (cuuint64_t)(h->p.ny + 2 * h->gy), (cuuint64_t)h->vs.q};
    const cuuint64_t strides[2] = {(cuuint64_t)h->pitch * b, (cuuint64_t)h->plane * b};
    const cuuint32_t box[3] = {(cuuint32_t)h->shape.box_w, (cuuint32_t)h->shape.box_h, (cuuint32_t)h->shape.box_d};
    const cuuint32_t estr[3] = {1, 1, 1};
    for (int i = 0; i < 2; ++i) {
        const CUresult r = enc(&h->tmap[i], dt, 3, h->buf[i], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return h->fail(LB_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    }
    if (h->use_st) {
        // loads: the whole padded buffer, the store-staged kernel's box; stores: the nx x ny
        // cells of each buffer (the rim is written by the kernel's own image stores), one
        // tile of all q velocities per store
        const cuuint32_t lbox[3] = {(cuuint32_t)h->shape.st_box_w, (cuuint32_t)h->shape.st_box_h,
                                    (cuuint32_t)h->shape.box_d};
        const cuuint64_t odims[3] = {(cuuint64_t)h->p.nx, (cuuint64_t)h->p.ny, (cuuint64_t)h->vs.q};
        const cuuint32_t obox[3] = {(cuuint32_t)h->shape.st_tw, (cuuint32_t)h->shape.st_rows, (cuuint32_t)h->vs.q};
        for (int i = 0; i < 2; ++i) {
            CUresult r = enc(&h->tmap_stl[i], dt, 3, h->buf[i], dims, strides, lbox, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r == CUDA_SUCCESS) {
                void* cells = static_cast<char*>(h->buf[i]) + h->origin * (long long)b;
                r = enc(&h->tmap_out[i], dt, 3, cells, odims, strides, obox, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            }
            if (r != CUDA_SUCCESS)
                return h->fail(LB_ERR_CUDA, "cuTensorMapEncodeTiled (store-staged) failed: " + std::to_string((int)r));
        }
    }
    return LB_OK;
}

lb_status build_graph(lb_handle* h, int from, int nsteps, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return h->cuda_fail(e, "cudaStreamBeginCapture");
    const long long before = h->launches;
    lb_status st = LB_OK;
    int b = from;
    for (int i = 0; i < nsteps && st == LB_OK; ++i) {
        st = step_once(h, b);
        b = 1 - b;
    }
    e = cudaStreamEndCapture(h->stream, &g);
    h->launches = before;  // captured launches are counted at replay
    if (st != LB_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return h->cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return h->cuda_fail(e, "cudaGraphInstantiate");
    return LB_OK;
}

constexpr int kChunk = 32;

// 16-bit storage takes its scale from the initial amplitude (unless storage_scale is set)
bool scale_from_amplitude(const lb_handle* h) {
    return (h->p.precision == LB_BF16 || h->p.precision == LB_F16) && !(h->p.storage_scale > 0);
}

lb_status set_scale_and_tables(lb_handle* h, double amp) {
    double scale = 1.0;
    if (h->p.precision == LB_BF16 || h->p.precision == LB_F16) {
        double s = h->p.storage_scale;
        if (s <= 0) s = std::max(2.0 * amp, 1e-6);
        scale = lbh::pow2_near(s);
    }
    // graphs bake the tables into their kernel parameters: rebuild when the scale changes
    if (scale == h->scale && (h->chunk[0] || h->pair[0] || h->single[0] || h->chunk[1] || h->pair[1] ||
                              h->single[1]))
        return LB_OK;
    h->scale = scale;
    for (int i = 0; i < 2; ++i) {
        if (h->chunk[i]) cudaGraphExecDestroy(h->chunk[i]);
        if (h->pair[i]) cudaGraphExecDestroy(h->pair[i]);
        if (h->single[i]) cudaGraphExecDestroy(h->single[i]);
        h->chunk[i] = h->pair[i] = h->single[i] = nullptr;
    }
    return LB_OK;
}

lb_status init_common(lb_handle* h, double u0, double u1, const double* d_rho, const double* d_ux,
                      const double* d_uy, const double* d_T) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(h->level_d, 0, sizeof(long long), h->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(h->ticket, 0, sizeof(unsigned int), h->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(h->status, 0, sizeof(int), h->stream)) != cudaSuccess)
        return h->cuda_fail(e, "cudaMemsetAsync");
    lb_status st = launch_any(h, lbk::kInit, nullptr, h->buf[1], 0, h->grid_init, nullptr, nullptr, nullptr,
                              nullptr, nullptr, nullptr, u0, u1, d_rho, d_ux, d_uy, d_T);
    if (st != LB_OK) return st;
    // level 0: collide f~(0) (no streaming) -> f*(0) in buf[0], record 0
    st = launch_any(h, h->p.force_amp != 0.0 ? lbk::kStepForced : lbk::kStep, h->buf[1], h->buf[0], 1, h->grid);
    if (st != LB_OK) return st;
    h->cur = 0;
    h->raw_prev = true;
    h->level = 0;
    h->initialized = true;
    for (long long& l : h->ev_level) l = -1;  // markers of the previous run are stale
    return h->mark_level();
}

}  // namespace

void lbh::set_last_error(const std::string& m) { g_create_error = m; }

extern "C" {

void lb_params_default(lb_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->quadrature = LB_D2Q16_GH;
    p->n_eq = 2;
    p->nx = 64;
    p->ny = 1;
    p->kn = 0.1;
    p->precision = LB_F32;
    p->kn_convention = LB_KN_LAMBDA;
    p->cfl = 1.0;
    p->isothermal = 0;
    p->diag_capacity = 65536;
    p->storage_scale = 0.0;
    p->step_kernel = 0;
    p->force_amp = 0.0;
    p->force_freq = 0.0;
    p->test_withhold_stage = 0;
    p->scheme = LB_SCHEME_SECOND_ORDER;
    p->streaming = LB_STREAM_LAX_WENDROFF;
}

const char* lb_status_string(lb_status s) {
    switch (s) {
        case LB_OK: return "ok";
        case LB_ERR_ARG: return "invalid argument";
        case LB_ERR_UNSUPPORTED: return "unsupported";
        case LB_ERR_NOMEM: return "out of memory";
        case LB_ERR_CUDA: return "CUDA error";
        case LB_ERR_UNSTABLE: return "non-finite state";
        case LB_ERR_TIMEOUT: return "device wait timed out";
        case LB_ERR_BUDGET: return "over device-memory budget";
        case LB_ERR_STATE: return "call out of order";
        default: return "unknown status";
    }
}

const char* lb_last_error(const lb_handle* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

lb_status lb_quadrature_info(lb_quadrature quad, int* q, int* degree, double* xi, double* w, int* e) {
    lbh::VelocitySetInfo vs;
    std::string err;
    if (!lbh::build_velocity_set(quad, &vs, &err)) {
        g_create_error = err;
        return LB_ERR_ARG;
    }
    if (q) *q = vs.q;
    if (degree) *degree = vs.degree;
    if (xi) std::copy(vs.xi.begin(), vs.xi.end(), xi);
    if (w) std::copy(vs.w.begin(), vs.w.end(), w);
    if (e) {
        if (!vs.on_lattice) return LB_ERR_ARG;
        for (int a = 0; a < vs.q; ++a) {
            e[2 * a] = vs.ex[a];
            e[2 * a + 1] = vs.ey[a];
        }
    }
    return LB_OK;
}

lb_status lb_create(lb_quadrature q, int n_eq, int nx, int ny, double kn, lb_handle** out) {
    lb_params p;
    lb_params_default(&p);
    p.quadrature = q;
    p.n_eq = n_eq;
    p.nx = nx;
    p.ny = ny;
    p.kn = kn;
    return lb_create_ex(&p, out);
}

lb_status lb_create_ex(const lb_params* pin, lb_handle** out) {
    if (!pin || !out) {
        g_create_error = "null argument";
        return LB_ERR_ARG;
    }
    const lb_params& P = *pin;
    auto reject = [](lb_status s, const std::string& m) {
        g_create_error = m;
        return s;
    };
    if (P.nx < 2 || (P.nx & 1)) return reject(LB_ERR_ARG, "nx must be even and >= 2");
    if (P.ny < 1) return reject(LB_ERR_ARG, "ny must be >= 1");
    if ((long long)P.nx * P.ny > (1LL << 31) - 1) return reject(LB_ERR_ARG, "grid too large");
    if (P.n_eq < 1 || P.n_eq > 4) return reject(LB_ERR_ARG, "n_eq must be 1, 2, 3 or 4");
    if (P.scheme != LB_SCHEME_SECOND_ORDER && P.scheme != LB_SCHEME_FIRST_ORDER)
        return reject(LB_ERR_ARG, "unknown scheme");
    if (P.streaming != LB_STREAM_LAX_WENDROFF && P.streaming != LB_STREAM_UPWIND2)
        return reject(LB_ERR_ARG, "unknown streaming");
    const bool upwind = P.streaming == LB_STREAM_UPWIND2;
    if (upwind && (P.precision == LB_BF16 || P.precision == LB_F16))
        return reject(LB_ERR_UNSUPPORTED, "second-order upwind streaming is built for F32/F64 storage");
    if (!(P.kn > 0) || !std::isfinite(P.kn)) return reject(LB_ERR_ARG, "kn must be positive");
    if (!(P.cfl > 0 && P.cfl <= 1.0)) return reject(LB_ERR_ARG, "cfl must be in (0, 1]");
    if (P.diag_capacity < 1) return reject(LB_ERR_ARG, "diag_capacity must be >= 1");
    if ((P.alloc == nullptr) != (P.free == nullptr)) return reject(LB_ERR_ARG, "alloc and free go together");
    if (P.kn_convention != LB_KN_LAMBDA && P.kn_convention != LB_KN_PAPER)
        return reject(LB_ERR_ARG, "unknown kn_convention");
    if (P.step_kernel < 0 || P.step_kernel > 3) return reject(LB_ERR_ARG, "step_kernel must be 0, 1, 2 or 3");
    if (!std::isfinite(P.force_amp) || !std::isfinite(P.force_freq))
        return reject(LB_ERR_ARG, "force_amp and force_freq must be finite");

    lb_handle* h = new (std::nothrow) lb_handle();
    if (!h) return reject(LB_ERR_NOMEM, "host allocation");
    h->p = P;
    std::string err;
    if (!lbh::build_velocity_set(P.quadrature, &h->vs, &err)) {
        delete h;
        return reject(LB_ERR_ARG, err);
    }
    if (h->vs.degree < P.n_eq + 2) {
        delete h;
        return reject(LB_ERR_UNSUPPORTED, "quadrature degree < N + 2: rho, u and T would not be conserved");
    }
    h->launch = lbk::find_launcher(P.quadrature, P.precision);
    if (!h->launch) {
        delete h;
        return reject(LB_ERR_UNSUPPORTED, (P.precision == LB_BF16 || P.precision == LB_F16)
                                              ? "16-bit storage is built for the Gauss-Hermite product sets only"
                                              : "this (quadrature, precision) unit is not in the build");
    }
    if (upwind && h->vs.on_lattice) {
        delete h;
        return reject(LB_ERR_ARG, "on-lattice sets stream by the exact shift; upwind streaming is for the "
                                  "Gauss-Hermite product sets");
    }
    if (upwind) {  // the kernel takes the upstream side from the node's index: ascending, symmetric nodes
        for (int i = 0; i < h->vs.na; ++i)
            if ((h->vs.axis[i] < 0) != (i < h->vs.na / 2)) {
                delete h;
                return reject(LB_ERR_UNSUPPORTED, "axis nodes not in ascending symmetric order");
            }
    }
    h->dx = 2.0 * M_PI / P.nx;
    double amax = 0;
    for (double a : h->vs.axis) amax = std::max(amax, std::fabs(a));
    h->dt = h->vs.on_lattice ? h->dx / h->vs.c : P.cfl * h->dx / amax;
    h->tau = (P.kn_convention == LB_KN_LAMBDA) ? P.kn * std::sqrt(2.0 / M_PI) : P.kn;
    if (P.scheme == LB_SCHEME_FIRST_ORDER) {
        // Eq. slb: omega = dt / tau, linearly unstable for omega >= 2
        if (!(h->tau > 0.5 * h->dt)) {
            delete h;
            return reject(LB_ERR_ARG, "the first-order scheme needs tau > dt/2 (omega = dt/tau < 2)");
        }
        h->omega = h->dt / h->tau;
    } else {
        h->omega = h->dt / (h->tau + 0.5 * h->dt);
    }
    {
        lbk::Launch L{};
        L.kind = lbk::kQueryShape;
        L.n_eq = P.n_eq;
        L.upwind = upwind;  // the TMA-staged kernel (and box) of this streaming
        L.args = &h->shape;
        if (h->launch(L) != cudaSuccess) {
            h->shape.V = 1;
            h->shape.rows = 8;
            h->shape.threads = 256;
            h->shape.occupancy = 0;
        }
    }
    const int tw = 32 * h->shape.V;
    h->gy = upwind ? std::max(h->vs.halo, 2) : h->vs.halo;  // upwind: two upstream rows
    h->pitch = (P.nx + 2 * lbk::kGhostX + 63) / 64 * 64 + LB_PITCH_PAD;
    h->plane = (long long)h->pitch * (P.ny + 2 * h->gy);
    h->origin = (long long)h->gy * h->pitch + lbk::kGhostX;
    h->ncell = (long long)P.nx * P.ny;
    h->ntiles_x = (P.nx + tw - 1) / tw;
    h->x0_last = P.nx >= tw ? P.nx - tw : 0;
    h->ntiles = h->ntiles_x * ((P.ny + h->shape.rows - 1) / h->shape.rows);
    h->pop_bytes = (size_t)h->vs.q * h->plane * storage_bytes(P.precision);

    cudaError_t e;
    if (P.stream) {
        h->stream = static_cast<cudaStream_t>(P.stream);
    } else {
        if ((e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking)) != cudaSuccess) {
            delete h;
            return reject(LB_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
        }
        h->own_stream = true;
    }
    const int nsm = sm_count();
    if (nsm <= 0) {
        h->release();
        delete h;
        return reject(LB_ERR_CUDA, "no CUDA device");
    }
    const int occ = std::max(1, h->shape.occupancy);
    if (P.force_amp != 0.0 && P.step_kernel >= 2) {
        delete h;
        return reject(LB_ERR_UNSUPPORTED, "the TMA-staged step kernel runs the free wave; forced runs use the plain kernel");
    }
    if (h->shape.tma && P.force_amp == 0.0) {
        const int ttw = h->shape.tma_tw;
        h->tma_ntiles_x = (P.nx + ttw - 1) / ttw;
        h->tma_x0_last = P.nx >= ttw ? P.nx - ttw : 0;
        h->tma_ntiles = h->tma_ntiles_x * ((P.ny + h->shape.tma_rows - 1) / h->shape.tma_rows);
        h->tma_grid = std::max(1, std::min(h->tma_ntiles, nsm * std::max(1, h->shape.tma_occupancy)));
        // auto: TMA staging once the grid fills a tile row and every SM gets work
        const bool big = P.nx >= ttw && h->tma_ntiles >= nsm;
        h->use_tma = P.step_kernel >= 2 || (P.step_kernel == 0 && big);
        // the store-staged kernel (Lax-Wendroff sets): automatic on the same grids where it is
        // the faster.  Its stores cover whole 16-byte granules of a row, so nx must be a multiple
        // of 16 / (bytes per population) (else the store of the last tile would reach the
        // periodic images past nx)
        if (h->shape.st && !upwind && P.nx % (int)(16 / storage_bytes(P.precision)) == 0) {
            h->st_ntiles_x = (P.nx + h->shape.st_tw - 1) / h->shape.st_tw;
            h->st_ntiles = h->st_ntiles_x * ((P.ny + h->shape.st_rows - 1) / h->shape.st_rows);
            h->st_grid = std::max(1, std::min(h->st_ntiles, nsm * std::max(1, h->shape.st_occupancy)));
            h->use_st = P.step_kernel == 3 || (P.step_kernel == 0 && h->shape.st_auto && big && h->st_ntiles >= nsm);
        }
        if (P.step_kernel == 3 && !h->use_st) {
            delete h;
            return reject(LB_ERR_UNSUPPORTED,
                          "no store-staged TMA step kernel for this set, storage, streaming or nx (a multiple of 16 bytes)");
        }
    } else if (P.step_kernel >= 2) {
        delete h;
        return reject(LB_ERR_UNSUPPORTED, "no TMA-staged step kernel for this storage");
    }
    h->grid = std::max(1, std::min(h->ntiles, nsm * occ));
    h->grid_init = (int)std::max<long long>(1, std::min<long long>((h->ncell + 255) / 256, 4LL * nsm));
    const size_t rbytes = P.precision == LB_F64 ? 8 : 4;
    h->buf[0] = h->dalloc(h->pop_bytes);
    h->buf[1] = h->dalloc(h->pop_bytes);
    h->sin_d = h->dalloc(rbytes * P.nx);
    h->cos_d = h->dalloc(rbytes * P.nx);
    h->partials = static_cast<double*>(
        h->dalloc(sizeof(double) * lbk::kDiagSlots * (size_t)std::max({h->grid, h->tma_grid, h->st_grid})));
    h->ticket = static_cast<unsigned int*>(h->dalloc(256));
    h->level_d = static_cast<long long*>(h->dalloc(256));
    h->status = static_cast<int*>(h->dalloc(256));
    h->ring = static_cast<lb_diag*>(h->dalloc(sizeof(lb_diag) * (size_t)P.diag_capacity));
    if (!h->buf[0] || !h->buf[1] || !h->sin_d || !h->cos_d || !h->partials || !h->ticket || !h->level_d ||
        !h->status || !h->ring) {
        h->release();
        delete h;
        return reject(LB_ERR_NOMEM, "device allocation failed");
    }
    std::vector<double> sd(P.nx), cd(P.nx);
    for (int i = 0; i < P.nx; ++i) {
        sd[i] = std::sin(2.0 * M_PI * i / P.nx);
        cd[i] = std::cos(2.0 * M_PI * i / P.nx);
    }
    if (P.precision == LB_F64) {
        e = cudaMemcpyAsync(h->sin_d, sd.data(), 8 * P.nx, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->cos_d, cd.data(), 8 * P.nx, cudaMemcpyHostToDevice, h->stream);
    } else {
        std::vector<float> sf(sd.begin(), sd.end()), cf(cd.begin(), cd.end());
        e = cudaMemcpyAsync(h->sin_d, sf.data(), 4 * P.nx, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->cos_d, cf.data(), 4 * P.nx, cudaMemcpyHostToDevice, h->stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(h->ticket, 0, 256, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->buf[0], 0, h->pop_bytes, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->buf[1], 0, h->pop_bytes, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        h->release();
        delete h;
        return reject(LB_ERR_CUDA, std::string("setup copies: ") + cudaGetErrorString(e));
    }
    if (h->use_tma) {
        const lb_status st = encode_maps(h);
        if (st != LB_OK) {
            const std::string m = h->err;
            h->release();
            delete h;
            return reject(st, m);
        }
    }
    *out = h;
    return LB_OK;
}

lb_status lb_destroy(lb_handle* h) {
    if (!h) return LB_OK;
    h->release();
    delete h;
    return LB_OK;
}

lb_status lb_init_shear_wave(lb_handle* h, double u0, double u1) {
    if (!h) return LB_ERR_ARG;
    if (!std::isfinite(u0) || !std::isfinite(u1)) return h->fail(LB_ERR_ARG, "non-finite amplitude");
    set_scale_and_tables(h, std::fabs(u0) + std::fabs(u1));
    return init_common(h, u0, u1, nullptr, nullptr, nullptr, nullptr);
}

lb_status lb_init_fields(lb_handle* h, const double* rho, const double* ux, const double* uy, const double* T) {
    if (!h || !rho || !ux || !uy) return h ? h->fail(LB_ERR_ARG, "rho, ux, uy are required") : LB_ERR_ARG;
    const size_t n = (size_t)h->ncell;
    double amp = 0;
    if (scale_from_amplitude(h))  // a host pass over the fields: only when the scale depends on it
        for (size_t i = 0; i < n; ++i) amp = std::max(amp, std::max(std::fabs(ux[i]), std::fabs(uy[i])));
    set_scale_and_tables(h, amp);
    if (!h->mom) {
        h->mom = static_cast<double*>(h->dalloc(sizeof(double) * 5 * n));
        if (!h->mom) return h->fail(LB_ERR_NOMEM, "moments scratch");
    }
    double* d = h->mom;
    cudaError_t e = cudaMemcpyAsync(d, rho, 8 * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + n, ux, 8 * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + 2 * n, uy, 8 * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && T) e = cudaMemcpyAsync(d + 3 * n, T, 8 * n, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "initial fields upload");
    lb_status st = init_common(h, 0, 0, d, d + n, d + 2 * n, T ? d + 3 * n : nullptr);
    if (st != LB_OK) return st;
    e = cudaStreamSynchronize(h->stream);  // host arrays may be released by the caller
    return e == cudaSuccess ? LB_OK : h->cuda_fail(e, "init sync");
}

lb_status lb_step(lb_handle* h, int n) {
    if (!h || n < 0) return h ? h->fail(LB_ERR_ARG, "n must be >= 0") : LB_ERR_ARG;
    if (!h->initialized) return h->fail(LB_ERR_STATE, "lb_step before an init call");
    lb_status st;
    while (n > 0) {
        // graphs of 32, 2 or 1 levels, one per buffer parity, built on first use: a replay
        // costs one launch call and no parameter upload
        cudaGraphExec_t* g = nullptr;
        int len = 0;
        if (n >= kChunk) {
            g = &h->chunk[h->cur];
            len = kChunk;
        } else if (n >= 2) {
            g = &h->pair[h->cur];
            len = 2;
        } else {
            g = &h->single[h->cur];
            len = 1;
        }
        if (!*g && (st = build_graph(h, h->cur, len, g)) != LB_OK) return st;
        const cudaError_t e = cudaGraphLaunch(*g, h->stream);
        if (e != cudaSuccess) return h->cuda_fail(e, "cudaGraphLaunch");
        h->launches += len;
        // an even number of levels returns cur to itself; an odd one flips it
        if (len & 1) h->cur = 1 - h->cur;
        h->level += len;
        h->raw_prev = false;
        n -= len;
        if (n == 0) return h->mark_level();
    }
    return LB_OK;
}

// ---- slab decomposition: the ghost and boundary row blocks of the state the next step reads
namespace {
// element offset (in a plane) of the gy rows starting at row r0 (r0 in [-gy, ny + gy - gy])
long long row_block(const lb_handle* h, int r0) { return (long long)(r0 + h->gy) * h->pitch; }

lb_status halo_copy(lb_handle* h, int side, void* dst, const void* src, bool pack) {
    if (!h->initialized) return h->fail(LB_ERR_STATE, "init first");
    if ((side != 0 && side != 1) || (pack ? !dst : !src)) return h->fail(LB_ERR_ARG, "side 0 or 1 and a device buffer");
    const size_t b = storage_bytes(h->p.precision);
    const size_t block = (size_t)h->gy * h->pitch * b;   // gy whole padded rows of one plane
    const size_t plane = (size_t)h->plane * b;
    char* state = static_cast<char*>(h->buf[h->cur]);
    // pack: boundary rows 0..gy-1 or ny-gy..ny-1; unpack: ghost rows -gy..-1 or ny..ny+gy-1
    const int r0 = pack ? (side == 0 ? 0 : h->p.ny - h->gy) : (side == 0 ? -h->gy : h->p.ny);
    char* rows = state + row_block(h, r0) * (long long)b;
    const cudaError_t e = pack ? cudaMemcpy2DAsync(dst, block, rows, plane, block, h->vs.q, cudaMemcpyDeviceToDevice,
                                                   h->stream)
                               : cudaMemcpy2DAsync(rows, plane, src, block, block, h->vs.q, cudaMemcpyDeviceToDevice,
                                                   h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, pack ? "halo pack" : "halo unpack");
    return LB_OK;
}
}  // namespace

lb_status lb_halo_bytes(const lb_handle* h, size_t* bytes) {
    if (!h || !bytes) return LB_ERR_ARG;
    *bytes = (size_t)h->vs.q * h->gy * h->pitch * storage_bytes(h->p.precision);
    return LB_OK;
}

lb_status lb_halo_pack(lb_handle* h, int side, void* dst) {
    if (!h) return LB_ERR_ARG;
    return halo_copy(h, side, dst, nullptr, true);
}

lb_status lb_halo_unpack(lb_handle* h, int side, const void* src) {
    if (!h) return LB_ERR_ARG;
    return halo_copy(h, side, nullptr, src, false);
}

lb_status lb_synchronize(lb_handle* h) {
    if (!h) return LB_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "cudaStreamSynchronize");
    int status = 0;
    e = cudaMemcpy(&status, h->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return h->cuda_fail(e, "status read");
    if (status & 2) return h->fail(LB_ERR_TIMEOUT, "a bounded wait in the step kernel ran out");
    if (status & 1) return h->fail(LB_ERR_UNSTABLE, "the state became non-finite");
    return LB_OK;
}

lb_status lb_moments_device(lb_handle* h, double* rho, double* ux, double* uy, double* T, double* sxy) {
    if (!h) return LB_ERR_ARG;
    if (!h->initialized) return h->fail(LB_ERR_STATE, "lb_moments before an init call");
    // the state f~(n) = stream(buffer read by the last launch); streamed by the TMA-staged
    // kernel when the steps are (the raw state right after init has nothing to stream)
    const int prev = 1 - h->cur;
    if (h->use_tma && !h->raw_prev)
        return launch_any(h, lbk::kMomentsTma, h->buf[prev], nullptr, 0, h->tma_grid, rho, ux, uy, T, sxy, nullptr);
    return launch_any(h, lbk::kMoments, h->buf[prev], nullptr, h->raw_prev ? 1 : 0, h->grid, rho, ux, uy, T, sxy,
                      nullptr);
}

lb_status lb_moments(lb_handle* h, double* rho, double* ux, double* uy, double* T, double* sxy) {
    if (!h) return LB_ERR_ARG;
    if (!h->initialized) return h->fail(LB_ERR_STATE, "lb_moments before an init call");
    const size_t n = (size_t)h->ncell;
    if (!h->mom) {
        h->mom = static_cast<double*>(h->dalloc(sizeof(double) * 5 * n));
        if (!h->mom) return h->fail(LB_ERR_NOMEM, "moments scratch");
    }
    double* d = h->mom;
    lb_status st = lb_moments_device(h, rho ? d : nullptr, ux ? d + n : nullptr, uy ? d + 2 * n : nullptr,
                                      T ? d + 3 * n : nullptr, sxy ? d + 4 * n : nullptr);
    if (st != LB_OK) return st;
    double* outs[5] = {rho, ux, uy, T, sxy};
    for (int k = 0; k < 5; ++k) {
        if (!outs[k]) continue;
        const cudaError_t e = cudaMemcpyAsync(outs[k], d + k * n, 8 * n, cudaMemcpyDeviceToHost, h->stream);
        if (e != cudaSuccess) return h->cuda_fail(e, "moments read-back");
    }
    return lb_synchronize(h);
}

lb_status lb_populations(lb_handle* h, double* f) {
    if (!h || !f) return h ? h->fail(LB_ERR_ARG, "null output") : LB_ERR_ARG;
    if (!h->initialized) return h->fail(LB_ERR_STATE, "lb_populations before an init call");
    const size_t n = (size_t)h->ncell * h->vs.q;
    if (!h->pop) {
        h->pop = static_cast<double*>(h->dalloc(sizeof(double) * n));
        if (!h->pop) return h->fail(LB_ERR_NOMEM, "population scratch");
    }
    const int prev = 1 - h->cur;
    const bool tma = h->use_tma && !h->raw_prev;
    lb_status st = launch_any(h, tma ? lbk::kMomentsTma : lbk::kMoments, h->buf[prev], nullptr,
                              h->raw_prev ? 1 : 0, tma ? h->tma_grid : h->grid, nullptr, nullptr, nullptr, nullptr,
                              nullptr, h->pop);
    if (st != LB_OK) return st;
    const cudaError_t e = cudaMemcpyAsync(f, h->pop, 8 * n, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "population read-back");
    return lb_synchronize(h);
}

lb_status lb_diagnostics(lb_handle* h, lb_diag* out, int max_records, int* n_out) {
    if (!h || !out || !n_out || max_records < 0) return h ? h->fail(LB_ERR_ARG, "bad arguments") : LB_ERR_ARG;
    if (!h->initialized) return h->fail(LB_ERR_STATE, "lb_diagnostics before an init call");
    lb_status st = lb_synchronize(h);
    if (st != LB_OK && st != LB_ERR_UNSTABLE) return st;
    const long long total = h->level + 1;  // records for levels 0..n
    const long long cap = h->p.diag_capacity;
    const long long cnt = std::min<long long>(std::min(total, cap), max_records);
    const long long first = total - cnt;
    for (long long i = 0; i < cnt;) {
        const long long slot = (first + i) % cap;
        const long long run = std::min(cnt - i, cap - slot);
        const cudaError_t e = cudaMemcpy(out + i, h->ring + slot, sizeof(lb_diag) * run, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return h->cuda_fail(e, "diagnostics read-back");
        i += run;
    }
    *n_out = (int)cnt;
    return st;
}

lb_status lb_diagnostics_at(lb_handle* h, long long level, lb_diag* out) {
    if (!h || !out) return h ? h->fail(LB_ERR_ARG, "null output") : LB_ERR_ARG;
    if (!h->initialized) return h->fail(LB_ERR_STATE, "lb_diagnostics_at before an init call");
    const long long cap = h->p.diag_capacity;
    if (level < 0 || level > h->level || level <= h->level - cap)
        return h->fail(LB_ERR_ARG, "level not in the diagnostics ring");
    // the first completion marker at or past the level (a later one is also sufficient)
    int best = -1;
    for (int i = 0; i < lb_handle::kMarks; ++i)
        if (h->ev_level[i] >= level && (best < 0 || h->ev_level[i] < h->ev_level[best])) best = i;
    cudaError_t e = best >= 0 ? cudaEventSynchronize(h->ev[best]) : cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "waiting for the level");
    // the copy runs on a stream of its own, so it does not wait for the levels still
    // running on the handle's stream
    if (!h->copy_stream && (e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return h->cuda_fail(e, "cudaStreamCreate");
    e = cudaMemcpyAsync(out, h->ring + level % cap, sizeof(lb_diag), cudaMemcpyDeviceToHost, h->copy_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->copy_stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "diagnostics read-back");
    if (out->flags != 0.0) return h->fail(LB_ERR_UNSTABLE, "non-finite diagnostics record");
    return LB_OK;
}

lb_status lb_fit_decay(lb_handle* h, double t_start, double floor_rel, double* rate, int* npoints,
                       double* shear_ratio) {
    if (!h || !rate || !npoints) return h ? h->fail(LB_ERR_ARG, "null output") : LB_ERR_ARG;
    if (!h->initialized) return h->fail(LB_ERR_STATE, "lb_fit_decay before an init call");
    const long long total = h->level + 1;
    if (total > h->p.diag_capacity) return h->fail(LB_ERR_ARG, "records no longer in the ring (raise diag_capacity)");
    std::vector<lb_diag> rec((size_t)total);
    int n = 0;
    lb_status st = lb_diagnostics(h, rec.data(), (int)total, &n);
    if (st != LB_OK) return st;
    const double a0 = std::fabs(rec[0].amp);
    double st_ = 0, sl = 0, stt = 0, stl = 0, smax = 0;
    int m = 0;
    for (int i = 0; i < n; ++i) {
        if (rec[i].t < t_start) continue;
        const double a = std::fabs(rec[i].amp);
        if (!(a >= floor_rel * a0) || a == 0.0) break;
        const double l = std::log(a);
        st_ += rec[i].t;
        sl += l;
        stt += rec[i].t * rec[i].t;
        stl += rec[i].t * l;
        smax = std::max(smax, std::fabs(rec[i].shear));
        ++m;
    }
    if (m < 3) return h->fail(LB_ERR_ARG, "fewer than 3 records in the fit window");
    const double den = m * stt - st_ * st_;
    if (!(den > 0)) return h->fail(LB_ERR_ARG, "degenerate fit window");
    *rate = -(m * stl - st_ * sl) / den;
    *npoints = m;
    if (shear_ratio) *shear_ratio = a0 > 0 ? smax / a0 : 0.0;
    return LB_OK;
}

lb_status lb_get_info(const lb_handle* h, lb_info_t* o) {
    if (!h || !o) return LB_ERR_ARG;
    o->q = h->vs.q;
    o->degree = h->vs.degree;
    o->on_lattice = h->vs.on_lattice ? 1 : 0;
    o->halo = h->vs.halo;
    o->dx = h->dx;
    o->dt = h->dt;
    o->tau = h->tau;
    o->omega = h->omega;
    o->c_lattice = h->vs.c;
    o->time_level = h->level;
    o->tma_staged = h->use_st ? 2 : h->use_tma ? 1 : 0;
    o->records = h->initialized ? h->level + 1 : 0;
    o->bytes_per_cell_update = 2 * (size_t)h->vs.q * storage_bytes(h->p.precision);
    o->device_bytes = h->device_bytes;
    o->storage_scale = h->scale;
    return LB_OK;
}

long long lb_kernel_launches(const lb_handle* h) { return h ? h->launches : 0; }

}  // extern "C"
