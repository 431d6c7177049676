// lb_solve_static: one small standing-shear-wave solve whose device state lives
// in a fixed, file-scope __device__ array instead of memory the library
// allocates.  It runs the persistent multi-instance kernel (lb_batch_kernel)
// with a single instance; every device pointer that kernel reads or writes
// points into lb_static_scratch.
//
// Layout of the scratch for one call (offsets rounded up to 256 bytes):
//   [0, 256)     the instance descriptor (BatchInst), uploaded per call
//   [256, 512)   order[0] = 0, then the work-queue counter and the list length
//   trig         sin(x_i), cos(x_i): 2 nx floats, uploaded per call
//   hist         (A(n), S(n)) per level: max_steps + 1 float2, written by the kernel
//   pop[0..1]    the two population buffers: q nx ny elements each, written by the kernel
// Only the work-queue counter must be zero before the launch (cleared here with
// a memset); the kernel writes level 0 of the populations and every history
// record before reading them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "lb.h"
#include "lb_batch.h"
#include "lb_host.h"

static __device__ __align__(256) unsigned char lb_static_scratch[LB_STATIC_SCRATCH_BYTES];
static_assert(sizeof(lbk::BatchInst) <= 256, "the instance descriptor fills the first 256 bytes of the scratch");

namespace {

constexpr size_t kAlign = 256;
constexpr int kMaxDevices = 64;
constexpr int kThreads = 256;        // the batch defaults, so results match an lb_batch run
constexpr int kSmemBytes = 96 * 1024;

size_t round_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct DeviceSetup {
    bool ready = false;
    unsigned char* base = nullptr;   // device address of lb_static_scratch on this device
    bool kernel_ready[3] = {false, false, false};  // F32, F16, BF16
};

std::mutex g_setup_mu;                // guards the one-time set-up only
DeviceSetup g_dev[kMaxDevices];
bool g_tabs_ready = false;
lbh::VelocitySetInfo g_sets[3];
lbk::Tab<float> g_tab[3];

lb_status fail(lb_status s, const std::string& m) {
    lbh::set_last_error(m);
    return s;
}

lb_status cuda_fail(cudaError_t e, const char* where) {
    return fail(LB_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

int precision_index(lb_precision p) {
    switch (p) {
        case LB_F32: return 0;
        case LB_F16: return 1;
        case LB_BF16: return 2;
        default: return -1;
    }
}

int set_index(lb_quadrature q) {
    switch (q) {
        case LB_D2Q16_GH: return 0;
        case LB_D2Q36_GH: return 1;
        case LB_D2Q64_GH: return 2;
        default: return -1;
    }
}

// One-time, per-process: the three Gauss-Hermite product sets and their kernel
// tables (host work only).  Called with g_setup_mu held.
lb_status setup_tables() {
    if (g_tabs_ready) return LB_OK;
    const lb_quadrature qs[3] = {LB_D2Q16_GH, LB_D2Q36_GH, LB_D2Q64_GH};
    for (int i = 0; i < 3; ++i) {
        std::string e;
        if (!lbh::build_velocity_set(qs[i], &g_sets[i], &e)) return fail(LB_ERR_ARG, e);
        double amax = 0;
        for (double a : g_sets[i].axis) amax = std::max(amax, std::fabs(a));
        lbh::build_tab<float>(g_sets[i], 1.0 / amax, 1.0, 1.0, g_tab[i]);
    }
    g_tabs_ready = true;
    return LB_OK;
}

// One-time, per device (that device current): the scratch address and the
// kernel's shared-memory attribute for this storage type.
lb_status setup_device(int dev, int pi, unsigned char** base) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    lb_status st = setup_tables();
    if (st != LB_OK) return st;
    DeviceSetup& d = g_dev[dev];
    if (!d.ready) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, lb_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(lb_static_scratch)");
        d.base = static_cast<unsigned char*>(p);
        d.ready = true;
    }
    if (!d.kernel_ready[pi]) {
        int occ = 0;
        cudaError_t e = pi == 0   ? lbk::batch_setup_f32(kThreads, kSmemBytes, &occ)
                        : pi == 1 ? lbk::batch_setup_f16(kThreads, kSmemBytes, &occ)
                                  : lbk::batch_setup_bf16(kThreads, kSmemBytes, &occ);
        if (e != cudaSuccess) return cuda_fail(e, "kernel set-up");
        if (occ < 1) return fail(LB_ERR_CUDA, "kernel set-up: zero occupancy");
        d.kernel_ready[pi] = true;
    }
    *base = d.base;
    return LB_OK;
}

}  // namespace

extern "C" {

lb_status lb_solve_static(const lb_instance_desc* d, lb_precision precision, lb_kn_convention kn_convention,
                          float* history, int max_records, lb_instance_state* state, void* stream) {
    // ---- arguments (no CUDA call before they are known to be valid)
    if (!d) return fail(LB_ERR_ARG, "null instance descriptor");
    const int pi = precision_index(precision);
    if (pi < 0) return fail(LB_ERR_UNSUPPORTED, "storage must be F32, F16 or BF16");
    if (kn_convention != LB_KN_LAMBDA && kn_convention != LB_KN_PAPER) return fail(LB_ERR_ARG, "unknown kn_convention");
    const int si = set_index(d->quadrature);
    if (si < 0) return fail(LB_ERR_UNSUPPORTED, "lb_solve_static runs the Gauss-Hermite product sets");
    static const int kQ[3] = {16, 36, 64}, kDegree[3] = {7, 11, 15};
    if (d->n_eq < 2 || d->n_eq > 4 || kDegree[si] < d->n_eq + 2) return fail(LB_ERR_ARG, "n_eq out of range for the set");
    if (d->nx < 2 || d->ny < 1 || (long long)d->nx * d->ny > (1 << 26)) return fail(LB_ERR_ARG, "bad grid");
    if (!(d->kn > 0) || d->max_steps < 0 || !(d->stop_ratio >= 0) || !std::isfinite(d->u0))
        return fail(LB_ERR_ARG, "bad kn, max_steps, stop_ratio or u0");
    if (max_records < 0 || (max_records > 0 && !history)) return fail(LB_ERR_ARG, "history is required when max_records > 0");
    const size_t eb = precision == LB_F32 ? 4 : 2;
    const size_t ncell = (size_t)d->nx * (size_t)d->ny;
    const size_t pop_bytes = (size_t)kQ[si] * ncell * eb;
    const size_t trig_off = 512;
    const size_t hist_off = trig_off + round_up(sizeof(float) * 2 * (size_t)d->nx);
    const size_t pop_off = hist_off + round_up(sizeof(float2) * ((size_t)d->max_steps + 1));
    const size_t need = pop_off + 2 * round_up(pop_bytes);
    if (need > (size_t)LB_STATIC_SCRATCH_BYTES)
        return fail(LB_ERR_BUDGET, "the solve needs " + std::to_string(need) + " bytes of device scratch; "
                                   "lb_solve_static holds at most " + std::to_string((size_t)LB_STATIC_SCRATCH_BYTES) +
                                   " (use an lb_batch or an lb_handle for larger problems)");

    // ---- one-time set-up of the current device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(LB_ERR_UNSUPPORTED, "device ordinal beyond 63");
    unsigned char* base = nullptr;
    lb_status st = setup_device(dev, pi, &base);
    if (st != LB_OK) return st;
    const lbh::VelocitySetInfo& vs = g_sets[si];
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // ---- the instance (the same constants lb_batch_add derives)
    lbk::BatchInst in{};
    in.off[0] = 0;
    in.off[1] = (long long)(round_up(pop_bytes) / eb);
    in.hist_off = 0;
    in.trig_off = 0;
    in.set = si;
    in.n_eq = d->n_eq;
    in.nx = d->nx;
    in.ny = d->ny;
    in.max_level = d->max_steps;
    const double dx = 2.0 * M_PI / d->nx;
    double amax = 0;
    for (double a : vs.axis) amax = std::max(amax, std::fabs(a));
    const double dt = dx / amax;
    const double tau = kn_convention == LB_KN_LAMBDA ? d->kn * std::sqrt(2.0 / M_PI) : d->kn;
    const double omega = lbh::snap_unit(dt / (tau + 0.5 * dt));
    in.omega = (float)omega;
    {
        lbk::Tab<float> rt = g_tab[si];
        lbh::build_relax<float>(g_sets[si], in.omega, rt);
        std::memcpy(in.ow, rt.ow, sizeof(in.ow));
        std::memcpy(in.owlo, rt.owlo, sizeof(in.owlo));
        std::memcpy(in.hn1lo, rt.hn1lo, sizeof(in.hn1lo));
        std::memcpy(in.whn1lo, rt.whn1lo, sizeof(in.whn1lo));
    }
    in.sigma_fac = (float)(1.0 - 0.5 * omega);
    in.scale = (float)lbh::pow2_near(std::max(2.0 * std::fabs(d->u0), 1e-6));
    in.stop_ratio2 = (float)(d->stop_ratio * d->stop_ratio);
    in.u0 = d->u0;
    in.dt = dt;

    // ---- uploads: descriptor, work list, trig table (pageable sources: each copy has
    // consumed its source when it returns, so the stack buffers can be reused)
    const int ints[2] = {0, 1};  // order[0], list length
    e = cudaMemcpyAsync(base, &in, sizeof(in), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + 256, &ints[0], sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + 256 + 64, 0, sizeof(int), s);  // work-queue counter
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + 256 + 128, &ints[1], sizeof(int), cudaMemcpyHostToDevice, s);
    float chunk[1024];
    for (int half = 0; half < 2 && e == cudaSuccess; ++half) {
        for (int i0 = 0; i0 < d->nx && e == cudaSuccess; i0 += 1024) {
            const int m = std::min(1024, d->nx - i0);
            for (int i = 0; i < m; ++i) {
                const double x = 2.0 * M_PI * (i0 + i) / d->nx;
                chunk[i] = (float)(half == 0 ? std::sin(x) : std::cos(x));
            }
            e = cudaMemcpyAsync(base + trig_off + sizeof(float) * ((size_t)half * d->nx + i0), chunk,
                                sizeof(float) * m, cudaMemcpyHostToDevice, s);
        }
    }
    if (e != cudaSuccess) return cuda_fail(e, "scratch upload");

    // ---- one launch: one CTA advances the instance until it finishes
    lbk::BatchArgs args{};
    args.inst = reinterpret_cast<lbk::BatchInst*>(base);
    args.order = reinterpret_cast<const int*>(base + 256);
    args.next = reinterpret_cast<int*>(base + 256 + 64);
    args.n_order = reinterpret_cast<const int*>(base + 256 + 128);
    args.chunk = 1 << 30;
    args.smem_cap = kSmemBytes;
    args.arena = base + pop_off;
    args.hist = reinterpret_cast<float2*>(base + hist_off);
    args.trig = reinterpret_cast<const float*>(base + trig_off);
    for (int i = 0; i < 3; ++i) args.tab[i] = g_tab[i];
    e = pi == 0   ? lbk::batch_launch_f32(&args, 1, kThreads, kSmemBytes, s)
        : pi == 1 ? lbk::batch_launch_f16(&args, 1, kThreads, kSmemBytes, s)
                  : lbk::batch_launch_bf16(&args, 1, kThreads, kSmemBytes, s);
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");

    // ---- results (device-to-pageable copies return once they have completed)
    lbk::BatchInst out{};
    e = cudaMemcpyAsync(&out, base, sizeof(out), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "instance read-back");
    if (out.status & 1) return fail(LB_ERR_UNSTABLE, "the state became non-finite");
    const int n = std::min(out.level, max_records);
    if (n > 0) {
        e = cudaMemcpyAsync(history, base + hist_off, sizeof(float2) * (size_t)n, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "history read-back");
    }
    if (state) {
        state->level = out.level;
        state->done = out.done;
        state->status = out.status;
        state->q = vs.q;
        state->dt = dt;
        state->omega = in.omega;
        state->tau = tau;
        state->bytes = need;
    }
    return LB_OK;
}

}  // extern "C"
