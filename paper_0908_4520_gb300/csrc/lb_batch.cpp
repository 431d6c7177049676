// C-ABI of batches (lb_batch_*): a device arena with first-fit allocation
// and budget-based admission, per-slot device descriptors, a work list
// ordered by remaining cost, and one persistent kernel launch per run,
// replayed from a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "lb.h"
#include "lb_batch.h"
#include "lb_host.h"

namespace {

thread_local std::string g_batch_error;

// First-fit allocator of byte ranges in [0, cap).
class RangeAllocator {
   public:
    explicit RangeAllocator(size_t cap = 0) { reset(cap); }
    void reset(size_t cap) {
        free_.clear();
        if (cap) free_[0] = cap;
        used_ = 0;
    }
    // returns false if no free range fits
    bool alloc(size_t bytes, size_t align, size_t* off) {
        bytes = (bytes + align - 1) / align * align;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            const size_t start = (it->first + align - 1) / align * align;
            const size_t end = it->first + it->second;
            if (start + bytes <= end) {
                const size_t lo = it->first, hi_start = start + bytes;
                free_.erase(it);
                if (start > lo) free_[lo] = start - lo;
                if (end > hi_start) free_[hi_start] = end - hi_start;
                *off = start;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes, size_t align) {
        bytes = (bytes + align - 1) / align * align;
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        // coalesce with neighbours
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
                it = prev;
            }
        }
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
    }
    size_t used() const { return used_; }

   private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0;
};

constexpr size_t kAlign = 256;

size_t elem_bytes(lb_precision p) { return p == LB_F32 ? 4 : 2; }

int set_index(lb_quadrature q) {
    switch (q) {
        case LB_D2Q16_GH: return 0;
        case LB_D2Q36_GH: return 1;
        case LB_D2Q64_GH: return 2;
        default: return -1;
    }
}

}  // namespace

struct lb_batch {
    lb_batch_params p{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void* arena = nullptr;
    RangeAllocator ranges;
    lbh::VelocitySetInfo sets[3];
    lbk::BatchArgs args{};
    lbk::BatchInst* inst_d = nullptr;
    int* order_d = nullptr;
    int* counters_d = nullptr;  // [0] next, [1] next_small, [2] n_order, [3] n_small
    int* order_small_d = nullptr;
    int warp_cells = 0;
    unsigned long long* clock_d = nullptr;  // per CTA: start, end of the last launch (%globaltimer, ns)
    std::vector<lbk::BatchInst> inst;
    std::vector<char> live, dirty;
    std::vector<std::vector<std::pair<size_t, size_t>>> ranges_of;
    std::vector<double> tau;
    int threads = 256, smem = 96 * 1024, grid = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_chunk = -1;
    bool in_flight = false;
    bool stale = false;  // host view of the slots predates the last launch
    long long launches = 0;
    std::string err;

    lb_status fail(lb_status s, const std::string& m) {
        err = m;
        return s;
    }
    lb_status cuda_fail(cudaError_t e, const char* where) {
        err = std::string(where) + ": " + cudaGetErrorString(e);
        return LB_ERR_CUDA;
    }
    // wait for a launch in flight and refresh the host view of the slots
    lb_status settle() {
        if (in_flight) {
            const cudaError_t e = cudaStreamSynchronize(stream);
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
            in_flight = false;
        }
        if (stale) {
            const cudaError_t e =
                cudaMemcpy(inst.data(), inst_d, sizeof(lbk::BatchInst) * inst.size(), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(e, "slot read-back");
            stale = false;
        }
        return LB_OK;
    }
};

namespace {

cudaError_t batch_launch(lb_batch* b) {
    switch (b->p.precision) {
        case LB_F32: return lbk::batch_launch_f32(&b->args, b->grid, b->threads, b->smem, b->stream);
        case LB_F16: return lbk::batch_launch_f16(&b->args, b->grid, b->threads, b->smem, b->stream);
        case LB_BF16: return lbk::batch_launch_bf16(&b->args, b->grid, b->threads, b->smem, b->stream);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t batch_setup(lb_precision prec, int threads, int smem, int* occ) {
    switch (prec) {
        case LB_F32: return lbk::batch_setup_f32(threads, smem, occ);
        case LB_F16: return lbk::batch_setup_f16(threads, smem, occ);
        case LB_BF16: return lbk::batch_setup_bf16(threads, smem, occ);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

extern "C" {

void lb_batch_params_default(lb_batch_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->precision = LB_F32;
    p->kn_convention = LB_KN_LAMBDA;
    p->budget_bytes = (size_t)1 << 30;
    p->max_slots = 4096;
    p->threads = 0;
    p->smem_bytes = -1;
    p->warp_cells = -1;
}

const char* lb_batch_last_error(const lb_batch* b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

lb_status lb_batch_create(const lb_batch_params* pin, lb_batch** out) {
    if (!pin || !out) {
        g_batch_error = "null argument";
        return LB_ERR_ARG;
    }
    const lb_batch_params& P = *pin;
    if (P.precision != LB_F32 && P.precision != LB_F16 && P.precision != LB_BF16) {
        g_batch_error = "batch storage must be F32, F16 or BF16";
        return LB_ERR_UNSUPPORTED;
    }
    if (P.max_slots < 1 || P.budget_bytes < kAlign) {
        g_batch_error = "max_slots >= 1 and a positive budget are required";
        return LB_ERR_ARG;
    }
    if (P.threads != 0 && (P.threads < 64 || P.threads > 256 || P.threads % 32)) {
        g_batch_error = "threads must be 0 or a multiple of 32 in [64, 256]";
        return LB_ERR_ARG;
    }
    if (P.kn_convention != LB_KN_LAMBDA && P.kn_convention != LB_KN_PAPER) {
        g_batch_error = "unknown kn_convention";
        return LB_ERR_ARG;
    }
    lb_batch* b = new (std::nothrow) lb_batch();
    if (!b) {
        g_batch_error = "host allocation";
        return LB_ERR_NOMEM;
    }
    b->p = P;
    b->threads = P.threads ? P.threads : 256;
    b->smem = P.smem_bytes < 0 ? 96 * 1024 : P.smem_bytes;
    b->warp_cells = P.warp_cells < 0 ? 512 : P.warp_cells;
    auto bail = [&](lb_status s, const std::string& m) {
        g_batch_error = m;
        if (b->graph) cudaGraphExecDestroy(b->graph);
        if (b->arena) cudaFree(b->arena);
        if (b->inst_d) cudaFree(b->inst_d);
        if (b->order_d) cudaFree(b->order_d);
        if (b->counters_d) cudaFree(b->counters_d);
        if (b->order_small_d) cudaFree(b->order_small_d);
        if (b->clock_d) cudaFree(b->clock_d);
        if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
        delete b;
        return s;
    };
    const lb_quadrature qs[3] = {LB_D2Q16_GH, LB_D2Q36_GH, LB_D2Q64_GH};
    for (int i = 0; i < 3; ++i) {
        std::string e;
        if (!lbh::build_velocity_set(qs[i], &b->sets[i], &e)) return bail(LB_ERR_ARG, e);
        // Courant numbers a_i dt / dx = a_i / max|a| (cfl 1) do not depend on nx
        double amax = 0;
        for (double a : b->sets[i].axis) amax = std::max(amax, std::fabs(a));
        lbh::build_tab<float>(b->sets[i], 1.0 / amax, 1.0, 1.0, b->args.tab[i]);
    }
    cudaError_t e;
    if (P.stream) {
        b->stream = static_cast<cudaStream_t>(P.stream);
    } else {
        if ((e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking)) != cudaSuccess)
            return bail(LB_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
        b->own_stream = true;
    }
    int occ = 0;
    if ((e = batch_setup(P.precision, b->threads, b->smem, &occ)) != cudaSuccess || occ < 1)
        return bail(LB_ERR_ARG, std::string("kernel configuration does not fit: ") +
                                    (e != cudaSuccess ? cudaGetErrorString(e) : "zero occupancy"));
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    b->grid = std::max(1, nsm * occ);
    if (cudaMalloc(&b->arena, P.budget_bytes) != cudaSuccess) return bail(LB_ERR_NOMEM, "arena allocation");
    if (cudaMalloc(&b->inst_d, sizeof(lbk::BatchInst) * P.max_slots) != cudaSuccess ||
        cudaMalloc(&b->order_d, sizeof(int) * P.max_slots) != cudaSuccess ||
        cudaMalloc(&b->counters_d, 256) != cudaSuccess ||
        cudaMalloc(&b->order_small_d, sizeof(int) * P.max_slots) != cudaSuccess ||
        cudaMalloc(&b->clock_d, sizeof(unsigned long long) * 2 * b->grid) != cudaSuccess)
        return bail(LB_ERR_NOMEM, "descriptor allocation");
    b->ranges.reset(P.budget_bytes);
    b->inst.assign(P.max_slots, lbk::BatchInst{});
    b->live.assign(P.max_slots, 0);
    b->dirty.assign(P.max_slots, 0);
    b->ranges_of.assign(P.max_slots, {});
    b->tau.assign(P.max_slots, 0.0);
    b->args.inst = b->inst_d;
    b->args.order = b->order_d;
    b->args.next = b->counters_d;
    b->args.next_small = b->counters_d + 1;
    b->args.n_order = b->counters_d + 2;
    b->args.n_small = b->counters_d + 3;
    b->args.order_small = b->order_small_d;
    b->args.smem_cap = b->smem;
    b->args.arena = b->arena;
    b->args.hist = static_cast<float2*>(b->arena);
    b->args.trig = static_cast<const float*>(b->arena);
    b->args.cta_clock = b->clock_d;
    if ((e = cudaMemsetAsync(b->clock_d, 0, sizeof(unsigned long long) * 2 * b->grid, b->stream)) != cudaSuccess)
        return bail(LB_ERR_CUDA, cudaGetErrorString(e));
    if ((e = cudaMemsetAsync(b->counters_d, 0, 256, b->stream)) != cudaSuccess)
        return bail(LB_ERR_CUDA, cudaGetErrorString(e));
    *out = b;
    return LB_OK;
}

lb_status lb_batch_destroy(lb_batch* b) {
    if (!b) return LB_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    cudaFree(b->arena);
    cudaFree(b->inst_d);
    cudaFree(b->order_d);
    cudaFree(b->counters_d);
    cudaFree(b->order_small_d);
    cudaFree(b->clock_d);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return LB_OK;
}

lb_status lb_batch_run_profile(lb_batch* b, double* span_s, double* tail_s, int* ctas) {
    if (!b) return LB_ERR_ARG;
    lb_status st = b->settle();
    if (st != LB_OK) return st;
    std::vector<unsigned long long> c(2 * (size_t)b->grid);
    const cudaError_t e =
        cudaMemcpy(c.data(), b->clock_d, sizeof(unsigned long long) * c.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return b->cuda_fail(e, "clock read");
    unsigned long long first = ~0ull, last = 0, second = 0;
    int n = 0;
    for (int i = 0; i < b->grid; ++i) {
        if (c[2 * i + 1] == 0) continue;  // no launch yet
        ++n;
        first = std::min(first, c[2 * i]);
        const unsigned long long end = c[2 * i + 1];
        if (end > last) {
            second = last;
            last = end;
        } else if (end > second) {
            second = end;
        }
    }
    if (n == 0) return b->fail(LB_ERR_STATE, "no batch launch has run");
    if (span_s) *span_s = (double)(last - first) * 1e-9;
    if (tail_s) *tail_s = n > 1 ? (double)(last - second) * 1e-9 : 0.0;
    if (ctas) *ctas = n;
    return LB_OK;
}

lb_status lb_batch_add(lb_batch* b, const lb_instance_desc* d, int* slot) {
    if (!b || !d || !slot) return b ? b->fail(LB_ERR_ARG, "null argument") : LB_ERR_ARG;
    const int si = set_index(d->quadrature);
    if (si < 0) return b->fail(LB_ERR_UNSUPPORTED, "batches run the Gauss-Hermite product sets");
    const lbh::VelocitySetInfo& vs = b->sets[si];
    if (d->n_eq < 2 || d->n_eq > 4 || vs.degree < d->n_eq + 2) return b->fail(LB_ERR_ARG, "n_eq out of range for the set");
    if (d->nx < 2 || d->ny < 1 || (long long)d->nx * d->ny > (1 << 26)) return b->fail(LB_ERR_ARG, "bad grid");
    if (!(d->kn > 0) || d->max_steps < 0 || !(d->stop_ratio >= 0) || !std::isfinite(d->u0))
        return b->fail(LB_ERR_ARG, "bad kn, max_steps, stop_ratio or u0");
    lb_status st = b->settle();
    if (st != LB_OK) return st;
    int s = -1;
    for (int i = 0; i < b->p.max_slots; ++i)
        if (!b->live[i]) {
            s = i;
            break;
        }
    if (s < 0) return b->fail(LB_ERR_BUDGET, "no free slot");
    const size_t eb = elem_bytes(b->p.precision);
    const size_t ncell = (size_t)d->nx * d->ny;
    const size_t pop_bytes = (size_t)vs.q * ncell * eb;
    const size_t sizes[4] = {pop_bytes, pop_bytes, sizeof(float2) * ((size_t)d->max_steps + 1),
                             sizeof(float) * 2 * (size_t)d->nx};
    size_t offs[4];
    for (int k = 0; k < 4; ++k) {
        if (!b->ranges.alloc(sizes[k], kAlign, &offs[k])) {
            for (int j = 0; j < k; ++j) b->ranges.release(offs[j], sizes[j], kAlign);
            return b->fail(LB_ERR_BUDGET, "instance does not fit the remaining arena budget");
        }
    }
    b->ranges_of[s].clear();
    for (int k = 0; k < 4; ++k) b->ranges_of[s].push_back({offs[k], sizes[k]});
    lbk::BatchInst in{};
    in.off[0] = (long long)(offs[0] / eb);
    in.off[1] = (long long)(offs[1] / eb);
    in.hist_off = (long long)(offs[2] / sizeof(float2));
    in.trig_off = (long long)(offs[3] / sizeof(float));
    in.set = si;
    in.n_eq = d->n_eq;
    in.nx = d->nx;
    in.ny = d->ny;
    in.max_level = d->max_steps;
    in.level = 0;
    in.cur = 0;
    in.done = 0;
    in.status = 0;
    in.isothermal = 0;
    const double dx = 2.0 * M_PI / d->nx;
    double amax = 0;
    for (double a : vs.axis) amax = std::max(amax, std::fabs(a));
    const double dt = dx / amax;
    const double tau = b->p.kn_convention == LB_KN_LAMBDA ? d->kn * std::sqrt(2.0 / M_PI) : d->kn;
    const double omega = lbh::snap_unit(dt / (tau + 0.5 * dt));
    in.omega = (float)omega;
    {
        lbk::Tab<float> rt = b->args.tab[si];
        lbh::build_relax<float>(b->sets[si], in.omega, rt);
        std::memcpy(in.ow, rt.ow, sizeof(in.ow));
        std::memcpy(in.owlo, rt.owlo, sizeof(in.owlo));
        std::memcpy(in.hn1lo, rt.hn1lo, sizeof(in.hn1lo));
        std::memcpy(in.whn1lo, rt.whn1lo, sizeof(in.whn1lo));
    }
    in.sigma_fac = (float)(1.0 - 0.5 * omega);
    in.scale = (float)lbh::pow2_near(std::max(2.0 * std::fabs(d->u0), 1e-6));
    in.stop_ratio2 = (float)(d->stop_ratio * d->stop_ratio);
    in.h0 = 0.f;
    in.u0 = d->u0;
    in.dt = dt;
    b->inst[s] = in;
    b->tau[s] = tau;
    std::vector<float> trig(2 * (size_t)d->nx);
    for (int i = 0; i < d->nx; ++i) {
        trig[i] = (float)std::sin(2.0 * M_PI * i / d->nx);
        trig[d->nx + i] = (float)std::cos(2.0 * M_PI * i / d->nx);
    }
    cudaError_t e = cudaMemcpy(static_cast<char*>(b->arena) + offs[3], trig.data(), sizes[3], cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->inst_d + s, &b->inst[s], sizeof(lbk::BatchInst), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        for (auto& r : b->ranges_of[s]) b->ranges.release(r.first, r.second, kAlign);
        b->ranges_of[s].clear();
        return b->cuda_fail(e, "slot upload");
    }
    b->live[s] = 1;
    *slot = s;
    return LB_OK;
}

lb_status lb_batch_remove(lb_batch* b, int slot) {
    if (!b || slot < 0 || slot >= (b ? b->p.max_slots : 0) || !b->live[slot])
        return b ? b->fail(LB_ERR_ARG, "no such slot") : LB_ERR_ARG;
    lb_status st = b->settle();
    if (st != LB_OK) return st;
    for (auto& r : b->ranges_of[slot]) b->ranges.release(r.first, r.second, kAlign);
    b->ranges_of[slot].clear();
    b->live[slot] = 0;
    return LB_OK;
}

lb_status lb_batch_run(lb_batch* b, int chunk) {
    if (!b || chunk < 0) return b ? b->fail(LB_ERR_ARG, "chunk must be >= 0") : LB_ERR_ARG;
    lb_status st = b->settle();
    if (st != LB_OK) return st;
    const int ch = chunk == 0 ? (1 << 30) : chunk;
    // work lists: live, unfinished slots by decreasing remaining cost; instances of at most
    // warp_cells cells go to the warp queue
    std::vector<int> order, small;
    std::vector<double> cost(b->p.max_slots, 0.0);
    for (int s = 0; s < b->p.max_slots; ++s) {
        if (!b->live[s] || b->inst[s].done) continue;
        const lbk::BatchInst& in = b->inst[s];
        const double levels = std::min<double>(in.max_level - in.level + 1, ch);
        cost[s] = levels * (double)in.nx * in.ny * b->sets[in.set].q;
        ((long long)in.nx * in.ny <= b->warp_cells ? small : order).push_back(s);
    }
    auto by_cost = [&](int x, int y) { return cost[x] > cost[y]; };
    std::stable_sort(order.begin(), order.end(), by_cost);
    std::stable_sort(small.begin(), small.end(), by_cost);
    const int counts[2] = {(int)order.size(), (int)small.size()};
    const int n = counts[0] + counts[1];
    cudaError_t e = cudaSuccess;
    if (counts[0])
        e = cudaMemcpyAsync(b->order_d, order.data(), sizeof(int) * counts[0], cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && counts[1])
        e = cudaMemcpyAsync(b->order_small_d, small.data(), sizeof(int) * counts[1], cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->counters_d + 2, counts, sizeof(counts), cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return b->cuda_fail(e, "work list upload");
    if (n == 0) return LB_OK;
    if (!b->graph || b->graph_chunk != ch) {
        if (b->graph) cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        b->args.chunk = ch;
        cudaGraph_t g = nullptr;
        if ((e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return b->cuda_fail(e, "cudaStreamBeginCapture");
        cudaError_t e1 = cudaMemsetAsync(b->counters_d, 0, 2 * sizeof(int), b->stream);  // both queue heads
        cudaError_t e2 = batch_launch(b);
        e = cudaStreamEndCapture(b->stream, &g);
        if (e1 != cudaSuccess || e2 != cudaSuccess || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return b->cuda_fail(e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e), "batch graph capture");
        }
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return b->cuda_fail(e, "cudaGraphInstantiate");
        b->graph_chunk = ch;
    }
    if ((e = cudaGraphLaunch(b->graph, b->stream)) != cudaSuccess) return b->cuda_fail(e, "cudaGraphLaunch");
    ++b->launches;
    b->in_flight = true;
    b->stale = true;
    return LB_OK;
}

lb_status lb_batch_sync(lb_batch* b) {
    if (!b) return LB_ERR_ARG;
    lb_status st = b->settle();
    if (st != LB_OK) return st;
    for (int s = 0; s < b->p.max_slots; ++s)
        if (b->live[s] && (b->inst[s].status & 1)) return b->fail(LB_ERR_UNSTABLE, "an instance became non-finite");
    return LB_OK;
}

lb_status lb_batch_state(lb_batch* b, int slot, lb_instance_state* o) {
    if (!b || !o || slot < 0 || slot >= b->p.max_slots || !b->live[slot])
        return b ? b->fail(LB_ERR_ARG, "no such slot") : LB_ERR_ARG;
    lb_status st = b->settle();
    if (st != LB_OK) return st;
    const lbk::BatchInst& in = b->inst[slot];
    o->level = in.level;
    o->done = in.done;
    o->status = in.status;
    o->q = b->sets[in.set].q;
    o->dt = in.dt;
    o->omega = in.omega;
    o->tau = b->tau[slot];
    size_t bytes = 0;
    for (auto& r : b->ranges_of[slot]) bytes += (r.second + kAlign - 1) / kAlign * kAlign;
    o->bytes = bytes;
    return LB_OK;
}

lb_status lb_batch_history(lb_batch* b, int slot, double* amp, double* shear, int max, int* n_out) {
    if (!b || !n_out || max < 0 || slot < 0 || slot >= b->p.max_slots || !b->live[slot])
        return b ? b->fail(LB_ERR_ARG, "no such slot") : LB_ERR_ARG;
    lb_status st = b->settle();
    if (st != LB_OK) return st;
    const lbk::BatchInst& in = b->inst[slot];
    const int n = std::min(in.level, max);
    std::vector<float2> h((size_t)std::max(n, 1));
    if (n > 0) {
        const cudaError_t e = cudaMemcpy(h.data(), static_cast<float2*>(b->arena) + in.hist_off,
                                         sizeof(float2) * n, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return b->cuda_fail(e, "history read-back");
    }
    for (int i = 0; i < n; ++i) {
        if (amp) amp[i] = h[i].x;
        if (shear) shear[i] = h[i].y;
    }
    *n_out = n;
    return LB_OK;
}

lb_status lb_batch_fit(lb_batch* b, int slot, double t_start, double floor_rel, double* rate, int* npoints) {
    if (!b || !rate || !npoints) return b ? b->fail(LB_ERR_ARG, "null output") : LB_ERR_ARG;
    int n = 0;
    if (slot < 0 || slot >= b->p.max_slots || !b->live[slot]) return b->fail(LB_ERR_ARG, "no such slot");
    std::vector<double> amp((size_t)std::max(1, b->inst[slot].level));
    lb_status st = lb_batch_history(b, slot, amp.data(), nullptr, (int)amp.size(), &n);
    if (st != LB_OK) return st;
    const double dt = b->inst[slot].dt;
    const double a0 = n > 0 ? std::fabs(amp[0]) : 0.0;
    double s_t = 0, s_l = 0, s_tt = 0, s_tl = 0;
    int m = 0;
    for (int i = 0; i < n; ++i) {
        const double t = i * dt;
        if (t < t_start) continue;
        const double a = std::fabs(amp[i]);
        if (!(a >= floor_rel * a0) || a == 0.0) break;
        const double l = std::log(a);
        s_t += t;
        s_l += l;
        s_tt += t * t;
        s_tl += t * l;
        ++m;
    }
    if (m < 3) return b->fail(LB_ERR_ARG, "fewer than 3 records in the fit window");
    const double den = m * s_tt - s_t * s_t;
    if (!(den > 0)) return b->fail(LB_ERR_ARG, "degenerate fit window");
    *rate = -(m * s_tl - s_t * s_l) / den;
    *npoints = m;
    return LB_OK;
}

size_t lb_batch_bytes_in_use(const lb_batch* b) { return b ? b->ranges.used() : 0; }

long long lb_batch_kernel_launches(const lb_batch* b) { return b ? b->launches : 0; }

}  // extern "C"
