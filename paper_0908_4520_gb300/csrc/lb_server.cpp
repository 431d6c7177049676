// C-ABI of the request loop (lb_server_*): a FIFO queue, admission by device
// memory, continuous batching of small requests in one lb_batch, large
// requests on lattices of their own (second stream), retirement with FP64
// decay fits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "lb.h"

namespace {

thread_local std::string g_server_error;

struct SmallJob {
    lb_request req;
    int slot;
    double admitted;
};

struct LargeJob {
    lb_request req;
    lb_handle* h;
    double admitted;
    size_t bytes;
    double h0;
};

struct History {
    std::vector<double> amp, shear;
};

double fit_rate(const std::vector<double>& amp, double dt, double t_start, double floor_rel, int* npts) {
    *npts = 0;
    if (amp.empty()) return 0.0;
    const double a0 = std::fabs(amp[0]);
    double st = 0, sl = 0, stt = 0, stl = 0;
    int m = 0;
    for (size_t i = 0; i < amp.size(); ++i) {
        const double t = i * dt;
        if (t < t_start) continue;
        const double a = std::fabs(amp[i]);
        if (!(a >= floor_rel * a0) || a == 0.0) break;
        const double l = std::log(a);
        st += t;
        sl += l;
        stt += t * t;
        stl += t * l;
        ++m;
    }
    const double den = m * stt - st * st;
    if (m < 3 || !(den > 0)) return 0.0;
    *npts = m;
    return -(m * stl - st * sl) / den;
}

double shear_ratio(const std::vector<double>& amp, const std::vector<double>& shear) {
    if (amp.empty() || amp[0] == 0.0) return 0.0;
    double m = 0;
    for (double s : shear) m = std::max(m, std::fabs(s));
    return m / std::fabs(amp[0]);
}

}  // namespace

struct lb_server {
    lb_server_params p{};
    lb_batch* batch = nullptr;
    cudaStream_t large_stream = nullptr;
    std::deque<lb_request> queue;
    std::vector<SmallJob> small;
    std::vector<LargeJob> large;
    std::vector<lb_response> finished;
    std::map<long long, History> histories;
    size_t large_bytes = 0;
    std::string err;

    lb_status fail(lb_status s, const std::string& m) {
        err = m;
        return s;
    }
};

namespace {

size_t large_estimate(const lb_instance_desc& d, lb_precision prec) {
    const size_t eb = prec == LB_F32 ? 4 : 2;
    const size_t q = d.quadrature == LB_D2Q16_GH ? 16 : (d.quadrature == LB_D2Q36_GH ? 36 : 64);
    const size_t pitch = ((size_t)d.nx + 16 + 63) / 64 * 64;
    return 2 * q * ((size_t)d.ny + 2) * pitch * eb + sizeof(lb_diag) * ((size_t)d.max_steps + 2) +
           (size_t)d.nx * 16 + (1 << 20);
}

bool is_large(const lb_server* s, const lb_instance_desc& d) { return (long long)d.nx * d.ny >= s->p.large_cells; }

lb_status admit_large(lb_server* s, const lb_request& r, double now, bool* admitted) {
    *admitted = false;
    const size_t est = large_estimate(r.desc, s->p.batch.precision);
    if ((int)s->large.size() >= s->p.max_large || s->large_bytes + est > s->p.budget_bytes) return LB_OK;
    lb_params lp;
    lb_params_default(&lp);
    lp.quadrature = r.desc.quadrature;
    lp.n_eq = r.desc.n_eq;
    lp.nx = r.desc.nx;
    lp.ny = r.desc.ny;
    lp.kn = r.desc.kn;
    lp.precision = s->p.batch.precision;
    lp.kn_convention = s->p.batch.kn_convention;
    lp.diag_capacity = r.desc.max_steps + 2;
    lp.stream = s->large_stream;
    lb_handle* h = nullptr;
    lb_status st = lb_create_ex(&lp, &h);
    if (st != LB_OK) return s->fail(st, std::string("large request: ") + lb_last_error(nullptr));
    st = lb_init_shear_wave(h, r.desc.u0, 0.0);
    if (st != LB_OK) {
        lb_destroy(h);
        return s->fail(st, "large request init");
    }
    lb_info_t info;
    lb_get_info(h, &info);
    s->large.push_back(LargeJob{r, h, now, info.device_bytes, 0.0});
    s->large_bytes += info.device_bytes;
    *admitted = true;
    return LB_OK;
}

}  // namespace

extern "C" {

void lb_server_params_default(lb_server_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    lb_batch_params_default(&p->batch);
    p->chunk = 200;
    p->large_cells = 65536;
    p->budget_bytes = (size_t)8 << 30;
    p->max_large = 4;
}

const char* lb_server_last_error(const lb_server* s) { return s ? s->err.c_str() : g_server_error.c_str(); }

lb_status lb_server_create(const lb_server_params* p, lb_server** out) {
    if (!p || !out || p->chunk < 1 || p->large_cells < 1 || p->max_large < 0) {
        g_server_error = "bad arguments";
        return LB_ERR_ARG;
    }
    lb_server* s = new (std::nothrow) lb_server();
    if (!s) return LB_ERR_NOMEM;
    s->p = *p;
    if (cudaStreamCreateWithFlags(&s->large_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete s;
        g_server_error = "stream creation";
        return LB_ERR_CUDA;
    }
    const lb_status st = lb_batch_create(&p->batch, &s->batch);
    if (st != LB_OK) {
        g_server_error = std::string("batch: ") + lb_batch_last_error(nullptr);
        cudaStreamDestroy(s->large_stream);
        delete s;
        return st;
    }
    *out = s;
    return LB_OK;
}

lb_status lb_server_destroy(lb_server* s) {
    if (!s) return LB_OK;
    for (auto& j : s->large) lb_destroy(j.h);
    lb_batch_destroy(s->batch);
    cudaStreamDestroy(s->large_stream);
    delete s;
    return LB_OK;
}

lb_status lb_server_submit(lb_server* s, const lb_request* r) {
    if (!s || !r) return s ? s->fail(LB_ERR_ARG, "null request") : LB_ERR_ARG;
    if (r->desc.quadrature != LB_D2Q16_GH && r->desc.quadrature != LB_D2Q36_GH && r->desc.quadrature != LB_D2Q64_GH)
        return s->fail(LB_ERR_UNSUPPORTED, "requests use the Gauss-Hermite product sets");
    s->queue.push_back(*r);
    return LB_OK;
}

lb_status lb_server_step(lb_server* s, double now, int* active, int* queued) {
    if (!s) return LB_ERR_ARG;
    lb_status st;
    // 1. admission, FIFO within each kind (a request that does not fit waits; later ones may go)
    for (auto it = s->queue.begin(); it != s->queue.end();) {
        bool admitted = false;
        if (is_large(s, it->desc)) {
            if ((st = admit_large(s, *it, now, &admitted)) != LB_OK) return st;
        } else {
            int slot = -1;
            st = lb_batch_add(s->batch, &it->desc, &slot);
            if (st == LB_OK) {
                s->small.push_back(SmallJob{*it, slot, now});
                admitted = true;
            } else if (st != LB_ERR_BUDGET) {
                return s->fail(st, std::string("batch add: ") + lb_batch_last_error(s->batch));
            }
        }
        it = admitted ? s->queue.erase(it) : std::next(it);
    }
    // 2. one chunk for everything admitted: the batch on its stream, large lattices on theirs
    if (!s->small.empty() && (st = lb_batch_run(s->batch, s->p.chunk)) != LB_OK)
        return s->fail(st, std::string("batch run: ") + lb_batch_last_error(s->batch));
    for (auto& j : s->large) {
        lb_info_t info;
        lb_get_info(j.h, &info);
        const long long left = (long long)j.req.desc.max_steps - info.time_level;
        const int n = (int)std::min<long long>(left, s->p.chunk);
        if (n > 0 && (st = lb_step(j.h, n)) != LB_OK) return s->fail(st, lb_last_error(j.h));
    }
    if ((st = lb_batch_sync(s->batch)) != LB_OK && st != LB_ERR_UNSTABLE) return s->fail(st, "batch sync");
    // 3. retire
    for (size_t k = 0; k < s->small.size();) {
        SmallJob& j = s->small[k];
        lb_instance_state is;
        lb_batch_state(s->batch, j.slot, &is);
        if (!is.done) {
            ++k;
            continue;
        }
        History hist;
        hist.amp.resize(std::max(is.level, 1));
        hist.shear.resize(std::max(is.level, 1));
        int n = 0;
        lb_batch_history(s->batch, j.slot, hist.amp.data(), hist.shear.data(), is.level, &n);
        hist.amp.resize(n);
        hist.shear.resize(n);
        lb_response r{};
        r.id = j.req.id;
        r.arrival = j.req.arrival;
        r.admitted = j.admitted;
        r.finished = now;
        r.levels = is.level;
        r.status = (is.status & 1) ? LB_ERR_UNSTABLE : LB_OK;
        r.decay_rate = fit_rate(hist.amp, is.dt, 5.0 * is.tau, 1e-4, &r.fit_points);
        r.shear_amp = shear_ratio(hist.amp, hist.shear);
        s->finished.push_back(r);
        s->histories[r.id] = std::move(hist);
        lb_batch_remove(s->batch, j.slot);
        s->small[k] = s->small.back();
        s->small.pop_back();
    }
    for (size_t k = 0; k < s->large.size();) {
        LargeJob& j = s->large[k];
        const lb_status sst = lb_synchronize(j.h);
        lb_info_t info;
        lb_get_info(j.h, &info);
        lb_diag last;
        int n = 0;
        lb_diagnostics(j.h, &last, 1, &n);
        if (j.h0 == 0.0) {
            int n0 = 0;
            std::vector<lb_diag> all((size_t)info.records);
            lb_diagnostics(j.h, all.data(), (int)all.size(), &n0);
            if (n0 > 0) j.h0 = all[0].hnorm;
        }
        const double ratio = j.req.desc.stop_ratio;
        const bool stopped = info.time_level > 0 && ratio > 0 && j.h0 > 0 && last.hnorm <= ratio * ratio * j.h0;
        const bool done = sst != LB_OK || info.time_level >= j.req.desc.max_steps || stopped;
        if (!done) {
            ++k;
            continue;
        }
        std::vector<lb_diag> rec((size_t)info.records);
        int nr = 0;
        lb_diagnostics(j.h, rec.data(), (int)rec.size(), &nr);
        History hist;
        for (int i = 0; i < nr; ++i) {
            hist.amp.push_back(rec[i].amp);
            hist.shear.push_back(rec[i].shear);
        }
        lb_response r{};
        r.id = j.req.id;
        r.arrival = j.req.arrival;
        r.admitted = j.admitted;
        r.finished = now;
        r.levels = (int)info.time_level + 1;
        r.status = sst;
        r.decay_rate = fit_rate(hist.amp, info.dt, 5.0 * info.tau, 1e-4, &r.fit_points);
        r.shear_amp = shear_ratio(hist.amp, hist.shear);
        s->finished.push_back(r);
        s->histories[r.id] = std::move(hist);
        s->large_bytes -= j.bytes;
        lb_destroy(j.h);
        s->large[k] = s->large.back();
        s->large.pop_back();
    }
    if (active) *active = (int)(s->small.size() + s->large.size());
    if (queued) *queued = (int)s->queue.size();
    return LB_OK;
}

lb_status lb_server_poll(lb_server* s, lb_response* out, int max, int* n_out) {
    if (!s || !n_out || max < 0 || (!out && max > 0)) return s ? s->fail(LB_ERR_ARG, "bad arguments") : LB_ERR_ARG;
    const int n = std::min<int>(max, (int)s->finished.size());
    for (int i = 0; i < n; ++i) out[i] = s->finished[i];
    s->finished.erase(s->finished.begin(), s->finished.begin() + n);
    *n_out = n;
    return LB_OK;
}

lb_status lb_server_history(lb_server* s, long long id, double* amp, double* shear, int max, int* n_out) {
    if (!s || !n_out) return s ? s->fail(LB_ERR_ARG, "bad arguments") : LB_ERR_ARG;
    auto it = s->histories.find(id);
    if (it == s->histories.end()) return s->fail(LB_ERR_ARG, "no stored history for this id");
    const int n = std::min<int>(max, (int)it->second.amp.size());
    for (int i = 0; i < n; ++i) {
        if (amp) amp[i] = it->second.amp[i];
        if (shear) shear[i] = it->second.shear[i];
    }
    *n_out = n;
    s->histories.erase(it);
    return LB_OK;
}

}  // extern "C"
