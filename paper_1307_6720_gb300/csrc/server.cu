// Request server: continuous batching of independent equilibrium solves.
//
// A worker thread admits queued requests in arrival order as solver slots
// and device memory free up, keeps solver hierarchies resident between
// requests (one pool of handles per grid shape), and runs every admitted
// request on its handle's own stream, so requests that arrive while others
// are on the GPU overlap with them.  Device memory is budgeted: a new
// hierarchy is created only if the bytes of all resident hierarchies plus
// the new one stay within the budget; otherwise idle hierarchies of other
// shapes are released first, and a request waits until memory frees up.
// A request larger than the whole budget is rejected (MHS_ERR_REJECTED).
// Each request runs exactly the kernels of a solo solve of the same
// problem, so its result does not depend on what else is in flight.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <numeric>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "mhs_internal.h"
#include "solver.h"

namespace mhs {

namespace {

using Clock = std::chrono::steady_clock;

struct ShapeKey {
    int nx, ny, nz;
    double Lx, Ly, Lz;
    bool operator<(const ShapeKey& o) const {
        return std::tie(nx, ny, nz, Lx, Ly, Lz) < std::tie(o.nx, o.ny, o.nz, o.Lx, o.Ly, o.Lz);
    }
};

struct Slot {
    mhs_ctx* h = nullptr;
    ShapeKey key{};
    size_t bytes = 0;
    bool busy = false;
    Clock::time_point last_used;
};

struct Request {
    long long ticket = 0;
    mhs_request req{};
    std::vector<double> bz;   // copy of B_z taken at submission
    Clock::time_point t_submit, t_start, t_done;
    int state = 0;            // 0 queued, 1 running, 2 done
    mhs_status status = MHS_OK;
    mhs_solve_info info{};
    Slot* slot = nullptr;
    cudaEvent_t done_ev = nullptr;
};

}  // namespace

struct Server {
    size_t budget = 0, in_use = 0;
    int max_inflight = 16;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> queue;
    std::vector<std::shared_ptr<Request>> running;
    std::map<long long, std::shared_ptr<Request>> all;
    std::vector<std::unique_ptr<Slot>> slots;
    std::vector<double> latencies_ms;
    long long next_ticket = 1;
    long long completed = 0, rejected = 0;
    Clock::time_point t_first_submit, t_last_done;
    bool have_first = false, stop = false;
    int device = 0;
    std::thread worker;
    std::string last_error;

    void run();
    Slot* acquire(const mhs_request& r, bool* too_big);
    void start(const std::shared_ptr<Request>& q);
    void finish(const std::shared_ptr<Request>& q);
};

namespace {

size_t handle_bytes(mhs_ctx* c) { return handle_bytes_held(c); }

size_t estimate_bytes(const mhs_request& r) { return handle_bytes_estimate(r.nx, r.ny, r.nz, r.Lx, r.Ly, r.Lz); }

}  // namespace

// Free slot for the request's shape, creating one within the budget if
// needed (releasing idle hierarchies of other shapes, oldest first).
Slot* Server::acquire(const mhs_request& r, bool* too_big) {
    const ShapeKey key{r.nx, r.ny, r.nz, r.Lx, r.Ly, r.Lz};
    *too_big = false;
    for (auto& s : slots)
        if (!s->busy && !(s->key < key) && !(key < s->key)) return s.get();
    const size_t need = estimate_bytes(r);
    if (need > budget) {
        *too_big = true;
        return nullptr;
    }
    while (in_use + need > budget) {
        Slot* victim = nullptr;
        for (auto& s : slots)
            if (!s->busy && (!victim || s->last_used < victim->last_used)) victim = s.get();
        if (!victim) return nullptr;   // wait for a running request to finish
        in_use -= victim->bytes;
        mhs_destroy(victim->h);
        slots.erase(std::find_if(slots.begin(), slots.end(), [&](auto& p) { return p.get() == victim; }));
    }
    mhs_handle h = nullptr;
    const mhs_status s = mhs_create(r.nx, r.ny, r.nz, r.Lx, r.Ly, r.Lz, r.alpha, &r.xi, &r.atm, &h);
    if (s != MHS_OK) throw Error(s, std::string("server: ") + mhs_last_error());
    auto slot = std::make_unique<Slot>();
    slot->h = h;
    slot->key = key;
    slot->bytes = std::max(handle_bytes(h), need);
    MHS_CUDA(cudaStreamCreateWithFlags(&h->bstream, cudaStreamNonBlocking));
    in_use += slot->bytes;
    slots.push_back(std::move(slot));
    return slots.back().get();
}

// Enqueue the request's whole solve and field recovery on its slot's stream.
void Server::start(const std::shared_ptr<Request>& q) {
    mhs_ctx* c = q->slot->h;
    const mhs_request& r = q->req;
    c->stream = c->bstream;
    mhs_status s = mhs_set_params(c, r.alpha, &r.xi, &r.atm);
    if (s != MHS_OK) throw Error(s, mhs_last_error());
    // options stored by the autotuner for this problem class, if any
    mhs_solver_opts tuned;
    if (tune_lookup(c, r.mode, &tuned) && std::memcmp(&tuned, &c->opts, sizeof tuned) != 0) {
        c->opts = tuned;
        choose_cuts(c);   // the handle keeps a captured solve per option set
    }
    const Geom& g2 = c->h2.g[0];
    MHS_CUDA(cudaMemcpy2DAsync(c->bz, g2.px * sizeof(double), q->bz.data(), g2.nx * sizeof(double),
                               g2.nx * sizeof(double), g2.ny, cudaMemcpyHostToDevice, c->stream));
    c->have_bz = true;
    solve_begin(c, r.tol, r.mode);
    const Geom& g = c->h3.g[0];
    if (r.phi)
        MHS_CUDA(cudaMemcpy2DAsync(r.phi, g.nx * sizeof(double), c->h3.d[0].u, g.px * sizeof(double),
                                   g.nx * sizeof(double), size_t(g.ny) * g.nz, cudaMemcpyDefault, c->stream));
    double* outs[5] = {r.Bx, r.By, r.Bz, r.p, r.rho};
    bool any = false;
    for (double* o : outs) any = any || o;
    if (any) {
        ensure_field_buffers(c);
        launch_fields(g, c->alpha, c->atm, c->prof, c->h3.d[0].u, c->fld[0], c->fld[1], c->fld[2], c->fld[3],
                      c->fld[4], (c->opts.flags & MHS_FLAG_BZ_MIMETIC) ? 1 : 0, c->stream);
        for (int k = 0; k < 5; ++k)
            if (outs[k])
                MHS_CUDA(cudaMemcpy2DAsync(outs[k], g.nx * sizeof(double), c->fld[k], g.px * sizeof(double),
                                           g.nx * sizeof(double), size_t(g.ny) * g.nz, cudaMemcpyDefault,
                                           c->stream));
    }
    if (!q->done_ev) MHS_CUDA(cudaEventCreateWithFlags(&q->done_ev, cudaEventDisableTiming));
    MHS_CUDA(cudaEventRecord(q->done_ev, c->stream));
}

void Server::finish(const std::shared_ptr<Request>& q) {
    mhs_ctx* c = q->slot->h;
    try {
        q->status = solve_end(c, q->req.tol, q->req.mode, &q->info);
    } catch (const Error& e) {
        q->status = e.status;
    }
    cudaEventDestroy(q->done_ev);
    q->done_ev = nullptr;
    q->slot->busy = false;
    q->slot->last_used = Clock::now();
    q->slot = nullptr;
}

void Server::run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
        // admit queued requests in arrival order while slots and memory allow
        while (!queue.empty() && int(running.size()) < max_inflight) {
            auto q = queue.front();
            bool too_big = false;
            Slot* s = nullptr;
            try {
                s = acquire(q->req, &too_big);
            } catch (const Error& e) {
                q->status = e.status;
                last_error = e.what();
                too_big = true;
            }
            if (too_big) {
                queue.pop_front();
                if (q->status == MHS_OK) q->status = MHS_ERR_REJECTED;
                q->state = 2;
                q->t_done = Clock::now();
                ++rejected;
                cv_done.notify_all();
                continue;
            }
            if (!s) break;   // out of memory budget until something finishes
            queue.pop_front();
            s->busy = true;
            q->slot = s;
            q->state = 1;
            q->t_start = Clock::now();
            try {
                start(q);
                running.push_back(q);
            } catch (const Error& e) {
                q->status = e.status;
                last_error = e.what();
                q->state = 2;
                q->t_done = Clock::now();
                s->busy = false;
                q->slot = nullptr;
                cv_done.notify_all();
            }
        }
        // retire finished requests
        bool progressed = false;
        for (size_t k = 0; k < running.size();) {
            auto q = running[k];
            const cudaError_t e = cudaEventQuery(q->done_ev);
            if (e == cudaErrorNotReady) {
                ++k;
                continue;
            }
            if (e != cudaSuccess) (void)cudaGetLastError();
            finish(q);
            q->state = 2;
            q->t_done = Clock::now();
            latencies_ms.push_back(std::chrono::duration<double, std::milli>(q->t_done - q->t_submit).count());
            ++completed;
            t_last_done = q->t_done;
            running.erase(running.begin() + k);
            progressed = true;
        }
        if (progressed) cv_done.notify_all();
        if (stop && queue.empty() && running.empty()) break;
        if (running.empty() && queue.empty()) {
            cv_work.wait(lk);
        } else if (!progressed) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        }
    }
}

}  // namespace mhs

struct mhs_server {
    mhs::Server s;
};

namespace {
thread_local std::string g_server_error;
}

extern "C" {

mhs_status mhs_server_create(size_t budget_bytes, int max_inflight, mhs_server_t* out) {
    if (!out || budget_bytes == 0 || max_inflight <= 0 || max_inflight > 1024) return MHS_ERR_INVALID_ARG;
    auto* sv = new (std::nothrow) mhs_server();
    if (!sv) return MHS_ERR_OUT_OF_MEMORY;
    sv->s.budget = budget_bytes;
    sv->s.max_inflight = max_inflight;
    if (cudaGetDevice(&sv->s.device) != cudaSuccess) {
        (void)cudaGetLastError();
        delete sv;
        return MHS_ERR_CUDA;
    }
    sv->s.worker = std::thread([sv] { sv->s.run(); });
    *out = sv;
    return MHS_OK;
}

mhs_status mhs_server_submit(mhs_server_t sv, const mhs_request* r, long long* ticket) {
    if (!sv || !r || !ticket || !r->bz) return MHS_ERR_INVALID_ARG;
    if (!(r->tol > 0 && r->tol < 1) || (r->mode != MHS_FP64 && r->mode != MHS_MIXED)) return MHS_ERR_INVALID_ARG;
    for (int n : {r->nx, r->ny, r->nz})
        if (n < 5 || n % 2 == 0) return MHS_ERR_INVALID_ARG;
    auto q = std::make_shared<mhs::Request>();
    q->req = *r;
    if (q->req.atm.g == 0.0 && q->req.atm.mu0 == 0.0) q->req.atm = mhs_atmos_params{1.0, 0.5, 150.0, 5.0, 10.0};
    q->bz.resize(size_t(r->nx) * r->ny);
    if (cudaMemcpy(q->bz.data(), r->bz, q->bz.size() * sizeof(double), cudaMemcpyDefault) != cudaSuccess) {
        (void)cudaGetLastError();
        return MHS_ERR_CUDA;
    }
    for (int j = 1; j < r->ny - 1; ++j)
        for (int i = 1; i < r->nx - 1; ++i)
            if (!std::isfinite(q->bz[size_t(j) * r->nx + i])) return MHS_ERR_NONFINITE;
    q->t_submit = mhs::Clock::now();
    std::lock_guard<std::mutex> lk(sv->s.mu);
    q->ticket = sv->s.next_ticket++;
    if (!sv->s.have_first) {
        sv->s.t_first_submit = q->t_submit;
        sv->s.have_first = true;
    }
    sv->s.queue.push_back(q);
    sv->s.all[q->ticket] = q;
    *ticket = q->ticket;
    sv->s.cv_work.notify_one();
    return MHS_OK;
}

static void report(const mhs::Request& q, mhs_solve_info* info, mhs_status* st, double* latency_ms) {
    if (info) *info = q.info;
    if (st) *st = q.status;
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(q.t_done - q.t_submit).count();
}

mhs_status mhs_server_poll(mhs_server_t sv, long long ticket, int* done, mhs_solve_info* info, mhs_status* st,
                           double* latency_ms) {
    if (!sv || !done) return MHS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->s.mu);
    auto it = sv->s.all.find(ticket);
    if (it == sv->s.all.end()) return MHS_ERR_INVALID_ARG;
    *done = it->second->state == 2;
    if (*done) {
        report(*it->second, info, st, latency_ms);
        sv->s.all.erase(it);
    }
    return MHS_OK;
}

mhs_status mhs_server_wait(mhs_server_t sv, long long ticket, double timeout_s, mhs_solve_info* info, mhs_status* st,
                           double* latency_ms) {
    if (!sv) return MHS_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(sv->s.mu);
    auto it = sv->s.all.find(ticket);
    if (it == sv->s.all.end()) return MHS_ERR_INVALID_ARG;
    auto q = it->second;
    const auto deadline = mhs::Clock::now() + std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9);
    while (q->state != 2)
        if (sv->s.cv_done.wait_until(lk, deadline) == std::cv_status::timeout && q->state != 2) return MHS_ERR_TIMEOUT;
    report(*q, info, st, latency_ms);
    sv->s.all.erase(ticket);
    return MHS_OK;
}

mhs_status mhs_server_stats(mhs_server_t sv, mhs_server_stats_t* out) {
    if (!sv || !out) return MHS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->s.mu);
    std::vector<double> l = sv->s.latencies_ms;
    std::sort(l.begin(), l.end());
    auto pct = [&](double p) { return l.empty() ? 0.0 : l[std::min(l.size() - 1, size_t(p * (l.size() - 1) + 0.5))]; };
    out->completed = sv->s.completed;
    out->rejected = sv->s.rejected;
    out->queued = (long long)sv->s.queue.size();
    out->running = (long long)sv->s.running.size();
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    out->mean_ms = l.empty() ? 0.0 : std::accumulate(l.begin(), l.end(), 0.0) / double(l.size());
    const double span = sv->s.completed > 0
                            ? std::chrono::duration<double>(sv->s.t_last_done - sv->s.t_first_submit).count()
                            : 0.0;
    out->solves_per_s = span > 0 ? double(sv->s.completed) / span : 0.0;
    out->device_bytes = sv->s.in_use;
    out->resident_hierarchies = (long long)sv->s.slots.size();
    return MHS_OK;
}

void mhs_server_destroy(mhs_server_t sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->s.mu);
        sv->s.stop = true;
        sv->s.cv_work.notify_all();
    }
    sv->s.worker.join();
    for (auto& s : sv->s.slots) mhs_destroy(s->h);
    delete sv;
}

}  // extern "C"
