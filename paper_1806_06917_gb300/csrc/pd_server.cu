// pd_server.cu -- the request server of include/pd.h: independent simulations
// submitted at any time, admitted by device-memory budget, stepped concurrently
// on their own streams in quanta of graph-replayed explicit steps, and
// collected through tickets. This is the paper's task model (Sec. 2: work
// expressed as futures that a runtime schedules as resources allow) applied to
// whole simulations on one GPU.
//
// Threads: the caller's threads only touch the queue and the ticket records
// (under one mutex). A setup thread builds each admitted simulation (tables,
// neighbour build, initial state) while the worker thread keeps stepping the
// running ones; from then on the worker owns the simulation, its stream and
// event. Every wait of either thread is bounded (event queries with short
// sleeps, timed condition-variable waits).
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pd_tile.cuh"

using namespace pdk;

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    uint64_t ticket = 0;
    pd_grid grid{};
    pd_material mat{};
    pd_run run{};
    int64_t nsteps = 0;
    std::vector<double> u0, v0, bc_val;
    std::vector<uint8_t> bc_kind;
    double *u_out = nullptr, *v_out = nullptr;
    size_t est_bytes = 0;
    // shared with the caller's threads (under the server mutex)
    pd_result res{};
    bool cancel = false;
    // worker only
    pd_sim *sim = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    int64_t inflight = 0;
};

bool ended(int state) { return state == PD_REQ_DONE || state == PD_REQ_CANCELLED || state == PD_REQ_FAILED; }

// Points of the lattice, slots of its tile grid, and an upper bound of the
// device bytes a simulation of it allocates (per-slot state and tables, the
// bond mask, the CSR with every stencil offset counted).
size_t estimate_bytes(const pd_grid &g, const pd_material &mt, int L)
{
    int b[3];
    brick_dims(g.dim, L, b);
    const long long nz = g.dim == 3 ? g.n[2] : 1;
    const long long tiles = (long long)((g.n[0] + b[0] - 1) / b[0]) * ((g.n[1] + b[1] - 1) / b[1]) *
                            ((nz + b[2] - 1) / b[2]);
    const long long slots = tiles << L;
    const long long np = (long long)g.n[0] * g.n[1] * nz;
    const int S = stencil_size(g.dim, g.m);
    const int W = (S + 31) / 32;
    const long long per_slot = 400 + 4LL * W + (mt.model == PD_MODEL_LPS ? 24 : 0);
    return (size_t)(slots * per_slot + np * (8 + 4LL * S) + (1 << 20));
}

// Tile size: the largest 2^L (L = 9..6) that still gives the simulation its
// share of the SMs when max_active simulations run at once.
int choose_tile_log2(const pd_grid &g, int max_active, int sms)
{
    const long long want = (sms + max_active - 1) / max_active;
    const long long nz = g.dim == 3 ? g.n[2] : 1;
    for (int L = 9; L > 6; --L) {
        int b[3];
        brick_dims(g.dim, L, b);
        const long long tiles = (long long)((g.n[0] + b[0] - 1) / b[0]) * ((g.n[1] + b[1] - 1) / b[1]) *
                                ((nz + b[2] - 1) / b[2]);
        if (tiles >= want) return L;
    }
    return 6;
}

}  // namespace

struct pd_server {
    int device = 0, sms = 152;
    size_t budget = 0, used = 0;
    int max_active = 16;
    int quantum = 64;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> queue;
    std::deque<Req *> setup_q;      // admitted, waiting for the setup thread
    std::vector<Req *> ready;       // set up, waiting for the worker
    int in_setup = 0;               // admitted but not yet handed to the worker
    std::condition_variable cv_setup;
    std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker, setup_worker;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
    void run();
    void run_setup();
    int setup(Req *r);
    void teardown(Req *r);
    void finish(Req *r, int state, int error, const char *msg);   // caller holds mu
};

void pd_server::finish(Req *r, int state, int error, const char *msg)
{
    r->res.state = state;
    r->res.error = error;
    r->res.end_s = now();
    if (msg) {
        strncpy(r->res.message, msg, sizeof(r->res.message) - 1);
        r->res.message[sizeof(r->res.message) - 1] = '\0';
    }
    cv_done.notify_all();
}

int pd_server::setup(Req *r)
{
    cudaError_t e = cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "server stream/event");
    int rc = pd_create(&r->sim, &r->grid, &r->mat, &r->run);
    if (rc != PD_OK) return rc;
    if ((rc = pd_build_neighbors(r->sim, r->stream)) != PD_OK) return rc;
    const double *u0 = r->u0.empty() ? nullptr : r->u0.data();
    const double *v0 = r->v0.empty() ? nullptr : r->v0.data();
    if ((u0 || v0) && (rc = pd_set_state(r->sim, u0, v0, r->stream)) != PD_OK) return rc;
    if (!r->bc_kind.empty() && (rc = pd_set_bc(r->sim, r->bc_kind.data(), r->bc_val.data(), r->stream)) != PD_OK)
        return rc;
    int64_t nb = 0;
    if ((rc = pd_bond_count(r->sim, &nb)) != PD_OK) return rc;
    std::lock_guard<std::mutex> lk(mu);
    r->res.bonds = nb;
    return PD_OK;
}

void pd_server::teardown(Req *r)
{
    if (r->stream) cudaStreamSynchronize(r->stream);
    if (r->sim) pd_destroy(r->sim);
    if (r->ev) cudaEventDestroy(r->ev);
    if (r->stream) cudaStreamDestroy(r->stream);
    r->sim = nullptr;
    r->ev = nullptr;
    r->stream = nullptr;
    r->inflight = 0;
}

void pd_server::run_setup()
{
    cudaSetDevice(device);
    while (true) {
        Req *r = nullptr;
        bool cancel = false;
        {
            std::unique_lock<std::mutex> lk(mu);
            while (setup_q.empty() && !stop) cv_setup.wait_for(lk, std::chrono::milliseconds(20));
            if (setup_q.empty()) break;                     // stop with nothing left
            r = setup_q.front();
            setup_q.pop_front();
            cancel = r->cancel || stop;
        }
        int rc = PD_OK;
        char msg[160] = {0};
        if (!cancel) {
            rc = setup(r);
            if (rc != PD_OK) pd_last_error(msg, sizeof(msg));
        }
        if (cancel || rc != PD_OK) teardown(r);
        {
            std::lock_guard<std::mutex> lk(mu);
            if (cancel || rc != PD_OK) {
                used -= r->est_bytes;
                --in_setup;
                if (cancel) finish(r, PD_REQ_CANCELLED, PD_OK, nullptr);
                else finish(r, PD_REQ_FAILED, rc, msg);
            } else {
                ready.push_back(r);
            }
        }
        cv_work.notify_all();
    }
}

void pd_server::run()
{
    cudaSetDevice(device);
    std::vector<Req *> active;
    while (true) {
        std::vector<Req *> admitted;
        {
            std::unique_lock<std::mutex> lk(mu);
            for (Req *r : ready) {
                --in_setup;
                active.push_back(r);
            }
            ready.clear();
            // admission in submission order; the head of the queue waits for memory.
            // Nothing is admitted once stopping (the setup thread may have exited).
            while (!stop && !queue.empty() && (int)active.size() + in_setup < max_active) {
                Req *r = queue.front();
                if (r->cancel) {
                    queue.pop_front();
                    finish(r, PD_REQ_CANCELLED, PD_OK, nullptr);
                    continue;
                }
                if (used + r->est_bytes > budget) break;
                queue.pop_front();
                used += r->est_bytes;
                r->res.state = PD_REQ_RUNNING;
                r->res.start_s = now();
                setup_q.push_back(r);
                ++in_setup;
                admitted.push_back(r);
            }
            if (!admitted.empty()) cv_setup.notify_one();
            if (stop) {
                for (Req *r : queue) finish(r, PD_REQ_CANCELLED, PD_OK, nullptr);
                queue.clear();
                for (Req *r : active) r->cancel = true;
                if (active.empty() && in_setup == 0) break;
            }
            if (active.empty()) {
                cv_work.wait_for(lk, std::chrono::milliseconds(20));
                continue;
            }
        }
        // issue the next quantum of every idle simulation
        for (Req *r : active) {
            if (r->inflight) continue;
            bool cancel;
            int64_t done;
            {
                std::lock_guard<std::mutex> lk(mu);
                cancel = r->cancel;
                done = r->res.steps_done;
            }
            if (cancel || done >= r->nsteps) continue;
            const int64_t q = std::min<int64_t>(quantum, r->nsteps - done);
            int rc = pd_step_explicit(r->sim, q, r->stream);
            cudaError_t e = rc == PD_OK ? cudaEventRecord(r->ev, r->stream) : cudaSuccess;
            if (rc != PD_OK || e != cudaSuccess) {
                char msg[160];
                if (rc == PD_OK) rc = cuda_fail(e, "server event");
                pd_last_error(msg, sizeof(msg));
                std::lock_guard<std::mutex> lk(mu);
                r->cancel = true;
                r->res.error = rc;
                strncpy(r->res.message, msg, sizeof(r->res.message) - 1);
                continue;
            }
            r->inflight = q;
        }
        // collect finished quanta and finished requests
        bool progressed = false;
        for (size_t i = 0; i < active.size();) {
            Req *r = active[i];
            if (r->inflight) {
                const cudaError_t q = cudaEventQuery(r->ev);
                if (q == cudaErrorNotReady) {
                    ++i;
                    continue;
                }
                progressed = true;
                std::lock_guard<std::mutex> lk(mu);
                if (q == cudaSuccess) r->res.steps_done += r->inflight;
                else r->res.error = cuda_fail(q, "server quantum");
                r->inflight = 0;
            }
            bool cancel, complete;
            int err;
            {
                std::lock_guard<std::mutex> lk(mu);
                cancel = r->cancel;
                err = r->res.error;
                complete = r->res.steps_done >= r->nsteps;
            }
            if (!cancel && !complete && err == PD_OK) {
                ++i;
                continue;
            }
            progressed = true;
            int rc = err;
            char msg[160] = {0};
            if (rc == PD_OK && !cancel && (r->u_out || r->v_out)) {
                rc = pd_get_state(r->sim, r->u_out, r->v_out, r->stream);
                if (rc != PD_OK) pd_last_error(msg, sizeof(msg));
            }
            teardown(r);
            {
                std::lock_guard<std::mutex> lk(mu);
                used -= r->est_bytes;
                if (rc != PD_OK) finish(r, PD_REQ_FAILED, rc, msg[0] ? msg : nullptr);
                else finish(r, cancel ? PD_REQ_CANCELLED : PD_REQ_DONE, PD_OK, nullptr);
            }
            active.erase(active.begin() + i);
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

extern "C" {

int pd_server_create(pd_server **out, const pd_server_opts *opts)
{
    if (!out) { set_error("null output"); return PD_EINVAL; }
    *out = nullptr;
    pd_server_opts o = {0, 16, 64};
    if (opts) o = *opts;
    if (o.max_active < 1 || o.max_active > 256) { set_error("max_active must be in [1, 256]"); return PD_EINVAL; }
    if (o.quantum_steps < 1) { set_error("quantum_steps must be >= 1"); return PD_EINVAL; }
    if (o.device_bytes < 0) { set_error("device_bytes must be >= 0"); return PD_EINVAL; }
    std::unique_ptr<pd_server> s(new pd_server());
    PD_CUDA(cudaGetDevice(&s->device));
    PD_CUDA(cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device));
    size_t fr = 0, tot = 0;
    PD_CUDA(cudaMemGetInfo(&fr, &tot));
    s->budget = o.device_bytes > 0 ? (size_t)o.device_bytes : fr / 2;
    s->max_active = o.max_active;
    s->quantum = o.quantum_steps;
    s->t0 = Clock::now();
    pd_server *raw = s.get();
    s->setup_worker = std::thread([raw] { raw->run_setup(); });
    s->worker = std::thread([raw] { raw->run(); });
    *out = s.release();
    return PD_OK;
}

int pd_server_destroy(pd_server *s)
{
    if (!s) return PD_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    s->cv_setup.notify_all();
    if (s->worker.joinable()) s->worker.join();
    if (s->setup_worker.joinable()) s->setup_worker.join();
    delete s;
    return PD_OK;
}

int pd_submit(pd_server *s, const pd_request *rq, uint64_t *ticket)
{
    if (!s || !rq || !ticket) { set_error("null argument"); return PD_EINVAL; }
    int rc = validate_description(&rq->grid, &rq->material, &rq->run);
    if (rc != PD_OK) return rc;
    if (rq->nsteps < 0) { set_error("nsteps must be >= 0"); return PD_EINVAL; }
    if (!rq->bc_kind != !rq->bc_val) { set_error("bc_kind and bc_val go together"); return PD_EINVAL; }
    std::unique_ptr<Req> r(new Req());
    r->grid = rq->grid;
    r->mat = rq->material;
    r->run = rq->run;
    r->nsteps = rq->nsteps;
    if (r->run.tile_log2 == 0) r->run.tile_log2 = choose_tile_log2(r->grid, s->max_active, s->sms);
    r->est_bytes = estimate_bytes(r->grid, r->mat, r->run.tile_log2);
    if (r->est_bytes > s->budget) {
        set_error("request needs about %zu device bytes, more than the server budget of %zu", r->est_bytes,
                  s->budget);
        return PD_EINVAL;
    }
    const size_t n = (size_t)rq->grid.n[0] * rq->grid.n[1] * (rq->grid.dim == 3 ? rq->grid.n[2] : 1) *
                     rq->grid.dim;
    if (rq->u0) r->u0.assign(rq->u0, rq->u0 + n);
    if (rq->v0) r->v0.assign(rq->v0, rq->v0 + n);
    if (rq->bc_kind) {
        r->bc_kind.assign(rq->bc_kind, rq->bc_kind + n);
        r->bc_val.assign(rq->bc_val, rq->bc_val + n);
    }
    r->u_out = rq->u_out;
    r->v_out = rq->v_out;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) { set_error("server is shutting down"); return PD_ESTATE; }
        r->ticket = s->next_ticket++;
        r->res.state = PD_REQ_QUEUED;
        r->res.tile_log2 = r->run.tile_log2;
        r->res.submit_s = s->now();
        *ticket = r->ticket;
        s->queue.push_back(r.get());
        s->reqs.emplace(r->ticket, std::move(r));
    }
    s->cv_work.notify_all();
    return PD_OK;
}

int pd_poll(pd_server *s, uint64_t ticket, pd_result *out)
{
    if (!s || !out) { set_error("null argument"); return PD_EINVAL; }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) { set_error("unknown ticket %llu", (unsigned long long)ticket); return PD_EINVAL; }
    *out = it->second->res;
    return PD_OK;
}

int pd_wait(pd_server *s, uint64_t ticket, double timeout_s, pd_result *out)
{
    if (!s || !out) { set_error("null argument"); return PD_EINVAL; }
    if (!(timeout_s >= 0.0)) { set_error("timeout must be >= 0"); return PD_EINVAL; }
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) { set_error("unknown ticket %llu", (unsigned long long)ticket); return PD_EINVAL; }
    Req *r = it->second.get();
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(std::min(timeout_s, 1e7)));
    while (!ended(r->res.state)) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !ended(r->res.state)) {
            *out = r->res;
            set_error("ticket %llu not done within %g s", (unsigned long long)ticket, timeout_s);
            return PD_ETIMEOUT;
        }
    }
    *out = r->res;
    return PD_OK;
}

int pd_cancel(pd_server *s, uint64_t ticket)
{
    if (!s) { set_error("null server"); return PD_EINVAL; }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) { set_error("unknown ticket %llu", (unsigned long long)ticket); return PD_EINVAL; }
        Req *r = it->second.get();
        r->cancel = true;
        if (r->res.state == PD_REQ_QUEUED) {
            // not admitted yet: it ends here
            for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
                if (*q == r) {
                    s->queue.erase(q);
                    break;
                }
            s->finish(r, PD_REQ_CANCELLED, PD_OK, nullptr);
        }
    }
    s->cv_work.notify_all();
    return PD_OK;
}

}  // extern "C"
