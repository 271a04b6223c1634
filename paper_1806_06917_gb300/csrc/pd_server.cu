// pd_server.cu -- the request server of include/pd.h: independent simulations
// submitted at any time (refused with PD_EBUSY while max_queued wait), admitted
// by device-memory budget, stepped concurrently in quanta and collected through
// tickets. Packed mode (the default): the FP32C PMB requests without breaking
// and the LPS requests without partial volume (m <= 3) advance together, one
// launch of the packed kernel (pd_packed.cu) per step of a quantum, the
// quantum's launches replayed from a captured graph, two quanta in flight; the
// other requests, and all of them in streams mode, step on their own streams in
// quanta of graph-replayed explicit steps, with a measured (tile, threads per
// pair) choice cached per request class. This is the paper's task model (Sec. 2:
// work expressed as futures that a runtime schedules as resources allow) applied
// to whole simulations on one GPU.
//
// Threads: the caller's threads only touch the queue and the ticket records
// (under one mutex). A setup thread builds each admitted simulation (tables,
// neighbour build, initial state, the packed kernel's LPS tables) while the
// worker thread keeps stepping the running ones; from then on the worker owns
// the simulation, its stream and event. Every wait of either thread is bounded
// (event queries with short sleeps, timed condition-variable waits), and so is
// every device-side wait of the packed kernel (PD_ETIMEOUT).
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <algorithm>
#include <map>
#include <tuple>

#include "pd_packed.cuh"

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
    bool packed = false;            // stepped by the packed kernel (else on its own stream)
    int64_t pk_pending = 0;         // steps in packed quanta still in flight
    bool tune = false;              // tile and threads per pair from the server's measured choices
    unsigned *dil_done = nullptr;   // LPS in the packed kernel: per-tile dilatation flags
    int pack_kind = 0;
};

bool ended(int state) { return state == PD_REQ_DONE || state == PD_REQ_CANCELLED || state == PD_REQ_FAILED; }

// Points of the lattice, slots of its tile grid, and an upper bound of the
// device bytes a simulation of it allocates (per-slot state and tables, the
// bond mask, the CSR with every stencil offset counted, the host-transfer
// staging of two fields each way).
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
    return (size_t)(slots * per_slot + np * (8 + 96 + 4LL * S) + (1 << 20));
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
    // the packed kernel: device request table for max_active requests, its
    // pinned host staging, counters and status; graphs of the rounds by
    // (rounds, grid, shared memory)
    int mode = PD_SERVE_PACKED;
    long long wait_ns = 2000000000LL;
    int stall = 0;
    int pack_max_tiles = 0;       // requests of more tiles than this are not packed (0: no limit)
    int max_queued = 0;           // pd_submit refuses while this many wait (0: no limit)
    // two of each, so that the next quantum is issued while the last one runs
    cudaStream_t pk_stream = nullptr;
    cudaEvent_t pk_ev[2] = {nullptr, nullptr};
    PackReq *d_req[2] = {nullptr, nullptr}, *h_req[2] = {nullptr, nullptr};
    int *d_idx[2] = {nullptr, nullptr}, *h_idx[2] = {nullptr, nullptr};   // offA, offB, nsteps
    unsigned *d_counters[2] = {nullptr, nullptr}, *d_status[2] = {nullptr, nullptr};
    unsigned *h_status[2] = {nullptr, nullptr};
    std::map<std::tuple<int, int, size_t, int, int>, cudaGraphExec_t> graphs;   // (rounds, grid, smem, buffer,
                                                                                // table version)
    // the packed kernel's LPS tables (PackTable.tabs), each horizon's taken from
    // the first simulation of that horizon set up; a later one whose tables differ
    // is not packed. tab_version counts the fills (graphs hold the tables they
    // were captured with).
    std::mutex tab_mu;
    std::vector<float4> pk_tabs = std::vector<float4>(PACK_TAB_N, make_float4(0.f, 0.f, 0.f, 0.f));
    bool tab_filled[PACK_LPS_MMAX + 1] = {};
    int tab_version = 0;
    struct PkQuantum {
        int buf;
        std::vector<std::pair<Req *, int>> list;   // requests and their steps
    };
    std::deque<PkQuantum> pk_q;                    // in flight, oldest first (at most 2)
    // measured (tile_log2, pair_threads) of the requests on their own streams, by
    // dimension, horizon, model, precision, state, integrator and size class
    // (log2 of the points), measured once per class with pd_tune
    std::mutex tune_mu;
    std::map<std::tuple<int, int, int, int, int, int, int>, std::pair<int, int>> tuned;
    int pk_init();
    void pk_free();
    int pk_issue(std::vector<Req *> &active);
    void pk_collect();

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
    if (r->tune) {
        const long long np = (long long)r->grid.n[0] * r->grid.n[1] * (r->grid.dim == 3 ? r->grid.n[2] : 1);
        int cls = 0;
        while ((1LL << (cls + 1)) <= np) ++cls;
        const auto key = std::make_tuple(r->grid.dim, r->grid.m, r->mat.model, r->run.precision, r->run.state,
                                         r->run.integrator, cls);
        std::pair<int, int> choice{0, 0};
        bool have = false;
        {
            std::lock_guard<std::mutex> lk(tune_mu);
            auto it = tuned.find(key);
            if (it != tuned.end()) {
                choice = it->second;
                have = true;
            }
        }
        if (!have) {
            int32_t tl = 0, pt = 0;
            pd_run rr = r->run;
            rr.tile_log2 = 0;
            rr.pair_threads = 0;
            if (pd_tune(&r->grid, &r->mat, &rr, 5, &tl, &pt, nullptr) == PD_OK) {
                choice = {tl, pt};
                std::lock_guard<std::mutex> lk(tune_mu);
                tuned[key] = choice;
            }
        }
        if (choice.first) {
            r->run.tile_log2 = choice.first;
            r->run.pair_threads = choice.second;
            std::lock_guard<std::mutex> lk(mu);
            r->res.tile_log2 = choice.first;
        }
    }
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
    if (mode == PD_SERVE_PACKED) {
        PackInfo pi;
        if ((rc = sim_pack_info(r->sim, &pi)) != PD_OK) return rc;
        if (pi.eligible && pi.kind == PK_LPS) {
            // its tables into the packed kernel's parameter bank (or the same already there)
            const size_t n = 3 * (size_t)pack_lps_stencil(pi.m);
            const int o0 = pack_tab_offset(pi.m, 0), o1 = pack_tab_offset(pi.m, 1);
            std::lock_guard<std::mutex> lk(tab_mu);
            if (!tab_filled[pi.m]) {
                std::copy(pi.htab_dil, pi.htab_dil + n, pk_tabs.begin() + o0);
                std::copy(pi.htab_force, pi.htab_force + n, pk_tabs.begin() + o1);
                tab_filled[pi.m] = true;
                ++tab_version;
            } else if (memcmp(pi.htab_dil, pk_tabs.data() + o0, n * sizeof(float4)) != 0 ||
                       memcmp(pi.htab_force, pk_tabs.data() + o1, n * sizeof(float4)) != 0) {
                pi.eligible = 0;
            }
        }
        if (pi.eligible) {
            r->packed = true;
            r->pack_kind = pi.kind;
            if (pi.kind == PK_LPS) {
                cudaError_t e = lib_malloc(reinterpret_cast<void **>(&r->dil_done), sizeof(unsigned) * pi.ntiles,
                                           r->stream);
                if (e == cudaSuccess)
                    e = cudaMemsetAsync(r->dil_done, 0, sizeof(unsigned) * pi.ntiles, r->stream);
                if (e != cudaSuccess) return cuda_fail(e, "server dilatation flags");
            }
        }
    }
    // everything above is in place before the worker (another stream) steps it
    e = cudaStreamSynchronize(r->stream);
    if (e != cudaSuccess) return cuda_fail(e, "server setup");
    std::lock_guard<std::mutex> lk(mu);
    r->res.bonds = nb;
    r->res.pair_threads = r->run.pair_threads;
    return PD_OK;
}

void pd_server::teardown(Req *r)
{
    if (r->dil_done) lib_free(r->dil_done, r->stream);
    r->dil_done = nullptr;
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
        // the packed requests: collect a finished quantum, issue the next
        pk_collect();
        if (pk_issue(active) != PD_OK) {
            char msg[160];
            pd_last_error(msg, sizeof(msg));
            std::lock_guard<std::mutex> lk(mu);
            for (Req *r : active)
                if (r->packed && !r->res.error) {
                    r->res.error = PD_ECUDA;
                    strncpy(r->res.message, msg, sizeof(r->res.message) - 1);
                }
        }
        // issue the next quantum of every idle simulation on its own stream
        for (Req *r : active) {
            if (r->inflight || r->packed) continue;
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
            if (r->pk_pending > 0) {
                ++i;                                        // in a packed quantum in flight
                continue;
            }
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

int pd_server::pk_init()
{
    const int n = max_active;
    PD_CUDA(cudaStreamCreateWithFlags(&pk_stream, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) {
        PD_CUDA(cudaEventCreateWithFlags(&pk_ev[k], cudaEventDisableTiming));
        PD_CUDA(cudaMalloc(&d_req[k], sizeof(PackReq) * n));
        PD_CUDA(cudaMallocHost(&h_req[k], sizeof(PackReq) * n));
        PD_CUDA(cudaMalloc(&d_idx[k], sizeof(int) * (3 * n + 2)));
        PD_CUDA(cudaMallocHost(&h_idx[k], sizeof(int) * (3 * n + 2)));
        PD_CUDA(cudaMalloc(&d_counters[k], sizeof(unsigned) * quantum));
        PD_CUDA(cudaMalloc(&d_status[k], sizeof(unsigned) * 4));
        PD_CUDA(cudaMallocHost(&h_status[k], sizeof(unsigned) * 4));
        memset(h_status[k], 0, sizeof(unsigned) * 4);
    }
    return PD_OK;
}

void pd_server::pk_free()
{
    if (pk_stream) cudaStreamSynchronize(pk_stream);
    for (auto &g : graphs) cudaGraphExecDestroy(g.second);
    graphs.clear();
    for (int k = 0; k < 2; ++k) {
        cudaFree(d_req[k]);
        cudaFreeHost(h_req[k]);
        cudaFree(d_idx[k]);
        cudaFreeHost(h_idx[k]);
        cudaFree(d_counters[k]);
        cudaFree(d_status[k]);
        cudaFreeHost(h_status[k]);
        if (pk_ev[k]) cudaEventDestroy(pk_ev[k]);
    }
    if (pk_stream) cudaStreamDestroy(pk_stream);
}

// The next packed quantum, issued while the one before it may still run (two
// in flight at most, in two sets of buffers): every packed request that is not
// cancelled, failed or done takes part with min(quantum, steps left after the
// quantum in flight) steps, and its simulation's bookkeeping (staging parity,
// step count) advances now, at issue. Requests are sorted by their step count
// (descending), so that those still stepping in round s are a prefix of the
// table; entries past the last request have no steps. The rounds are replayed
// from a captured graph (memsets of the counters and status, the round
// launches, the status read-back), cached by (rounds, grid, shared memory,
// buffer set).
int pd_server::pk_issue(std::vector<Req *> &active)
{
    if (pk_q.size() >= 2) return PD_OK;
    const int buf = pk_q.empty() ? 0 : 1 - pk_q.back().buf;
    std::vector<std::pair<Req *, int>> list;
    {
        std::lock_guard<std::mutex> lk(mu);
        for (Req *r : active) {
            const int64_t left = r->nsteps - r->res.steps_done - r->pk_pending;
            if (r->packed && !r->cancel && r->res.error == PD_OK && left > 0)
                list.emplace_back(r, (int)std::min<int64_t>(quantum, left));
        }
    }
    if (list.empty()) return PD_OK;
    std::stable_sort(list.begin(), list.end(), [](const std::pair<Req *, int> &x, const std::pair<Req *, int> &y) {
        return x.second > y.second;
    });
    const int n = max_active;
    int *offA = h_idx[buf], *offB = h_idx[buf] + (n + 1), *nst = h_idx[buf] + 2 * (n + 1);
    offA[0] = offB[0] = 0;
    size_t smem = 0;
    memset(h_req[buf], 0, sizeof(PackReq) * n);
    for (int i = 0; i < n; ++i) {
        int na = 0, nb = 0;
        nst[i] = 0;
        if (i < (int)list.size()) {
            PackInfo pi;
            int rc = sim_pack_info(list[i].first->sim, &pi);
            if (rc != PD_OK) return rc;
            if (!pi.eligible) { set_error("a packed request is no longer eligible"); return PD_ESTATE; }
            PackReq &q = h_req[buf][i];
            q.a[0] = pi.a[0];
            q.a[1] = pi.a[1];
            q.kind = pi.kind;
            q.split = pi.split;
            q.ntiles = pi.ntiles;
            q.nsteps = list[i].second;
            q.cur0 = pi.cur;
            q.vhalf0 = pi.vhalf;
            q.cd0 = pi.cd0;
            q.dil_done = list[i].first->dil_done;
            q.step0 = pi.step;
            if (pi.kind == PK_LPS) {
                q.tab_dil = pack_tab_offset(pi.m, 0);
                q.tab_force = pack_tab_offset(pi.m, 1);
            }
            nst[i] = q.nsteps;
            na = pi.ntiles;
            nb = pi.kind == PK_LPS ? pi.ntiles : 0;
            smem = std::max(smem, pi.smem);
        }
        offA[i + 1] = offA[i] + na;
        offB[i + 1] = offB[i] + nb;
    }
    const int rounds = list[0].second;
    int ctas = 0;
    int rc = pack_occupancy(smem, &ctas);
    if (rc != PD_OK) return rc;
    if (ctas < 1) { set_error("the packed kernel does not fit an SM with %zu bytes of shared memory", smem); return PD_EINVAL; }
    const int grid = ctas * sms;
    PD_CUDA(cudaMemcpyAsync(d_req[buf], h_req[buf], sizeof(PackReq) * n, cudaMemcpyHostToDevice, pk_stream));
    PD_CUDA(cudaMemcpyAsync(d_idx[buf], h_idx[buf], sizeof(int) * (3 * n + 2), cudaMemcpyHostToDevice, pk_stream));
    int version;
    {
        std::lock_guard<std::mutex> lk(tab_mu);
        version = tab_version;
    }
    const auto key = std::make_tuple(rounds, grid, smem, buf, version);
    auto it = graphs.find(key);
    if (it == graphs.end()) {
        // (about 15 KB of parameters: on the heap, copied into the launches)
        std::unique_ptr<PackTable> tp(new PackTable());
        PackTable &t = *tp;
        {
            std::lock_guard<std::mutex> lk(tab_mu);
            std::copy(pk_tabs.begin(), pk_tabs.end(), t.tabs);
        }
        t.req = d_req[buf];
        t.offA = d_idx[buf];
        t.offB = d_idx[buf] + (n + 1);
        t.nsteps = d_idx[buf] + 2 * (n + 1);
        t.counters = d_counters[buf];
        t.status = d_status[buf];
        t.wait_ns = wait_ns;
        t.nreq = n;
        t.stall = stall;
        PD_CUDA(cudaStreamBeginCapture(pk_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaMemsetAsync(d_counters[buf], 0, sizeof(unsigned) * rounds, pk_stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_status[buf], 0, sizeof(unsigned) * 4, pk_stream);
        int lrc = e == cudaSuccess ? pack_launch_rounds(t, rounds, grid, smem, pk_stream) : PD_OK;
        if (e == cudaSuccess && lrc == PD_OK)
            e = cudaMemcpyAsync(h_status[buf], d_status[buf], sizeof(unsigned) * 4, cudaMemcpyDeviceToHost,
                                pk_stream);
        cudaGraph_t graph = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(pk_stream, &graph);
        if (e == cudaSuccess) e = ee;
        cudaGraphExec_t exec = nullptr;
        if (e == cudaSuccess && lrc == PD_OK) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (lrc != PD_OK) return lrc;
        if (e != cudaSuccess) return cuda_fail(e, "packed quantum graph");
        it = graphs.emplace(key, exec).first;
    }
    PD_CUDA(cudaGraphLaunch(it->second, pk_stream));
    PD_CUDA(cudaEventRecord(pk_ev[buf], pk_stream));
    for (auto &x : list) {
        sim_pack_advance(x.first->sim, x.second);
        x.first->pk_pending += x.second;
    }
    pk_q.push_back(PkQuantum{buf, list});
    return PD_OK;
}

// The oldest packed quantum, once finished: its steps count, or, if a
// device-side wait ran out, every request of the quantum fails with
// PD_ETIMEOUT (their states are partly stepped). A test stall applies to the
// first quantum only.
void pd_server::pk_collect()
{
    while (!pk_q.empty()) {
        PkQuantum &pq = pk_q.front();
        const cudaError_t q = cudaEventQuery(pk_ev[pq.buf]);
        if (q == cudaErrorNotReady) return;
        const unsigned code = q == cudaSuccess ? h_status[pq.buf][0] : (unsigned)PACK_OK;
        char msg[160] = {0};
        if (q != cudaSuccess) {
            cuda_fail(q, "packed quantum");
            pd_last_error(msg, sizeof(msg));
        } else if (code != PACK_OK) {
            const unsigned *st = h_status[pq.buf];
            snprintf(msg, sizeof(msg), "packed kernel: a dilatation wait ran out after %lld ns (table entry %u, tile "
                     "%u, round %u)", wait_ns, st[1], st[2], st[3]);
        }
        {
            std::lock_guard<std::mutex> lk(mu);
            for (auto &x : pq.list) {
                Req *r = x.first;
                r->pk_pending -= x.second;
                if (q == cudaSuccess && code == PACK_OK) {
                    r->res.steps_done += x.second;
                } else if (r->res.error == PD_OK) {
                    r->res.error = q != cudaSuccess ? PD_ECUDA : PD_ETIMEOUT;
                    strncpy(r->res.message, msg, sizeof(r->res.message) - 1);
                }
            }
        }
        pk_q.pop_front();
        if (stall) {
            stall = 0;
            for (auto &g : graphs) cudaGraphExecDestroy(g.second);
            graphs.clear();
        }
    }
}

extern "C" {

int pd_server_create(pd_server **out, const pd_server_opts *opts)
{
    if (!out) { set_error("null output"); return PD_EINVAL; }
    *out = nullptr;
    pd_server_opts o = {0, 16, 64, PD_SERVE_PACKED, 0, 0, 0, 0, 0};
    if (opts) o = *opts;
    if (o.max_active < 1 || o.max_active > 256) { set_error("max_active must be in [1, 256]"); return PD_EINVAL; }
    if (o.quantum_steps < 1 || o.quantum_steps > 4096) { set_error("quantum_steps must be in [1, 4096]"); return PD_EINVAL; }
    if (o.device_bytes < 0) { set_error("device_bytes must be >= 0"); return PD_EINVAL; }
    if (o.mode != PD_SERVE_PACKED && o.mode != PD_SERVE_STREAMS) { set_error("unknown server mode"); return PD_EINVAL; }
    if (o.wait_limit_ms < 0) { set_error("wait_limit_ms must be >= 0"); return PD_EINVAL; }
    if (o.pack_max_tiles < 0) { set_error("pack_max_tiles must be >= 0"); return PD_EINVAL; }
    if (o.max_queued < 0) { set_error("max_queued must be >= 0"); return PD_EINVAL; }
    if (o.reserved != 0) { set_error("pd_server_opts.reserved must be 0"); return PD_EINVAL; }
    std::unique_ptr<pd_server> s(new pd_server());
    PD_CUDA(cudaGetDevice(&s->device));
    PD_CUDA(cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device));
    size_t fr = 0, tot = 0;
    PD_CUDA(cudaMemGetInfo(&fr, &tot));
    s->budget = o.device_bytes > 0 ? (size_t)o.device_bytes : fr / 2;
    s->max_active = o.max_active;
    s->quantum = o.quantum_steps;
    s->mode = o.mode;
    s->wait_ns = 1000000LL * (o.wait_limit_ms > 0 ? o.wait_limit_ms : 2000);
    s->stall = o.test_stall ? 1 : 0;
    s->pack_max_tiles = o.pack_max_tiles;
    s->max_queued = o.max_queued;
    if (s->mode == PD_SERVE_PACKED) {
        const int rc = s->pk_init();
        if (rc != PD_OK) {
            s->pk_free();
            return rc;
        }
    }
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
    s->pk_free();
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
    // FP32C PMB without breaking and LPS without partial volume go to the packed
    // kernel, which runs 2^9-point tiles and its own threads per point pair
    // (LPS up to m = 3: the force pass of a wider horizon would leave the packed
    // kernel one CTA per SM for every request of the quantum)
    // (and only requests below the size limit: a larger one fills the GPU with its
    // own kernels, which read their stencil table from the constant bank)
    const long long npts = (long long)r->grid.n[0] * r->grid.n[1] * (r->grid.dim == 3 ? r->grid.n[2] : 1);
    const bool packable = s->mode == PD_SERVE_PACKED && r->run.precision == PD_FP32C &&
                          ((r->mat.model == PD_MODEL_PMB && r->mat.s_c == 0.0) ||
                           (r->mat.model == PD_MODEL_LPS && !r->mat.vol_corr && r->grid.m <= 3)) &&
                          (r->run.tile_log2 == 0 || r->run.tile_log2 == 9) &&
                          (s->pack_max_tiles == 0 || (npts + 511) / 512 <= s->pack_max_tiles);
    if (packable) {
        const int W = (stencil_size(r->grid.dim, r->grid.m) + 31) / 32;
        const int split = r->mat.model == PD_MODEL_PMB ? pack_split_for(W) : 0;
        if (r->run.pair_threads == 0 || r->run.pair_threads == split) {
            r->run.tile_log2 = 9;
            r->run.pair_threads = split;
        }
    }
    if (r->run.tile_log2 == 0) {
        // measured at setup (once per class of request); the estimate takes the
        // largest footprint over the tile sizes the measurement may pick
        r->tune = true;
        r->run.tile_log2 = choose_tile_log2(r->grid, s->max_active, s->sms);
        for (int L = 6; L <= 9; ++L) r->est_bytes = std::max(r->est_bytes, estimate_bytes(r->grid, r->mat, L));
    } else {
        r->est_bytes = estimate_bytes(r->grid, r->mat, r->run.tile_log2);
    }
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
        if (s->max_queued > 0 && (long long)s->queue.size() >= s->max_queued) {
            set_error("%d requests wait for admission (max_queued)", s->max_queued);
            return PD_EBUSY;
        }
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
