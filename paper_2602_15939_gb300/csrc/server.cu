// server.cu -- continuous-batching run server of libpic (host C++).
//
// Independent runs (a box configuration, a Maxwellian load, uniform initial
// fields and a step count) are submitted to a queue.  A worker thread admits
// queued runs in arrival order whenever their estimated device footprint fits
// the HBM budget and an active slot is free, gives each admitted run its own
// handle and stream (so the kernels of all active runs overlap on the GPU),
// advances every active run by a chunk of steps per round (at most two
// chunks in flight per run), and retires finished runs: final diagnostics,
// time from submission to result, handle destroyed, memory returned to the
// budget -- which lets the next queued runs in while others keep stepping.
//
// With batching on (pic_server_set_batching), runs of one kind (precision,
// geometry and tile shape, shape order, box type) admitted in the same round
// with at least four rounds of steps left are grouped into cohorts of at
// least `min_batch` runs, each stepped as one pic_batch (one persistent
// particle kernel and batched grid work per step).  A cohort advances by
// chunks no longer than its shortest remaining run; when a member is done,
// the cohort is dissolved after its chunks complete, the finished runs
// retire, and the others step alone.  (PIC_SERVER_COHORT_POLICY=0 instead
// regroups every run of a kind with enough steps left, holding back new
// chunks until all of them are idle.)
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/pic.h"

extern "C" void pic_internal_set_global_error(const char* msg);
extern "C" cudaStream_t pic_internal_batch_stream(pic_batch* b);
extern "C" void pic_internal_batch_graphs(pic_batch* b, int on);

namespace {

using Clock = std::chrono::steady_clock;

struct Cohort;

struct Run {
    uint64_t ticket = 0;
    pic_run_spec spec{};
    uint64_t bytes = 0;
    Clock::time_point t_submit;
    pic_handle* h = nullptr;
    cudaStream_t stream = nullptr;
    int64_t remaining = 0;
    std::deque<cudaEvent_t> inflight;
    bool done = false;
    pic_status status = PIC_OK;
    std::string error;
    pic_diag diag{};
    double latency_s = 0.0;
    bool kept = false;  // the finished box is held for pic_take_result
    Cohort* co = nullptr;  // the cohort stepping this run, if any
    bool hold = false;     // queue no new chunk: the run is draining to join a cohort
    bool alone = false;    // a cohort could not be made with this run: it steps alone
    bool fresh = true;     // admitted and not yet stepped
};

struct Cohort {
    pic_batch* b = nullptr;
    std::vector<Run*> runs;
    std::deque<cudaEvent_t> inflight;
    bool failed = false;
};

}  // namespace

struct pic_server {
    int device = 0;
    uint64_t budget = 0;
    int max_active = 0;
    int steps_per_round = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Run*> queue;
    std::vector<Run*> active;
    std::map<uint64_t, Run*> all;
    uint64_t next_ticket = 1;
    uint64_t bytes_in_use = 0;
    uint64_t peak_bytes = 0;
    int starting = 0;  // admitted runs being set up (neither queued nor active)
    int min_batch = 0;  // 0: no cohorts; else the fewest runs of one kind stepped as a batch
    bool cohort_graphs = false;  // capture cohorts' step cycles in graphs
    int cohort_policy = 1;  // 1: group only runs admitted together; 0: regroup idle runs (draining them)
    int64_t cohorts_formed = 0;
    std::vector<Cohort*> cohorts;  // worker thread only
    int64_t completed = 0;
    int peak_active = 0;
    bool stop = false;
    std::thread worker;
};

// ---- footprint and admission (host arithmetic only) ------------------------------------------

// The tile pic_init will use: the configuration's, or its automatic choice
// (estimated for a 152-SM device).
static void tile_shape(const pic_config& c, int& tx, int& ty, int& tz) {
    const int geom = c.ndim == 3 ? 0 : (c.plane == PIC_PLANE_XY ? 1 : 2);
    const int req = c.tile[0] ? c.tile[0] : (geom == 2 ? c.tile[2] : (c.tile[1] ? c.tile[1] : c.tile[2]));
    const long long sms = 152;
    int side = req;
    if (!side) {
        if (geom == 0) {
            const long long t8 = ((c.nx + 7ll) / 8) * ((c.ny + 7ll) / 8) * ((c.nz + 7ll) / 8);
            side = t8 < 2 * sms ? 4 : 8;
        } else {
            const long long a = c.nx, b = geom == 1 ? c.ny : c.nz;
            auto tiles = [&](long long s) { return ((a + s - 1) / s) * ((b + s - 1) / s); };
            side = tiles(16) < 2 * sms ? 8 : ((c.precision != PIC_FP64 && tiles(32) >= 8 * sms) ? 32 : 16);
        }
    }
    tx = side;
    ty = geom == 2 ? 1 : side;
    tz = geom == 1 ? 1 : side;
}

extern "C" pic_status pic_run_footprint(const pic_run_spec* s, uint64_t* bytes) {
    if (!s || !bytes) {
        pic_internal_set_global_error("pic_run_footprint: NULL argument");
        return PIC_ERR_ARG;
    }
    const pic_config& c = s->cfg;
    if (c.nx < 1 || c.ny < 1 || c.nz < 1 || s->nspecies < 1 || s->nspecies > PIC_MAX_SPECIES || s->ppc < 0) {
        pic_internal_set_global_error("pic_run_footprint: bad grid, species count or ppc");
        return PIC_ERR_ARG;
    }
    const bool fp64 = c.precision == PIC_FP64;
    const uint64_t es = fp64 ? 8 : 4;
    const bool ay = !(c.ndim == 2 && c.plane == PIC_PLANE_XZ), az = !(c.ndim == 2 && c.plane == PIC_PLANE_XY);
    const uint64_t a = 16 / es;
    const uint64_t px = ((uint64_t)c.nx + 5 + a - 1) / a * a, py = ay ? c.ny + 5 : 1, pz = az ? c.nz + 5 : 1;
    const uint64_t cells = (uint64_t)c.nx * c.ny * c.nz, padded = px * py * pz;
    uint64_t fields = 4;  // E, B, J, J scratch
    if (c.box == PIC_BOX_SHEAR || c.box == PIC_BOX_SHEAR_EXPAND) fields += 4;
    uint64_t total = fields * 3 * padded * es + (fp64 ? 0 : 3 * padded * 4) + 3 * cells * 8;
    int tx, ty, tz;
    tile_shape(c, tx, ty, tz);
    const uint64_t ntiles = (uint64_t)((c.nx + tx - 1) / tx) * ((c.ny + ty - 1) / ty) * ((c.nz + tz - 1) / tz);
    const double slack = c.capacity_slack > 0 ? c.capacity_slack : 0.3;
    uint64_t tcap = (uint64_t)std::ceil((double)s->ppc * tx * ty * tz * (1.0 + slack)) + 32;
    tcap = (tcap + 3) & ~3ull;
    const uint64_t nact = c.ndim == 3 ? 3 : 2;
    const bool leaky_disp = c.box == PIC_BOX_LEAKY && c.escape_mode == PIC_ESC_DISPLACEMENT;
    const uint64_t bpp = 4 + nact * es + 3 * es + 4 + (leaky_disp ? 3 * es : 0);
    const uint64_t n = (uint64_t)s->ppc * cells;
    const uint64_t lcap = std::max<uint64_t>(4096, n / 32);
    total += (uint64_t)s->nspecies * 2 * (ntiles * tcap + lcap) * bpp + (uint64_t)s->nspecies * 4 * ntiles * 4;
    *bytes = total + (1u << 20);  // counters, contexts, reduction scratch
    return PIC_OK;
}

extern "C" int pic_admission_count(uint64_t budget, uint64_t in_use, int active, int max_active,
                                   const uint64_t* queued_bytes, int nqueued) {
    // FIFO: admit the longest prefix of the queue that fits the memory budget
    // and the free active slots (a run that can never fit is admitted alone).
    int k = 0;
    uint64_t used = in_use;
    while (k < nqueued && active + k < max_active) {
        const uint64_t b = queued_bytes[k];
        const bool fits = used + b <= budget;
        const bool alone = active + k == 0;  // nothing else running: admit even if over budget
        if (!fits && !alone) break;
        used += b;
        ++k;
    }
    return k;
}

// ---- the worker ------------------------------------------------------------------------------

static pic_status start_run(pic_server* S, Run* r) {
    pic_config cfg = r->spec.cfg;
    cfg.device = S->device;
    pic_status st = pic_init(&cfg, &r->h);
    if (st != PIC_OK) {
        r->error = pic_last_error(nullptr);
        return st;
    }
    if (cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) != cudaSuccess) {
        r->error = "cudaStreamCreate failed";
        return PIC_ERR_CUDA;
    }
    st = pic_set_stream(r->h, r->stream);
    // the worker keeps at most two chunks of a run queued: capacity checks need not wait
    if (st == PIC_OK) st = pic_set_capacity_check(r->h, 8, 0);
    const pic_run_spec& s = r->spec;
    uint32_t id_base = 0;
    const uint64_t per_species = (uint64_t)s.ppc * cfg.nx * cfg.ny * cfg.nz;
    for (int k = 0; st == PIC_OK && k < s.nspecies; ++k) {
        st = pic_load_maxwellian(r->h, k, s.q[k], s.m[k], s.ppc, s.theta, s.drift, s.noise_sigma, s.load_seed + 7919u * k,
                                 id_base);
        id_base += (uint32_t)per_species;
    }
    if (st == PIC_OK) st = pic_set_uniform_fields(r->h, s.E0, s.B0);
    if (st != PIC_OK) r->error = pic_last_error(r->h);
    r->remaining = s.nsteps;
    return st;
}

static void finish_run(pic_server* S, Run* r, pic_status st) {
    if (st == PIC_OK && r->h) {
        st = pic_diagnostics(r->h, &r->diag);
        if (st != PIC_OK) r->error = pic_last_error(r->h);
    }
    for (cudaEvent_t e : r->inflight) cudaEventDestroy(e);
    r->inflight.clear();
    // a kept box leaves the run's stream (synchronised by the diagnostics) for its own
    const bool keep = st == PIC_OK && r->h && r->spec.keep_state && pic_set_stream(r->h, nullptr) == PIC_OK;
    if (r->h && !keep) pic_destroy(r->h);
    if (!keep) r->h = nullptr;
    if (r->stream) cudaStreamDestroy(r->stream);
    r->stream = nullptr;
    r->latency_s = std::chrono::duration<double>(Clock::now() - r->t_submit).count();
    std::lock_guard<std::mutex> lock(S->mu);
    r->status = st;
    r->done = true;
    r->kept = keep;
    if (!keep) S->bytes_in_use -= r->bytes;  // a kept box holds its memory until taken
    S->completed += 1;
    S->cv.notify_all();
}

static void worker_main(pic_server* S) {
    cudaSetDevice(S->device);
    for (;;) {
        std::vector<Run*> admit;
        {
            std::unique_lock<std::mutex> lock(S->mu);
            S->cv.wait(lock, [&] { return S->stop || !S->queue.empty() || !S->active.empty(); });
            if (S->stop && S->active.empty()) break;
            std::vector<uint64_t> qb;
            for (Run* q : S->queue) qb.push_back(q->bytes);
            const int k = pic_admission_count(S->budget, S->bytes_in_use, (int)S->active.size(), S->max_active, qb.data(),
                                              (int)qb.size());
            for (int i = 0; i < k; ++i) {
                Run* r = S->queue.front();
                S->queue.pop_front();
                S->bytes_in_use += r->bytes;
                S->starting += 1;
                admit.push_back(r);
            }
            S->peak_bytes = std::max(S->peak_bytes, S->bytes_in_use);
        }
        for (Run* r : admit) {
            pic_status st = start_run(S, r);
            if (st != PIC_OK) {
                finish_run(S, r, st);
                std::lock_guard<std::mutex> lock(S->mu);
                S->starting -= 1;
                S->cv.notify_all();
                continue;
            }
            std::lock_guard<std::mutex> lock(S->mu);
            S->starting -= 1;
            S->active.push_back(r);
            S->peak_active = std::max(S->peak_active, (int)S->active.size());
        }
        std::vector<Run*> act;
        int min_batch = 0;
        {
            std::lock_guard<std::mutex> lock(S->mu);
            act = S->active;
            min_batch = S->min_batch;
        }
        for (Run* r : act)
            while (!r->inflight.empty() && cudaEventQuery(r->inflight.front()) == cudaSuccess) {
                cudaEventDestroy(r->inflight.front());
                r->inflight.pop_front();
            }
        // cohorts: drop completed chunks; dissolve those with a finished (or
        // failed) member once their chunks are done
        for (size_t c = 0; c < S->cohorts.size();) {
            Cohort* co = S->cohorts[c];
            while (!co->inflight.empty() && cudaEventQuery(co->inflight.front()) == cudaSuccess) {
                cudaEventDestroy(co->inflight.front());
                co->inflight.pop_front();
            }
            bool end = co->failed;
            for (Run* r : co->runs) end |= r->remaining <= 0;
            if (end && co->inflight.empty()) {
                if (pic_batch_destroy(co->b) != PIC_OK)
                    for (Run* r : co->runs) {
                        r->error = pic_last_error(nullptr);
                        r->remaining = -1;
                    }
                for (Run* r : co->runs) r->co = nullptr;
                delete co;
                S->cohorts.erase(S->cohorts.begin() + c);
            } else {
                ++c;
            }
        }
        // new cohorts from runs of one kind with several rounds left (a
        // cohort's set-up must be repaid): once there are min_batch of them,
        // they get no new chunks of their own, and when all are idle they are
        // grouped
        for (Run* r : act) r->hold = false;
        if (min_batch > 0) {
            std::map<std::vector<int>, std::vector<Run*>> kinds;
            const int64_t min_left = 4ll * S->steps_per_round;
            for (Run* r : act) {
                if (r->co || r->alone || r->remaining < min_left) continue;
                if (S->cohort_policy == 1 && !r->fresh) continue;
                const pic_config& c = r->spec.cfg;
                const int t = c.ndim == 3 ? 0 : (c.tile[0] ? c.tile[0] : (c.plane == PIC_PLANE_XY ? c.tile[1] : c.tile[2]));
                kinds[{c.precision, c.ndim, c.plane, t, c.shape_order, c.box, c.escape_mode}]
                    .push_back(r);
            }
            for (auto& kv : kinds) {
                std::vector<Run*>& rs = kv.second;
                if ((int)rs.size() < min_batch) continue;
                bool idle = true;
                for (Run* r : rs) idle = idle && r->inflight.empty();
                if (S->cohort_policy == 1) idle = true;  // fresh runs have nothing in flight
                if (!idle) {
                    for (Run* r : rs) r->hold = true;
                    continue;
                }
                std::vector<pic_handle*> hs;
                for (Run* r : rs) hs.push_back(r->h);
                pic_batch* b = nullptr;
                if (pic_batch_create(hs.data(), (int)hs.size(), &b) != PIC_OK) {
                    for (Run* r : rs) r->alone = true;
                    continue;
                }
                pic_internal_batch_graphs(b, S->cohort_graphs ? 1 : 0);
                for (Run* r : rs) r->fresh = false;
                Cohort* co = new Cohort();
                co->b = b;
                co->runs = rs;
                for (Run* r : rs) r->co = co;
                S->cohorts.push_back(co);
                S->cohorts_formed += 1;
            }
        }
        // one round: keep up to two chunks of steps queued per cohort and per lone run
        for (Cohort* co : S->cohorts) {
            int64_t k = S->steps_per_round;
            for (Run* r : co->runs) k = std::min(k, r->remaining);
            if (co->failed || k <= 0 || co->inflight.size() >= 2) continue;
            if (pic_batch_step(co->b, (int)k) != PIC_OK) {
                const std::string why = pic_last_error(nullptr);
                for (Run* r : co->runs) r->error = why;
                co->failed = true;
                continue;
            }
            for (Run* r : co->runs) r->remaining -= k;
            cudaEvent_t e;
            cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
            cudaEventRecord(e, pic_internal_batch_stream(co->b));
            co->inflight.push_back(e);
        }
        for (Cohort* co : S->cohorts)
            if (co->failed)
                for (Run* r : co->runs)
                    if (r->remaining >= 0) r->remaining = -1;
        for (Run* r : act) {
            if (r->co || r->hold) continue;
            if (r->remaining > 0 && r->inflight.size() < 2) {
                const int k = (int)std::min<int64_t>(r->remaining, S->steps_per_round);
                r->fresh = false;
                pic_status st = pic_step(r->h, k);
                if (st != PIC_OK) {
                    r->error = pic_last_error(r->h);
                    r->remaining = -1;
                    continue;
                }
                r->remaining -= k;
                cudaEvent_t e;
                cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
                cudaEventRecord(e, r->stream);
                r->inflight.push_back(e);
            }
        }
        // retire runs (out of any cohort) whose last chunk has completed
        std::vector<Run*> finished;
        for (Run* r : act) {
            if (r->co) continue;
            if (r->remaining < 0 || (r->remaining == 0 && (r->inflight.empty() || cudaEventQuery(r->inflight.back()) == cudaSuccess)))
                finished.push_back(r);
        }
        if (!finished.empty()) {
            // mark done first, then leave the active set, so a waiter never sees
            // a run that is neither active nor done
            for (Run* r : finished) finish_run(S, r, r->remaining < 0 ? PIC_ERR_STATE : PIC_OK);
            std::lock_guard<std::mutex> lock(S->mu);
            for (Run* r : finished) S->active.erase(std::find(S->active.begin(), S->active.end(), r));
            S->cv.notify_all();
        } else if (!act.empty()) {
            std::this_thread::sleep_for(std::chrono::microseconds(50));
        }
    }
}

// ---- C ABI ---------------------------------------------------------------------------------------

extern "C" pic_status pic_server_create(int device, uint64_t hbm_budget_bytes, int max_active, int steps_per_round,
                                        pic_server** out) {
    if (!out || max_active < 1 || steps_per_round < 1 || hbm_budget_bytes == 0) {
        pic_internal_set_global_error("pic_server_create: bad arguments");
        return PIC_ERR_ARG;
    }
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        pic_internal_set_global_error("pic_server_create: no such CUDA device");
        return PIC_ERR_CUDA;
    }
    // the served runs are FP32: load their kernels now, not at the first run of each kind
    if (pic_preload_kernels(device, PIC_FP32) != PIC_OK) return PIC_ERR_CUDA;
    pic_server* S = new pic_server();
    S->device = device;
    S->budget = hbm_budget_bytes;
    S->max_active = max_active;
    S->steps_per_round = steps_per_round;
    if (const char* e = getenv("PIC_SERVER_COHORT_GRAPHS")) S->cohort_graphs = atoi(e) != 0;
    if (const char* e = getenv("PIC_SERVER_COHORT_POLICY")) S->cohort_policy = atoi(e);
    S->worker = std::thread(worker_main, S);
    *out = S;
    return PIC_OK;
}

extern "C" pic_status pic_server_set_batching(pic_server* S, int min_batch) {
    if (!S || min_batch < 0 || min_batch == 1) {
        pic_internal_set_global_error("pic_server_set_batching: min_batch must be 0 (off) or >= 2");
        return PIC_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(S->mu);
    S->min_batch = min_batch;
    return PIC_OK;
}

extern "C" pic_status pic_submit(pic_server* S, const pic_run_spec* spec, uint64_t* ticket) {
    if (!S || !spec || !ticket || spec->nsteps < 0) {
        pic_internal_set_global_error("pic_submit: bad arguments");
        return PIC_ERR_ARG;
    }
    Run* r = new Run();
    r->spec = *spec;
    pic_status st = pic_run_footprint(spec, &r->bytes);
    if (st != PIC_OK) {
        delete r;
        return st;
    }
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->stop) {
        delete r;
        pic_internal_set_global_error("pic_submit: server is shutting down");
        return PIC_ERR_STATE;
    }
    r->ticket = S->next_ticket++;
    *ticket = r->ticket;
    S->all[r->ticket] = r;
    S->queue.push_back(r);
    S->cv.notify_all();
    return PIC_OK;
}

extern "C" pic_status pic_poll(pic_server* S, uint64_t ticket, int* done, pic_diag* out, double* latency_s) {
    if (!S || !done) {
        pic_internal_set_global_error("pic_poll: bad arguments");
        return PIC_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) {
        pic_internal_set_global_error("pic_poll: unknown ticket");
        return PIC_ERR_ARG;
    }
    Run* r = it->second;
    *done = r->done ? 1 : 0;
    if (!r->done) return PIC_OK;
    if (out) *out = r->diag;
    if (latency_s) *latency_s = r->latency_s;
    if (r->status != PIC_OK) pic_internal_set_global_error(r->error.c_str());
    return r->status;
}

extern "C" pic_status pic_take_result(pic_server* S, uint64_t ticket, pic_handle** out) {
    if (!S || !out) {
        pic_internal_set_global_error("pic_take_result: bad arguments");
        return PIC_ERR_ARG;
    }
    *out = nullptr;
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) {
        pic_internal_set_global_error("pic_take_result: unknown ticket");
        return PIC_ERR_ARG;
    }
    Run* r = it->second;
    if (!r->done || !r->kept || !r->h) {
        pic_internal_set_global_error(
            "pic_take_result: the run has not finished, failed, was not submitted with keep_state, or was taken");
        return PIC_ERR_STATE;
    }
    *out = r->h;
    r->h = nullptr;
    r->kept = false;
    S->bytes_in_use -= r->bytes;
    S->cv.notify_all();
    return PIC_OK;
}

extern "C" pic_status pic_server_wait(pic_server* S, uint64_t ticket, double timeout_s) {
    if (!S) return PIC_ERR_ARG;
    std::unique_lock<std::mutex> lock(S->mu);
    auto pred = [&] {
        if (ticket == 0) return S->queue.empty() && S->active.empty() && S->starting == 0;
        auto it = S->all.find(ticket);
        return it == S->all.end() || it->second->done;
    };
    if (!S->cv.wait_for(lock, std::chrono::duration<double>(timeout_s), pred)) {
        pic_internal_set_global_error("pic_server_wait: timed out");
        return PIC_ERR_TIMEOUT;
    }
    return PIC_OK;
}

extern "C" pic_status pic_server_stats(pic_server* S, pic_server_info* out) {
    if (!S || !out) return PIC_ERR_ARG;
    std::lock_guard<std::mutex> lock(S->mu);
    out->queued = (int32_t)S->queue.size();
    out->active = (int32_t)S->active.size();
    out->completed = S->completed;
    out->bytes_in_use = S->bytes_in_use;
    out->peak_bytes = S->peak_bytes;
    out->peak_active = S->peak_active;
    out->cohorts_formed = (int32_t)std::min<int64_t>(S->cohorts_formed, INT32_MAX);
    return PIC_OK;
}

extern "C" pic_status pic_server_destroy(pic_server* S) {
    if (!S) return PIC_OK;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
        // drop runs never admitted
        for (Run* r : S->queue) {
            r->done = true;
            r->status = PIC_ERR_STATE;
            r->error = "server destroyed before the run was admitted";
        }
        S->queue.clear();
        S->cv.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    for (auto& kv : S->all) {
        if (kv.second->h) pic_destroy(kv.second->h);  // kept boxes never taken
        delete kv.second;
    }
    delete S;
    return PIC_OK;
}
