// Continuous-batching server (fdog_server_*).
//
// Callers submit instances at any time; submission only queues them, with
// an upper bound of the device memory each needs, from the ILP's sizes.  One
// worker thread owns a private stream and an engine: it admits queued
// instances in arrival order while that memory fits the budget and a slot is
// free, builds each admitted one's decomposition on the device (BDDs, layout,
// slot lists; the host builder only for instances the device builder does not
// take) and corrects its memory to the arena it holds, and then advances
// every resident instance together, one scheduling step at a time (a chunk of
// dual iterations for the iterating ones, rounding tests and perturbations
// for the others).  Instances submitted already planned (fdog_plan, or
// params.planner = 1) keep their host plan.  An instance that finishes -- stopping rule met and rounding
// agreed -- is retired at once: its solution is kept on the host, its device
// memory freed for the next admission.  Each result is the one the instance
// would get alone (engine_step runs the same per-instance schedule).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "engine.h"

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Job {
    uint64_t ticket = 0;
    fdog_instance* inst = nullptr;
    int64_t bytes = 0;         // device memory accounted to the job (a bound until it is built)
    bool plan_on_admit = false;  // the worker plans it at admission
    double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
    int state = 0;  // 0 queued, 1 resident, 2 done (see status), 3 taken
    int status = FDOG_OK;
    int iters = 0, rounds = 0;
    double lb = 0.0;
};

}  // namespace

struct fdog_server {
    int device = 0;
    cudaStream_t stream = nullptr;
    fdog::Engine engine;
    fdog::Profiler prof;
    int64_t budget = 0;
    int64_t used = 0;
    int max_active = 0;
    int max_iters = 0;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::deque<Job*> queue;
    std::unordered_map<uint64_t, Job*> jobs;
    uint64_t next_ticket = 1;
    std::vector<fdog::Member> active;  // worker thread only
    std::vector<Job*> active_jobs;     // worker thread only
    std::vector<int> jit_universe;     // shapes of every submitted instance
    std::string last_error;
    int fatal = FDOG_OK;
    int64_t completed = 0;
    double busy_s = 0.0;
};

using namespace fdog;

namespace fdog {
int plan(fdog_instance* inst, bool compile_jit);
size_t arena_size(const fdog_instance* inst);
int64_t device_plan_bytes_bound(const fdog_instance* inst);
std::vector<int> jit_ids(const fdog_instance* inst);
int release_device(fdog_instance* inst);
int build_instance(fdog_instance* inst, int32_t device, void* cuda_stream, bool autotune);
}  // namespace fdog

namespace {

void fail_job(fdog_server* s, Job* j, int status) {
    j->status = status;
    j->state = 2;
    j->t_done = now_s();
}

void worker_main(fdog_server* s) {
    cudaSetDevice(s->device);
    for (;;) {
        std::vector<Job*> admit;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty() || !s->active.empty(); });
            if (s->stop) break;
            s->engine.jit_universe = s->jit_universe;  // modules cover every shape submitted so far
            // admission in arrival order by free HBM and free slots (the first
            // instance is admitted even if it alone exceeds the budget)
            while (!s->queue.empty() && static_cast<int>(s->active.size() + admit.size()) < s->max_active) {
                Job* j = s->queue.front();
                const bool empty = s->active.empty() && admit.empty();
                if (!empty && s->used + j->bytes > s->budget) break;
                s->queue.pop_front();
                s->used += j->bytes;
                admit.push_back(j);
            }
        }
        const double t0 = now_s();
        const size_t first = s->active.size();
        for (Job* j : admit) {
            // plans an unplanned instance on the server's stream, then uploads it; the server's
            // engine sets the launch shapes
            int rc = build_instance(j->inst, s->device, s->stream, false);
            std::vector<int> grown;
            if (rc == FDOG_OK && j->plan_on_admit) {
                // its shapes join the set the engine's specialised module covers
                std::lock_guard<std::mutex> lk(s->mu);
                for (int id : jit_ids(j->inst))
                    if (std::find(s->jit_universe.begin(), s->jit_universe.end(), id) == s->jit_universe.end()) {
                        s->jit_universe.push_back(id);
                        grown.push_back(id);
                    }
                if (!grown.empty()) grown = s->jit_universe;
            }
            if (!grown.empty()) {
                std::string why;
                rc = jit_compile(grown, why);  // cached per shape set: only new sets compile
                if (rc != FDOG_OK) j->inst->last_error = why;
            }
            std::lock_guard<std::mutex> lk(s->mu);
            if (rc != FDOG_OK) {
                s->used -= j->bytes;
                fail_job(s, j, rc);
                if (j->inst->built) release_device(j->inst);
                s->cv_done.notify_all();
                continue;
            }
            if (j->plan_on_admit) {
                // the bound accounted at admission becomes the arena the instance holds
                const int64_t exact = static_cast<int64_t>(j->inst->arena_bytes);
                s->used += exact - j->bytes;
                j->bytes = exact;
            }
            s->engine.jit_universe = s->jit_universe;
            j->t_admit = now_s();
            j->state = 1;
            Member m;
            m.inst = j->inst;
            s->active.push_back(m);
            s->active_jobs.push_back(j);
        }
        int rc = FDOG_OK;
        if (s->active.size() > first) rc = engine_admit(s->engine, s->active, first, s->max_iters);
        if (rc == FDOG_OK && !s->active.empty()) rc = engine_step(s->engine, s->active);
        s->busy_s += now_s() - t0;
        std::lock_guard<std::mutex> lk(s->mu);
        if (rc != FDOG_OK) {
            // an engine failure ends every resident job with that status
            s->fatal = rc;
            s->last_error = s->engine.err;
            for (size_t i = 0; i < s->active.size(); ++i) {
                s->used -= s->active_jobs[i]->bytes;
                fail_job(s, s->active_jobs[i], rc);
            }
            s->active.clear();
            s->active_jobs.clear();
            s->cv_done.notify_all();
            continue;
        }
        // retire finished instances: solution stays on the host, device memory is freed
        size_t w = 0;
        for (size_t i = 0; i < s->active.size(); ++i) {
            Member& m = s->active[i];
            Job* j = s->active_jobs[i];
            if (m.phase != kPhaseDone) {
                s->active[w] = m;
                s->active_jobs[w] = j;
                ++w;
                continue;
            }
            j->iters = m.dual_iters;
            j->rounds = m.inst->rounds;
            j->status = m.noconv ? FDOG_ENOCONVERGE : FDOG_OK;
            InstCtl c;
            if (read_ctl(m.inst, c) == FDOG_OK) j->lb = c.lb_last;
            release_device(m.inst);
            s->used -= j->bytes;
            j->state = 2;
            j->t_done = now_s();
            ++s->completed;
        }
        s->active.resize(w);
        s->active_jobs.resize(w);
        s->cv_done.notify_all();
    }
}

}  // namespace

extern "C" {

int fdog_server_create(int32_t device, int64_t hbm_budget, int32_t max_active, int32_t max_iters,
                       fdog_server** out) {
    if (!out || hbm_budget <= 0 || max_active <= 0 || max_iters < 0) return FDOG_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return FDOG_EINVAL;
    }
    fdog_server* s = new (std::nothrow) fdog_server();
    if (!s) return FDOG_ENOMEM;
    s->device = device;
    s->budget = hbm_budget;
    s->max_active = max_active;
    s->max_iters = max_iters;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    cudaDeviceProp prop;
    cudaError_t ce = cudaGetDeviceProperties(&prop, device);
    if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (prev >= 0) cudaSetDevice(prev);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return FDOG_ECUDA;
    }
    Engine& e = s->engine;
    e.device = device;
    e.stream = s->stream;
    e.cfg.num_sms = prop.multiProcessorCount;
    // the server's views change with every admission, so they are not autotuned: 4 warps per block and
    // a block per group of tiles, which served the mixed MRF / matching stream 9% faster than one
    // persistent wave (96 against 88 instances/s; 2 and 8 warps per block within 1%); 4 iterations per graph
    // replay, so that members that stop move on to rounding sooner (97 instances/s against 94-97 with 8
    // and 92-94 with 16)
    e.cfg.warps_per_block = 4;
    e.cfg.max_waves = 0;
    e.chunk = 4;
    e.cfg.prof = &s->prof;
    e.prof = nullptr;
    engine_use_side(e);
    s->worker = std::thread(worker_main, s);
    *out = s;
    return FDOG_OK;
}

int fdog_server_submit(fdog_server* s, fdog_instance* inst, uint64_t* ticket) {
    if (!s || !inst || !ticket) return FDOG_EINVAL;
    if (inst->built) return FDOG_ESTATE;
    if (inst->params.update == 1) {
        inst->last_error = "an instance with the serial update (update = 1) runs alone";
        return FDOG_EUNSUPPORTED;
    }
    if (inst->shard) {
        inst->last_error = "a shard of a split instance runs through fdog_shard_pass";
        return FDOG_EUNSUPPORTED;
    }
    Job* j = new (std::nothrow) Job();
    if (!j) return FDOG_ENOMEM;
    j->inst = inst;
    if (!inst->planned && inst->params.planner != 1) {
        // planned by the worker at admission, on the device where the builder takes it
        j->plan_on_admit = true;
        j->bytes = device_plan_bytes_bound(inst);
        j->t_submit = now_s();
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->fatal != FDOG_OK) {
            delete j;
            return s->fatal;
        }
        j->ticket = s->next_ticket++;
        s->jobs.emplace(j->ticket, j);
        s->queue.push_back(j);
        *ticket = j->ticket;
        s->cv_work.notify_one();
        return FDOG_OK;
    }
    // host planning in the caller's thread, and the specialised kernels
    int rc = plan(inst, false);
    if (rc != FDOG_OK) {
        delete j;
        return rc;
    }
    std::vector<int> ids = jit_ids(inst), added;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->fatal != FDOG_OK) {
            delete j;
            return s->fatal;
        }
        for (int id : ids)
            if (std::find(s->jit_universe.begin(), s->jit_universe.end(), id) == s->jit_universe.end()) {
                s->jit_universe.push_back(id);
                added.push_back(id);
            }
        ids = s->jit_universe;
    }
    if (!added.empty()) {
        // one module covers every shape submitted so far (cached per shape set,
        // so a server that has seen these shapes before only loads it)
        std::string why;
        rc = jit_compile(ids, why);
        if (rc != FDOG_OK) {
            std::lock_guard<std::mutex> lk(s->mu);
            for (int id : added)
                s->jit_universe.erase(std::find(s->jit_universe.begin(), s->jit_universe.end(), id));
            inst->last_error = why;
            delete j;
            return rc;
        }
    }
    j->bytes = static_cast<int64_t>(arena_size(inst));
    j->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        j->ticket = s->next_ticket++;
        s->jobs.emplace(j->ticket, j);
        s->queue.push_back(j);
    }
    s->cv_work.notify_one();
    *ticket = j->ticket;
    return FDOG_OK;
}

int fdog_server_poll(fdog_server* s, uint64_t ticket, int32_t* state, int32_t* status, double* lb,
                     double* latency_s) {
    if (!s) return FDOG_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return FDOG_EINVAL;
    const Job* j = it->second;
    if (state) *state = j->state;
    if (status) *status = j->status;
    if (lb) *lb = j->lb;
    if (latency_s) *latency_s = j->state >= 2 ? j->t_done - j->t_submit : now_s() - j->t_submit;
    return FDOG_OK;
}

int fdog_server_wait(fdog_server* s, uint64_t ticket, double timeout_s) {
    if (!s) return FDOG_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return FDOG_EINVAL;
    Job* j = it->second;
    const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return j->state >= 2; });
    return ok ? FDOG_OK : FDOG_ETIMEOUT;
}

int fdog_server_take(fdog_server* s, uint64_t ticket, fdog_instance** out) {
    if (!s || !out) return FDOG_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return FDOG_EINVAL;
    Job* j = it->second;
    if (j->state != 2) return FDOG_ESTATE;
    *out = j->inst;
    s->jobs.erase(it);
    delete j;
    return FDOG_OK;
}

int fdog_server_stats(fdog_server* s, int64_t* queued, int64_t* resident, int64_t* completed, int64_t* hbm_used,
                      double* busy_s, int64_t* kernel_launches) {
    if (!s) return FDOG_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (queued) *queued = static_cast<int64_t>(s->queue.size());
    if (resident) *resident = static_cast<int64_t>(s->active.size());
    if (completed) *completed = s->completed;
    if (hbm_used) *hbm_used = s->used;
    if (busy_s) *busy_s = s->busy_s;
    if (kernel_launches) *kernel_launches = s->prof.launches;
    return FDOG_OK;
}

const char* fdog_server_last_error(const fdog_server* s) { return s ? s->last_error.c_str() : ""; }

void fdog_server_destroy(fdog_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    for (auto& kv : s->jobs) {
        fdog_destroy(kv.second->inst);
        delete kv.second;
    }
    s->jobs.clear();
    const int dev = s->device;
    cudaStream_t st = s->stream;
    delete s;  // the engine's buffers are freed while the device is current
    if (st) cudaStreamDestroy(st);
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    cudaGetLastError();
}

}  // extern "C"
