// Execution engine over sets of instances (see engine.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "engine.h"

namespace fdog {

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

constexpr int kPhaseDual = 0;
constexpr int kPhaseTest = 1;
constexpr int kPhaseReopt = 2;
constexpr int kPhaseDone = 3;

}  // namespace

void BatchView::drop_graph() {
    if (graph) cudaGraphExecDestroy(graph);
    graph = nullptr;
    graph_chunk = 0;
}

BatchView::~BatchView() {
    drop_graph();
    if (dev) cudaFree(dev);
}

Engine::~Engine() {
    if (dev_status) cudaFree(dev_status);
    if (host_status) cudaFreeHost(host_status);
}

int view_build(Engine& e, BatchView& v, const std::vector<fdog_instance*>& members) {
    std::vector<uint64_t> uids(members.size());
    for (size_t i = 0; i < members.size(); ++i) uids[i] = members[i]->uid;
    if (v.dev && uids == v.uids) return FDOG_OK;
    v.drop_graph();
    v.members = members;
    v.uids.clear();  // set once the image is uploaded
    const int n = static_cast<int>(members.size());
    DevBatch b;
    b.n_inst = n;
    if (n == 0) {
        v.b = b;
        v.uids = std::move(uids);
        return FDOG_OK;
    }
    // host image: InstDev[n], then the int32 prefix arrays
    const size_t desc_bytes = align_up(sizeof(InstDev) * n, 256);
    const size_t n_ints = static_cast<size_t>(kNumClasses) * (2 * n + 1) + 6 * static_cast<size_t>(n + 1);
    const size_t bytes = desc_bytes + sizeof(int32_t) * n_ints;
    if (v.cap < bytes) {
        if (v.dev) cudaFree(v.dev);
        v.dev = nullptr;
        v.cap = 0;
        cudaError_t ce = cudaMalloc(&v.dev, bytes);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            v.dev = nullptr;
            e.err = "batch descriptor allocation failed";
            return FDOG_ENOMEM;
        }
        v.cap = bytes;
    }
    std::vector<char> img(bytes, 0);
    InstDev* hd = reinterpret_cast<InstDev*>(img.data());
    int32_t* ints = reinterpret_cast<int32_t*>(img.data() + desc_bytes);
    char* dbase = static_cast<char*>(v.dev);
    int32_t* dints = reinterpret_cast<int32_t*>(dbase + desc_bytes);
    size_t q = 0;
    std::vector<int> ids;
    for (int i = 0; i < n; ++i) {
        hd[i] = members[i]->hdesc;
        for (const ShapeDev& s : members[i]->dec.shape_dev)
            if (s.jit >= 0) ids.push_back(s.jit);
    }
    b.insts = reinterpret_cast<InstDev*>(dbase);
    for (int c = 0; c < kNumClasses; ++c) {
        int32_t* pre = ints + q;
        int32_t* first = ints + q + n + 1;
        pre[0] = 0;
        for (int i = 0; i < n; ++i) {
            const Decomposition& d = members[i]->dec;
            const int32_t cnt = d.cls_tile_begin[c + 1] - d.cls_tile_begin[c];
            pre[i + 1] = pre[i] + cnt;
            first[i] = d.cls_tile_begin[c];
            b.kmax[c] = std::max(b.kmax[c], d.kmax[c]);
            b.has_local[c] = b.has_local[c] || d.cls_has_local[c];
        }
        b.tile_prefix[c] = dints + q;
        b.tile_first[c] = dints + q + n + 1;
        b.tiles_total[c] = pre[n];
        q += 2 * n + 1;
    }
    auto prefix = [&](int32_t** dst, int32_t* total, auto count) {
        int32_t* pre = ints + q;
        pre[0] = 0;
        for (int i = 0; i < n; ++i) pre[i + 1] = pre[i] + count(members[i]);
        *dst = dints + q;
        *total = pre[n];
        q += n + 1;
    };
    prefix(&b.var_prefix, &b.vars_total, [](fdog_instance* m) { return m->n_vars; });
    prefix(&b.slot_prefix, &b.slots_total, [](fdog_instance* m) { return static_cast<int32_t>(m->dec.slots_pad); });
    prefix(&b.chunk_prefix, &b.chunks_total,
           [](fdog_instance* m) { return m->dec.tiles.empty() ? 0 : m->hdesc.n_chunks; });
    prefix(&b.objchunk_prefix, &b.objchunks_total,
           [](fdog_instance* m) { return m->n_vars > 0 ? m->hdesc.n_obj_chunks : 0; });
    prefix(&b.tile_all_prefix, &b.tiles_all_total,
           [](fdog_instance* m) { return static_cast<int32_t>(m->dec.tiles.size()); });
    prefix(&b.work_prefix, &b.work_total, [](fdog_instance* m) { return static_cast<int32_t>(m->dec.work.size()); });
    if (!ids.empty()) {
        int rc = jit_kernels(ids, b.jit, e.err);
        if (rc != FDOG_OK) return rc;
    }
    cudaError_t ce = cudaMemcpyAsync(v.dev, img.data(), bytes, cudaMemcpyHostToDevice, e.stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(e.stream);  // img is a host temporary
    if (ce != cudaSuccess) {
        e.err = std::string("batch descriptor upload: ") + cudaGetErrorString(ce);
        return FDOG_ECUDA;
    }
    v.b = b;
    v.uids = std::move(uids);
    return FDOG_OK;
}

int view_status(Engine& e, BatchView& v, std::vector<InstStatus>& out) {
    const int n = v.b.n_inst;
    out.resize(n);
    if (n == 0) return FDOG_OK;
    if (e.status_cap < n) {
        if (e.dev_status) cudaFree(e.dev_status);
        if (e.host_status) cudaFreeHost(e.host_status);
        e.dev_status = nullptr;
        e.host_status = nullptr;
        e.status_cap = 0;
        if (cudaMalloc(reinterpret_cast<void**>(&e.dev_status), sizeof(InstStatus) * n) != cudaSuccess ||
            cudaMallocHost(reinterpret_cast<void**>(&e.host_status), sizeof(InstStatus) * n) != cudaSuccess) {
            cudaGetLastError();
            e.err = "status buffer allocation failed";
            return FDOG_ENOMEM;
        }
        e.status_cap = n;
    }
    cudaError_t ce = launch_status(v.b, e.dev_status, e.cfg, e.stream);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(e.host_status, e.dev_status, sizeof(InstStatus) * n, cudaMemcpyDeviceToHost, e.stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(e.stream);
    if (ce != cudaSuccess) {
        e.err = std::string("status: ") + cudaGetErrorString(ce);
        return FDOG_ECUDA;
    }
    std::memcpy(out.data(), e.host_status, sizeof(InstStatus) * n);
    for (int i = 0; i < n; ++i) {
        v.members[i]->d2h_bytes += sizeof(InstStatus);
        if (out[i].error != 0) {
            e.err = "device-side error " + std::to_string(out[i].error);
            return FDOG_ETIMEOUT;
        }
    }
    return FDOG_OK;
}

int view_op(Engine& e, BatchView& v, int op, int arg) {
    cudaError_t ce = launch_instance_op(v.b, op, arg, e.cfg, e.stream);
    if (ce != cudaSuccess) {
        e.err = std::string("instance op: ") + cudaGetErrorString(ce);
        return FDOG_ECUDA;
    }
    return FDOG_OK;
}

int view_iterate(Engine& e, BatchView& v, int k) {
    if (k <= 0 || v.b.n_inst == 0) return FDOG_OK;
    // graphs need a capturable stream and are skipped while per-launch timing is on
    const bool graphs = e.chunk > 1 && e.stream != nullptr && !(e.prof && e.prof->on);
    int direct = k;
    cudaError_t ce = cudaSuccess;
    if (graphs && k >= e.chunk) {
        if (!v.graph || v.graph_chunk != e.chunk || v.graph_wpb != e.cfg.warps_per_block) {
            v.drop_graph();
            LaunchCfg cap = e.cfg;
            Profiler counter;  // counts the captured launches once
            cap.prof = &counter;
            cudaGraph_t g = nullptr;
            ce = cudaStreamBeginCapture(e.stream, cudaStreamCaptureModeThreadLocal);
            for (int t = 0; t < e.chunk && ce == cudaSuccess; ++t) ce = launch_iteration(v.b, cap, e.stream);
            cudaError_t ce2 = cudaStreamEndCapture(e.stream, &g);
            if (ce == cudaSuccess) ce = ce2;
            if (ce == cudaSuccess) ce = cudaGraphInstantiate(&v.graph, g, 0);
            if (g) cudaGraphDestroy(g);
            if (ce != cudaSuccess) {
                cudaGetLastError();
                v.graph = nullptr;
                e.err = std::string("graph capture: ") + cudaGetErrorString(ce);
                return FDOG_ECUDA;
            }
            v.graph_chunk = e.chunk;
            v.graph_wpb = e.cfg.warps_per_block;
            v.graph_launches_per_replay = counter.launches;
        }
        const int reps = k / e.chunk;
        for (int r = 0; r < reps && ce == cudaSuccess; ++r) {
            ce = cudaGraphLaunch(v.graph, e.stream);
            if (e.cfg.prof) e.cfg.prof->launches += v.graph_launches_per_replay;
        }
        direct = k - reps * e.chunk;
    }
    for (int t = 0; t < direct && ce == cudaSuccess; ++t) ce = launch_iteration(v.b, e.cfg, e.stream);
    if (ce != cudaSuccess) {
        e.err = std::string("iteration: ") + cudaGetErrorString(ce);
        return FDOG_ECUDA;
    }
    return FDOG_OK;
}

namespace {

int fail(Engine& e, cudaError_t ce, const char* where) {
    cudaGetLastError();
    e.err = std::string(where) + ": " + cudaGetErrorString(ce);
    return FDOG_ECUDA;
}

// add-back of Alg. 1 (lambda += T, T = 0) for every member
int addback_all(Engine& e, BatchView& v) {
    cudaError_t ce = launch_addback(v.b, e.cfg, e.stream);
    if (ce != cudaSuccess) return fail(e, ce, "add-back");
    for (fdog_instance* m : v.members) {
        m->pending_T = false;
        m->iterated = false;
    }
    return FDOG_OK;
}

// the agreement test of Alg. 2 (min-marginals, signs, perturbation of this round)
int test_all(Engine& e, BatchView& v, std::vector<InstStatus>& st) {
    cudaError_t ce = launch_sweep(v.b, kMinMarg, 0, e.cfg, e.stream);
    if (ce != cudaSuccess) return fail(e, ce, "rounding min-marginals");
    int rc = view_op(e, v, kOpClearDisagree, 0);
    if (rc != FDOG_OK) return rc;
    ce = launch_round_test(v.b, e.cfg, e.stream);
    if (ce != cudaSuccess) return fail(e, ce, "rounding test");
    return view_status(e, v, st);
}

// perturb, next round, K_r iterations of Alg. 1 limits
int perturb_all(Engine& e, BatchView& v) {
    cudaError_t ce = launch_round_apply(v.b, e.cfg, e.stream);
    if (ce != cudaSuccess) return fail(e, ce, "perturbation");
    int rc = view_op(e, v, kOpRoundNext, 0);
    if (rc == FDOG_OK) rc = view_op(e, v, kOpLimitReopt, 0);
    return rc;
}

// objective, exact acceptance of every row, solutions to the host
int finish_all(Engine& e, BatchView& v, const std::vector<int>& noconv) {
    cudaError_t ce = launch_objective(v.b, e.cfg, e.stream);
    if (ce != cudaSuccess) return fail(e, ce, "objective");
    int rc = view_op(e, v, kOpClearRejected, 0);
    if (rc != FDOG_OK) return rc;
    ce = launch_accept(v.b, e.cfg, e.stream);
    if (ce != cudaSuccess) return fail(e, ce, "acceptance");
    for (fdog_instance* m : v.members) {
        if (m->n_vars == 0 || m->dec.n_bdds == 0) continue;
        ce = copy_async(m, m->host_x, m->dev.x, m->n_vars, cudaMemcpyDeviceToHost);
        if (ce != cudaSuccess) return fail(e, ce, "solution copy");
    }
    std::vector<InstStatus> st;
    rc = view_status(e, v, st);
    if (rc != FDOG_OK) return rc;
    for (size_t i = 0; i < v.members.size(); ++i) {
        fdog_instance* m = v.members[i];
        std::vector<uint8_t> x(m->n_vars, 0);
        if (m->dec.n_bdds > 0) std::memcpy(x.data(), m->host_x, m->n_vars);
        for (int32_t j = 0; j < m->n_vars; ++j) {
            const int8_t f = m->dec.fixed[j];
            if (f == 0 || f == 1) x[j] = static_cast<uint8_t>(f);
            else if (f == 2) x[j] = m->cost[j] < 0 ? 1 : 0;
        }
        m->solution = std::move(x);
        m->objective = (m->dec.n_bdds > 0 ? st[i].objective : 0.0) + m->dec.const_obj;
        m->feasible = st[i].n_rejected == 0 ? 1 : 0;
        m->has_solution = true;
        m->rounds = st[i].round;
        m->noconverge = noconv[i] != 0;
    }
    return view_op(e, v, kOpStopRestore, 0);
}

}  // namespace

int engine_solve(Engine& e, const std::vector<fdog_instance*>& members, int max_iters, std::vector<int>* iters,
                 std::vector<int>* rounds, std::vector<int>* status) {
    const int n = static_cast<int>(members.size());
    std::vector<int> phase(n, max_iters > 0 ? kPhaseDual : kPhaseTest), noconv(n, 0), start_iter(n, 0),
        dual_iters(n, 0);
    std::vector<fdog_instance*> no_bdds;  // nothing to iterate: straight to rounding
    for (int i = 0; i < n; ++i)
        if (members[i]->dec.n_bdds == 0 && phase[i] == kPhaseDual) {
            phase[i] = kPhaseTest;
            no_bdds.push_back(members[i]);
        }
    BatchView& all = e.v_all;
    BatchView& iterating = e.v_iter;
    BatchView& moving = e.v_move;
    BatchView& testing = e.v_test;
    int rc = view_build(e, all, members);
    if (rc != FDOG_OK) return rc;
    std::vector<InstStatus> st;
    if ((rc = view_status(e, all, st)) != FDOG_OK) return rc;
    for (int i = 0; i < n; ++i) start_iter[i] = st[i].iter;
    if (max_iters > 0) {
        if ((rc = view_op(e, all, kOpLimit, max_iters)) != FDOG_OK) return rc;
        if (!no_bdds.empty()) {
            if ((rc = view_build(e, moving, no_bdds)) != FDOG_OK) return rc;
            if ((rc = view_op(e, moving, kOpRoundBegin, 0)) != FDOG_OK) return rc;
        }
    } else {
        if ((rc = addback_all(e, all)) != FDOG_OK) return rc;
        if ((rc = view_op(e, all, kOpRoundBegin, 0)) != FDOG_OK) return rc;
    }
    for (;;) {
        std::vector<fdog_instance*> it_set;
        for (int i = 0; i < n; ++i)
            if (phase[i] == kPhaseDual || phase[i] == kPhaseReopt) it_set.push_back(members[i]);
        if (!it_set.empty()) {
            if ((rc = view_build(e, iterating, it_set)) != FDOG_OK) return rc;
            if ((rc = view_iterate(e, iterating, e.chunk)) != FDOG_OK) return rc;
            for (fdog_instance* m : it_set) { m->pending_T = true; m->iterated = true; }
        }
        if ((rc = view_status(e, all, st)) != FDOG_OK) return rc;
        // dual phase finished (stopping rule or iteration budget): add back, start Alg. 2;
        // re-optimisation finished: add back, test again
        std::vector<fdog_instance*> to_begin, to_test;
        for (int i = 0; i < n; ++i) {
            const bool out_of_iters = st[i].done || st[i].iter >= st[i].iter_limit;
            if (phase[i] == kPhaseDual && out_of_iters) {
                dual_iters[i] = st[i].iter - start_iter[i];
                to_begin.push_back(members[i]);
                phase[i] = kPhaseTest;
            } else if (phase[i] == kPhaseReopt && out_of_iters) {
                to_test.push_back(members[i]);
                phase[i] = kPhaseTest;
            }
        }
        if (!to_begin.empty()) {
            if ((rc = view_build(e, moving, to_begin)) != FDOG_OK) return rc;
            if ((rc = addback_all(e, moving)) != FDOG_OK) return rc;
            if ((rc = view_op(e, moving, kOpRoundBegin, 0)) != FDOG_OK) return rc;
        }
        if (!to_test.empty()) {
            if ((rc = view_build(e, moving, to_test)) != FDOG_OK) return rc;
            if ((rc = addback_all(e, moving)) != FDOG_OK) return rc;
        }
        std::vector<fdog_instance*> t_set;
        std::vector<int> t_idx;
        for (int i = 0; i < n; ++i)
            if (phase[i] == kPhaseTest) { t_set.push_back(members[i]); t_idx.push_back(i); }
        if (!t_set.empty()) {
            if ((rc = view_build(e, testing, t_set)) != FDOG_OK) return rc;
            std::vector<InstStatus> ts;
            if ((rc = test_all(e, testing, ts)) != FDOG_OK) return rc;
            std::vector<fdog_instance*> p_set;
            for (size_t q = 0; q < t_set.size(); ++q) {
                const int i = t_idx[q];
                if (ts[q].n_disagree == 0 || t_set[q]->dec.n_bdds == 0) {
                    phase[i] = kPhaseDone;
                } else if (ts[q].round >= t_set[q]->params.max_rounds) {
                    phase[i] = kPhaseDone;
                    noconv[i] = 1;
                } else {
                    phase[i] = kPhaseReopt;
                    p_set.push_back(t_set[q]);
                }
            }
            if (!p_set.empty()) {
                if ((rc = view_build(e, moving, p_set)) != FDOG_OK) return rc;
                if ((rc = perturb_all(e, moving)) != FDOG_OK) return rc;
            }
        }
        if (std::all_of(phase.begin(), phase.end(), [](int p) { return p == kPhaseDone; })) break;
    }
    if ((rc = finish_all(e, all, noconv)) != FDOG_OK) return rc;
    if (iters) *iters = dual_iters;
    if (rounds || status) {
        if (rounds) rounds->resize(n);
        if (status) status->resize(n);
        for (int i = 0; i < n; ++i) {
            if (rounds) (*rounds)[i] = members[i]->rounds;
            if (status) (*status)[i] = noconv[i] ? FDOG_ENOCONVERGE : FDOG_OK;
        }
    }
    return FDOG_OK;
}

int view_autotune(Engine& e, BatchView& v) {
    if (v.b.n_inst == 0) return FDOG_OK;
    cudaEvent_t a = nullptr, z = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&z) != cudaSuccess) return fail(e, cudaGetLastError(), "autotune");
    const int saved = e.cfg.warps_per_block;
    int best = saved;
    float best_ms = 1e30f;
    LaunchCfg cfg = e.cfg;
    cfg.prof = nullptr;
    for (int wpb : {2, 4, 8}) {
        cfg.warps_per_block = wpb;
        cudaError_t ce = launch_sweep(v.b, kMinMarg, 0, cfg, e.stream);  // warm-up
        if (ce == cudaSuccess) ce = cudaEventRecord(a, e.stream);
        for (int r = 0; r < 3 && ce == cudaSuccess; ++r) ce = launch_sweep(v.b, kMinMarg, 0, cfg, e.stream);
        if (ce == cudaSuccess) ce = cudaEventRecord(z, e.stream);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(z);
        float ms = 0.f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, a, z);
        if (ce != cudaSuccess) {
            cudaEventDestroy(a);
            cudaEventDestroy(z);
            return fail(e, ce, "autotune");
        }
        if (ms < best_ms) { best_ms = ms; best = wpb; }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    e.cfg.warps_per_block = best;
    return FDOG_OK;
}

int engine_round(Engine& e, const std::vector<fdog_instance*>& members, std::vector<int>* rounds,
                 std::vector<int>* status) {
    return engine_solve(e, members, 0, nullptr, rounds, status);
}

}  // namespace fdog
