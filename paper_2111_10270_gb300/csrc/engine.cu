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
    if (dev_bar) cudaFree(dev_bar);
    if (dev_status) cudaFree(dev_status);
    if (host_status) cudaFreeHost(host_status);
    side.destroy();
}

void engine_use_side(Engine& e) {
    if (!e.side.ready && e.side.create(e.device) != cudaSuccess) cudaGetLastError();
    e.cfg.side = e.side.ready ? &e.side : nullptr;
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
    const size_t n_ints = static_cast<size_t>(kNumClasses) * (2 * n + 1) + 7 * static_cast<size_t>(n + 1);
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
    if (n == 1) b.l2 = members[0]->batch.l2;  // the instance's deferred terms stay in L2 during its sweeps
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
    prefix(&b.work_prefix, &b.work_total, [](fdog_instance* m) { return m->dec.wb_start[FDOG_WBUCKETS - 1]; });
    prefix(&b.wide_prefix, &b.wide_total, [](fdog_instance* m) {
        return m->dec.wb_start[FDOG_WBUCKETS] - m->dec.wb_start[FDOG_WBUCKETS - 1];
    });
    for (int i = 0; i < n; ++i) {
        const fdog_instance* m = members[i];
        if (m->params.update != 1) continue;
        if (n > 1) {
            e.err = "an instance with the serial update (update = 1) runs alone";
            return FDOG_EUNSUPPORTED;
        }
        const Decomposition& d = m->dec;
        b.serial.inst = reinterpret_cast<const InstDev*>(dbase);
        b.serial.lev_f_off = d.lev_f_off.data();
        b.serial.lev_b_off = d.lev_b_off.data();
        b.serial.n_lev_f = d.lev_f_off.empty() ? 0 : static_cast<int>(d.lev_f_off.size()) - 1;
        b.serial.n_lev_b = d.lev_b_off.empty() ? 0 : static_cast<int>(d.lev_b_off.size()) - 1;
        b.serial.lev_f = m->dev.lev_f;
        b.serial.lev_b = m->dev.lev_b;
    }
    if (!ids.empty()) {
        // a server keeps one module for every shape it has seen, so that views
        // of changing member sets do not each need a compile
        int rc = jit_kernels(e.jit_universe.empty() ? ids : e.jit_universe, b.jit, e.err);
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
    if (e.persistent && !(e.prof && e.prof->on) && persist_supported(v.b)) {
        // the k iterations as one cooperative launch with grid barriers
        if (!e.dev_bar && cudaMalloc(reinterpret_cast<void**>(&e.dev_bar), 4 * sizeof(unsigned)) != cudaSuccess) {
            cudaGetLastError();
            e.dev_bar = nullptr;
            e.err = "barrier state allocation failed";
            return FDOG_ENOMEM;
        }
        const cudaError_t pe = launch_persistent(v.b, k, e.dev_bar, e.persist_wait_s, e.cfg, e.stream);
        if (pe != cudaSuccess) {
            cudaGetLastError();
            e.err = std::string("persistent iterations: ") + cudaGetErrorString(pe);
            return FDOG_ECUDA;
        }
        return FDOG_OK;
    }
    // graphs need a capturable stream and are skipped while per-launch timing is on
    const bool graphs = e.chunk > 1 && e.stream != nullptr && !(e.prof && e.prof->on);
    int direct = k;
    cudaError_t ce = cudaSuccess;
    if (graphs && k >= e.chunk) {
        if (!v.graph || v.graph_chunk != e.chunk || v.graph_wpb != e.cfg.warps_per_block ||
            v.graph_waves != e.cfg.max_waves || v.graph_side != (e.cfg.side != nullptr)) {
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
            v.graph_waves = e.cfg.max_waves;
            v.graph_side = e.cfg.side != nullptr;
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
        // variables in BDDs from the device (left in the pinned staging buffer
        // until read or released); presolved and row-free ones from the plan
        uint8_t* x;
        if (m->dec.n_bdds > 0) {
            m->solution.clear();
            m->solution_pinned = true;
            x = m->host_x;
        } else {
            m->solution.assign(static_cast<size_t>(m->n_vars), 0);
            m->solution_pinned = false;
            x = m->solution.data();
        }
        for (const int32_t j : m->dec.outside) {
            const int8_t f = m->dec.fixed[j];
            x[j] = f == 2 ? (m->cost[j] < 0 ? 1 : 0) : static_cast<uint8_t>(f);
        }
        m->objective = (m->dec.n_bdds > 0 ? st[i].objective : 0.0) + m->dec.const_obj;
        m->feasible = st[i].n_rejected == 0 ? 1 : 0;
        m->has_solution = true;
        m->rounds = st[i].round;
        m->noconverge = noconv[i] != 0;
    }
    return view_op(e, v, kOpStopRestore, 0);
}

}  // namespace

int engine_admit(Engine& e, std::vector<Member>& ms, size_t first, int max_iters) {
    std::vector<fdog_instance*> fresh, no_bdds, test_now;
    for (size_t i = first; i < ms.size(); ++i) {
        Member& m = ms[i];
        m.phase = max_iters > 0 ? kPhaseDual : kPhaseTest;
        if (m.inst->dec.n_bdds == 0 && m.phase == kPhaseDual) m.phase = kPhaseTest;
        fresh.push_back(m.inst);
        if (m.phase == kPhaseTest) (max_iters > 0 ? no_bdds : test_now).push_back(m.inst);
    }
    if (fresh.empty()) return FDOG_OK;
    BatchView& v = e.v_move;
    int rc = view_build(e, v, fresh);
    if (rc != FDOG_OK) return rc;
    std::vector<InstStatus> st;
    if ((rc = view_status(e, v, st)) != FDOG_OK) return rc;
    for (size_t i = first; i < ms.size(); ++i) ms[i].start_iter = st[i - first].iter;
    if (max_iters > 0 && (rc = view_op(e, v, kOpLimit, max_iters)) != FDOG_OK) return rc;
    // members with nothing to iterate start rounding at once
    if (!no_bdds.empty()) {
        if ((rc = view_build(e, v, no_bdds)) != FDOG_OK) return rc;
        if ((rc = view_op(e, v, kOpRoundBegin, 0)) != FDOG_OK) return rc;
    }
    // rounding only: the pending add-back of Alg. 1 first
    if (!test_now.empty()) {
        if ((rc = view_build(e, v, test_now)) != FDOG_OK) return rc;
        if ((rc = addback_all(e, v)) != FDOG_OK) return rc;
        if ((rc = view_op(e, v, kOpRoundBegin, 0)) != FDOG_OK) return rc;
    }
    return FDOG_OK;
}

int engine_step(Engine& e, std::vector<Member>& ms) {
    const int n = static_cast<int>(ms.size());
    if (n == 0) return FDOG_OK;
    std::vector<fdog_instance*> it_set, all_set;
    for (const Member& m : ms) {
        if (m.phase == kPhaseDone) continue;
        all_set.push_back(m.inst);
        if (m.phase == kPhaseDual || m.phase == kPhaseReopt) it_set.push_back(m.inst);
    }
    int rc;
    if (!it_set.empty()) {
        if ((rc = view_build(e, e.v_iter, it_set)) != FDOG_OK) return rc;
        if ((rc = view_iterate(e, e.v_iter, e.chunk)) != FDOG_OK) return rc;
        for (fdog_instance* m : it_set) { m->pending_T = true; m->iterated = true; }
    }
    std::vector<InstStatus> st;
    std::vector<int> idx;  // member index of each entry of all_set
    for (int i = 0; i < n; ++i)
        if (ms[i].phase != kPhaseDone) idx.push_back(i);
    if (all_set.empty()) return FDOG_OK;
    if ((rc = view_build(e, e.v_all, all_set)) != FDOG_OK) return rc;
    if ((rc = view_status(e, e.v_all, st)) != FDOG_OK) return rc;
    // dual phase finished (stopping rule or iteration budget): add back, start Alg. 2;
    // re-optimisation finished: add back, test again
    std::vector<fdog_instance*> to_begin, to_test;
    for (size_t q = 0; q < idx.size(); ++q) {
        Member& m = ms[idx[q]];
        const bool out_of_iters = st[q].done || st[q].iter >= st[q].iter_limit;
        if (m.phase == kPhaseDual && out_of_iters) {
            m.dual_iters = st[q].iter - m.start_iter;
            to_begin.push_back(m.inst);
            m.phase = kPhaseTest;
        } else if (m.phase == kPhaseReopt && out_of_iters) {
            to_test.push_back(m.inst);
            m.phase = kPhaseTest;
        }
    }
    if (!to_begin.empty()) {
        if ((rc = view_build(e, e.v_move, to_begin)) != FDOG_OK) return rc;
        if ((rc = addback_all(e, e.v_move)) != FDOG_OK) return rc;
        if ((rc = view_op(e, e.v_move, kOpRoundBegin, 0)) != FDOG_OK) return rc;
    }
    if (!to_test.empty()) {
        if ((rc = view_build(e, e.v_move, to_test)) != FDOG_OK) return rc;
        if ((rc = addback_all(e, e.v_move)) != FDOG_OK) return rc;
    }
    std::vector<fdog_instance*> t_set;
    std::vector<int> t_idx;
    for (int i = 0; i < n; ++i)
        if (ms[i].phase == kPhaseTest) { t_set.push_back(ms[i].inst); t_idx.push_back(i); }
    std::vector<fdog_instance*> finished;
    std::vector<int> fin_noconv;
    if (!t_set.empty()) {
        if ((rc = view_build(e, e.v_test, t_set)) != FDOG_OK) return rc;
        std::vector<InstStatus> ts;
        if ((rc = test_all(e, e.v_test, ts)) != FDOG_OK) return rc;
        std::vector<fdog_instance*> p_set;
        for (size_t q = 0; q < t_set.size(); ++q) {
            Member& m = ms[t_idx[q]];
            if (ts[q].n_disagree == 0 || m.inst->dec.n_bdds == 0) {
                m.phase = kPhaseDone;
            } else if (ts[q].round >= m.inst->params.max_rounds) {
                m.phase = kPhaseDone;
                m.noconv = 1;
            } else {
                m.phase = kPhaseReopt;
                p_set.push_back(m.inst);
            }
            if (m.phase == kPhaseDone) {
                finished.push_back(m.inst);
                fin_noconv.push_back(m.noconv);
            }
        }
        if (!p_set.empty()) {
            if ((rc = view_build(e, e.v_move, p_set)) != FDOG_OK) return rc;
            if ((rc = perturb_all(e, e.v_move)) != FDOG_OK) return rc;
        }
    }
    if (!finished.empty()) {
        if ((rc = view_build(e, e.v_move, finished)) != FDOG_OK) return rc;
        if ((rc = finish_all(e, e.v_move, fin_noconv)) != FDOG_OK) return rc;
    }
    return FDOG_OK;
}

int engine_solve(Engine& e, const std::vector<fdog_instance*>& members, int max_iters, std::vector<int>* iters,
                 std::vector<int>* rounds, std::vector<int>* status) {
    std::vector<Member> ms(members.size());
    for (size_t i = 0; i < members.size(); ++i) ms[i].inst = members[i];
    int rc = engine_admit(e, ms, 0, max_iters);
    if (rc != FDOG_OK) return rc;
    while (!std::all_of(ms.begin(), ms.end(), [](const Member& m) { return m.phase == kPhaseDone; }))
        if ((rc = engine_step(e, ms)) != FDOG_OK) return rc;
    const size_t n = ms.size();
    if (iters) iters->resize(n);
    if (rounds) rounds->resize(n);
    if (status) status->resize(n);
    for (size_t i = 0; i < n; ++i) {
        if (iters) (*iters)[i] = ms[i].dual_iters;
        if (rounds) (*rounds)[i] = ms[i].inst->rounds;
        if (status) (*status)[i] = ms[i].noconv ? FDOG_ENOCONVERGE : FDOG_OK;
    }
    return FDOG_OK;
}

int view_autotune(Engine& e, BatchView& v, bool tune_grid) {
    if (v.b.n_inst == 0) return FDOG_OK;
    cudaEvent_t a = nullptr, z = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&z) != cudaSuccess) return fail(e, cudaGetLastError(), "autotune");
    int best = e.cfg.warps_per_block, best_waves = e.cfg.max_waves;
    float best_ms = 1e30f;
    LaunchCfg cfg = e.cfg;
    cfg.prof = nullptr;
    // The candidates are timed on real update passes: each member's
    // multipliers and deferred terms are saved in its min-marginal and
    // perturbation scratch arrays (which nothing reads before they are next
    // written) and its control block in its pinned host copy, the iteration
    // limits are opened for the trials, and all of it is restored afterwards,
    // so the dual state is unchanged.
    cudaError_t ce = cudaSuccess;
    auto save = [&](bool back) {
        for (fdog_instance* m : v.members) {
            if (ce == cudaSuccess) {
                ce = back ? cudaMemcpyAsync(m->dev.ctl, m->host_ctl, sizeof(InstCtl), cudaMemcpyHostToDevice, e.stream)
                          : cudaMemcpyAsync(m->host_ctl, m->dev.ctl, sizeof(InstCtl), cudaMemcpyDeviceToHost, e.stream);
                (back ? m->h2d_bytes : m->d2h_bytes) += static_cast<int64_t>(sizeof(InstCtl));
            }
            if (m->dec.n_bdds == 0 || ce != cudaSuccess) continue;
            const size_t nl = sizeof(float) * static_cast<size_t>(m->dec.slots_pad);
            const size_t nt = sizeof(float) * static_cast<size_t>(m->n_vars);
            ce = back ? cudaMemcpyAsync(m->dev.lam, m->dev.mm0, nl, cudaMemcpyDeviceToDevice, e.stream)
                      : cudaMemcpyAsync(m->dev.mm0, m->dev.lam, nl, cudaMemcpyDeviceToDevice, e.stream);
            if (ce == cudaSuccess)
                ce = back ? cudaMemcpyAsync(m->dev.T, m->dev.pert, nt, cudaMemcpyDeviceToDevice, e.stream)
                          : cudaMemcpyAsync(m->dev.pert, m->dev.T, nt, cudaMemcpyDeviceToDevice, e.stream);
        }
    };
    save(false);
    int rc = ce == cudaSuccess ? view_op(e, v, kOpLimit, 1 << 30) : FDOG_OK;
    // warps per block x grid mode (one persistent wave, or a block per tile group)
    for (int combo = 0; combo < (tune_grid ? 6 : 3) && ce == cudaSuccess && rc == FDOG_OK; ++combo) {
        const int wpb = 2 << (combo % 3), waves = tune_grid ? (combo < 3 ? 1 : 0) : e.cfg.max_waves;
        cfg.warps_per_block = wpb;
        cfg.max_waves = waves;
        ce = launch_sweep(v.b, kFwdUpdate, 0, cfg, e.stream);  // warm-up
        if (ce == cudaSuccess) ce = cudaEventRecord(a, e.stream);
        for (int r = 0; r < 2 && ce == cudaSuccess; ++r) {
            ce = launch_sweep(v.b, kFwdUpdate, 0, cfg, e.stream);
            if (ce == cudaSuccess) ce = launch_sweep(v.b, kBwdUpdate, 0, cfg, e.stream);
        }
        if (ce == cudaSuccess) ce = cudaEventRecord(z, e.stream);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(z);
        float ms = 0.f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, a, z);
        if (ce == cudaSuccess && ms < best_ms) { best_ms = ms; best = wpb; best_waves = waves; }
    }
    save(true);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(e.stream);
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    if (ce != cudaSuccess) return fail(e, ce, "autotune");
    if (rc != FDOG_OK) return rc;
    e.cfg.warps_per_block = best;
    e.cfg.max_waves = best_waves;
    // iterations per graph replay: about 1 ms of device work per replay (an
    // iteration costs about two and a half sweeps; four sweeps were timed), so
    // that the status read after a replay stays a small fraction of it;
    // results do not depend on it
    const double iter_ms = 2.5 * best_ms / 4.0;
    int chunk = 4;
    while (chunk < 32 && chunk * iter_ms < 1.0) chunk *= 2;
    e.chunk = chunk;
    return FDOG_OK;
}

int engine_round(Engine& e, const std::vector<fdog_instance*>& members, std::vector<int>* rounds,
                 std::vector<int>* status) {
    return engine_solve(e, members, 0, nullptr, rounds, status);
}

}  // namespace fdog
