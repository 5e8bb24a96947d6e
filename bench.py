#!/usr/bin/env python3
"""Benchmark of the FastDOG dual hot path on one GB300 (or N replicas).

One step = one complete solve of the workload resident in HBM, through the
C ABI: re-initialise the multipliers (Alg. 1 initialisation), dual
iterations (forward / backward sweeps, deferred averaging, lower bound) until
the 1e-4 relative stopping rule or the iteration cap, the final add-back, the
perturbation rounding loop (Alg. 2) and the objective of the rounded point.

Metric: BDD arc-updates per second = 4 x (BDD nodes) x (dual iterations run,
including the rounding rounds' re-optimisation), over the device-timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fastdog|reference]

N > 1 runs one independent replica per GPU (splitting one instance across
GPUs would need a per-pass exchange of the deferred sums of shared
variables), so scaling is weak and the value is the sum over ranks divided by
the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # large MRF: 512 x 512 4-connected grid, 4 labels, one-hot / marginalisation encoding
    "mrf512": dict(h=512, w=512, labels=4, seed=1, potts_max=2.0, max_iters=500,
                   desc="MRF grid 512x512, 4 labels, Potts U(0,2), unary N(0,1), seed 1"),
    # small case (the parity-test size)
    "mrf8": dict(h=8, w=8, labels=3, seed=0, potts_max=1.0, max_iters=200,
                 desc="MRF grid 8x8, 3 labels, Potts U(0,1), unary N(0,1), seed 0"),
    # QAP-shaped graph matching: 500 x 1000 nodes, 20 candidates, product terms (AND rows) between matches
    # whose left nodes and right nodes are 10-NN neighbours
    "qap500": dict(kind="qap", left=500, right=1000, cand=20, knn=10, seed=2, max_iters=500, sparse=True,
                   desc="QAP-shaped matching 500x1000, 20 candidates, AND products of 10-NN neighbour matches "
                        "(both sides), costs N(0,1), seed 2"),
    # the denser reading: products for every candidate pair of 10-NN left nodes (1.17M variables)
    "qap500_dense": dict(kind="qap", left=500, right=1000, cand=20, knn=10, seed=2, max_iters=500, sparse=False,
                         desc="QAP-shaped matching 500x1000, 20 candidates, AND products of every candidate pair of "
                              "10-NN left nodes, costs N(0,1), seed 2"),
    # one instance of the cell-tracking batch (its first child seed)
    "cell1": dict(kind="cell", seed=3, max_iters=500,
                  desc="cell-tracking instance (first of the seed-3 batch): frames U{10..80}, "
                       "detections/frame U{200..2000}"),
}
METRIC = ("BDD arc-updates/s (full FastDOG solve: dual iterations up to the workload's cap, 500 on the 512x512 grid, "
          "stopping early at the 1e-4 LB-gap rule, + perturbation rounding)")
UNIT = "arc-updates/s"
SWEEP_SRCS = [os.path.join(ROOT, "paper_2111_10270_gb300", "csrc", f)
              for f in ("jit.cpp", "jit_skeleton.cuh", "kernels.cu")]  # generator, skeleton, launch (L2 window)
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "sweep_traffic.txt")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fastdog", choices=["fastdog", "reference"])
    ap.add_argument("--workload", default="mrf512", choices=sorted(WORKLOADS))
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--max-iters", type=int, default=None, help="override the workload's iteration cap")
    ap.add_argument("--dual-only", action="store_true", help="steps without rounding (profiling runs)")
    ap.add_argument("--batch-instances", type=int, default=64,
                    help="cell-tracking batch size for the batched-vs-sequential section (0: skip)")
    ap.add_argument("--serve-instances", type=int, default=200,
                    help="requests of the serving stream replayed in the serving section (0: skip)")
    ap.add_argument("--schemes", type=int, default=1, help="update-scheme comparison section (0: skip)")
    ap.add_argument("--split", type=int, default=1, help="long-row splitting section (0: skip)")
    ap.add_argument("--lb-star", type=int, default=1, help="time to 1e-4 of the stored FP64 LB* (mrf512; 0: skip)")
    ap.add_argument("--per-workload", type=int, default=1,
                    help="dual throughput and roofline of the QAP and cell-tracking workloads (0: skip)")
    ap.add_argument("--threads", type=int, default=min(16, os.cpu_count() or 1),
                    help="host threads / processes for instance generation and planning")
    return ap.parse_args()


def aggregate_ranks(elapsed, work, device):
    """Whole-job figures of N independent replicas: the slowest rank's timed
    span and the work of all ranks (all-reduce MAX / SUM over the default
    process group, on `device`)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([elapsed, work], dtype=torch.float64, device=device)
    tmax = t[:1].clone()
    tsum = t[1:].clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(tsum[0])


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def make_workload(name):
    import ilpgen

    w = WORKLOADS[name]
    if w.get("kind") == "qap":
        return ilpgen.qap(w["seed"], w["left"], w["right"], w["cand"], w["knn"], sparse=w["sparse"]), w
    if w.get("kind") == "cell":
        return ilpgen.cell_tracking(ilpgen._child_seeds(w["seed"], 1)[0]), w
    return ilpgen.mrf_grid(w["h"], w["w"], w["labels"], w["seed"], potts_max=w["potts_max"]), w


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None

    def start(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.gpu_id is not None:
                cmd += ["-i", str(self.gpu_id)]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_smi_id(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else f"GPU-{u}"
    except Exception:
        return os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]


# ----------------------------------------------------------------------------
# the oracle (CPU baseline and reference arm)
# ----------------------------------------------------------------------------
def oracle_rate(g, iters_per_sample, samples):
    """Arc-updates/s of the FP64 oracle: `samples` timed samples of
    `iters_per_sample` dual iterations each on the full instance (the oracle's
    one-off BDD construction is not timed)."""
    import oracle

    oracle.build()
    p = oracle.Problem.from_ilp(g)
    arcs = 4 * p.N
    p.iterate(1)  # first pass also builds the shortest-path labels
    rates = []
    for _ in range(samples):
        t0 = time.perf_counter()
        p.iterate(iters_per_sample)
        dt = time.perf_counter() - t0
        rates.append(arcs * iters_per_sample / dt)
    return rates, p.N


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    g, w = make_workload(args.workload)
    n_steps = args.steps
    rates, nodes = oracle_rate(g, 1, args.warmup + n_steps)
    timed = rates[args.warmup:]
    value = len(timed) / sum(1.0 / r for r in timed)  # equal work per step: harmonic mean = total / total time
    ms = 4 * nodes / value * 1e3
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": n_steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["desc"], "step": "one FP64 oracle dual iteration on the full instance"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{n_steps} single dual iterations of the full {args.workload} instance "
                                   f"(single-threaded C, FP64); BDD construction not timed"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# the CUDA path
# ----------------------------------------------------------------------------
def solve(inst, max_iters, kr, dual_only=False):
    inst.reset()
    iters, lb = inst.iterate(max_iters)
    if dual_only:
        return {"iters": iters, "rounds": 0, "lb": lb, "obj": None, "feasible": None, "rc": 0, "dual_iters": iters}
    rc, rounds = inst.primal_round()
    x, obj, feas = inst.solution()
    return {"iters": iters, "rounds": rounds, "lb": lb, "obj": obj, "feasible": feas, "rc": rc,
            "dual_iters": iters + rounds * kr}


# ----------------------------------------------------------------------------
# batched and served instance streams (host preparation shared by both)
# ----------------------------------------------------------------------------
def generate(fn, args, threads):
    """Seeded instance generation in a spawn process pool (numpy work that
    threads barely overlap)."""
    import multiprocessing
    from concurrent.futures import ProcessPoolExecutor

    if threads <= 1 or len(args) <= 1:
        return [fn(a) for a in args]
    with ProcessPoolExecutor(max_workers=min(threads, len(args)),
                             mp_context=multiprocessing.get_context("spawn")) as ex:
        return list(ex.map(fn, args))


def pct(v, q):
    return float(np.percentile(np.asarray(v, dtype=np.float64), q)) if len(v) else None


def solve_built(inst, max_iters):
    inst.reset()
    n, lb = inst.iterate(max_iters)
    rc, rounds = inst.primal_round()
    x, obj, feas = inst.solution()
    return n, rounds, rc, x, obj, feas, lb


def batched_section(torch, P, dev, stream, params, n_inst, threads):
    """Cell-tracking-shaped batch: the same n_inst instances solved one at a
    time (plain per-instance path) and as one ragged batch, both device
    resident, both to the same stopping rule and rounding; instances/s of each
    and whether every result is identical."""
    import ilpgen

    seeds = ilpgen._child_seeds(3, n_inst)
    ilps = generate(ilpgen.cell_tracking, seeds, threads)
    # built one by one; each build plans its instance on the device (BDDs, layout)
    insts = [P.Instance.from_ilp(g, params).build(dev, stream) for g in ilps]
    plan_stats = [i.plan_stats() for i in insts]
    n_vars = sum(i.info()["n_vars"] for i in insts)
    max_iters = 500

    def sequential():
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = [solve_built(i, max_iters) for i in insts]
        torch.cuda.synchronize()
        return time.perf_counter() - t0, out

    batch = P.Batch(insts, stream)

    def batched():
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in insts:
            i.reset()
        iters, rounds, status = batch.solve(max_iters)
        sols = [i.solution() for i in insts]
        torch.cuda.synchronize()
        return time.perf_counter() - t0, (iters, rounds, status, sols)

    sequential()  # warm-up (graphs, modules)
    batched()
    t_seq, seq = sequential()
    t_bat, (iters, rounds, status, sols) = batched()
    same = all(seq[q][0] == iters[q] and seq[q][1] == rounds[q] and seq[q][2] == status[q]
               and np.array_equal(seq[q][3], sols[q][0]) and seq[q][4] == sols[q][1] for q in range(n_inst))
    feasible = sum(1 for q in range(n_inst) if sols[q][2])
    kr = params.rounding_dual_iters
    arcs = sum(4.0 * insts[q].info()["n_nodes"] * (int(iters[q]) + int(rounds[q]) * kr) for q in range(n_inst))
    batch.close()
    for i in insts:
        i.close()

    # the persistent kernel (one cooperative launch per chunk of iterations) against graph replays of the
    # per-pass kernels, both on the generic kernels, which are the persistent kernel's scope
    generic = [P.Instance.from_ilp(g, P.capi.default_params(tol=params.tol, jit=-1)).build(dev, stream)
               for g in ilps]
    timed = {}
    for mode in ("per_pass", "persistent"):
        b = P.Batch(generic, stream)
        if mode == "persistent":
            b.set_persistent(True)

        def run():
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for i in generic:
                i.reset()
            it, rd, st = b.solve(max_iters)
            out = [(int(it[q]), int(rd[q]), int(st[q])) + tuple(generic[q].solution()[1:]) for q in range(n_inst)]
            xs = [generic[q].solution()[0] for q in range(n_inst)]
            torch.cuda.synchronize()
            return time.perf_counter() - t0, out, xs

        run()  # warm-up
        timed[mode] = run()
        b.close()
    for i in generic:
        i.close()
    pp, pe = timed["per_pass"], timed["persistent"]
    persistent = {
        "kernels": "generic (params.jit = -1) for both",
        "per_pass_instances_per_s": n_inst / pp[0], "persistent_instances_per_s": n_inst / pe[0],
        "persistent_over_per_pass": pp[0] / pe[0],
        "results_identical": bool(pp[1] == pe[1] and all(np.array_equal(a, c) for a, c in zip(pp[2], pe[2]))),
    }
    return {
        "workload": f"cell-tracking batch: {n_inst} instances, frames U{{10..80}}, detections/frame U{{200..2000}}, "
                    f"seed 3 ({n_vars} variables in all)",
        "metric": "instances/s (solve to the 1e-4 LB-gap stopping rule + perturbation rounding, device resident)",
        "batched_instances_per_s": n_inst / t_bat, "sequential_instances_per_s": n_inst / t_seq,
        "speedup": t_seq / t_bat, "batched_s": t_bat, "sequential_s": t_seq,
        "results_identical": bool(same), "feasible": feasible,
        "rounding_noconverge": int(sum(1 for st in status if st == P.FDOG_ENOCONVERGE)),
        "rounds_p50": pct([int(r) for r in rounds], 50), "rounds_max": int(max(rounds)),
        "batched_arc_updates_per_s": arcs / t_bat, "sequential_arc_updates_per_s": arcs / t_seq,
        "dual_iters_p50": pct([r[0] for r in seq], 50), "dual_iters_max": max(r[0] for r in seq),
        "plan_s_p50": pct([t for _, t in plan_stats], 50),
        "planned_on_device": sum(1 for od, _ in plan_stats if od),
        "persistent_kernel": persistent,
    }


def serving_section(torch, P, dev, stream, params, n_req, threads):
    """Replays the first n_req requests of the seeded Poisson stream (200/s;
    MRF and QAP mix) twice: through the continuous-batching server, and one at
    a time in arrival order.  Each request is created from its host arrays at
    its arrival time and submitted unplanned: the server builds its
    decomposition on the device when it admits it; one at a time, each
    request is built (same device builder), solved, read back and freed.
    Latency = result time - arrival time, so planning is inside it."""
    import ilpgen

    specs = ilpgen.serving_stream(4)[:n_req]
    ilps = generate(ilpgen.stream_instance, specs, threads)
    arrivals = np.array([sp["arrival"] for sp in specs]) - specs[0]["arrival"]
    max_iters = 500
    free, _ = torch.cuda.mem_get_info(dev)
    budget = int(free * 0.8)  # every request that fits is admitted

    def run_server():
        srv = P.Server(dev, hbm_budget=budget, max_active=256, max_iters=max_iters)
        l0 = srv.stats()["kernel_launches"]
        t0 = time.perf_counter()
        tickets, delay = [], []
        for q, g in enumerate(ilps):
            d = t0 + arrivals[q] - time.perf_counter()
            if d > 0:
                time.sleep(d)
            tickets.append(srv.submit(P.Instance.from_ilp(g, params)))
            delay.append(time.perf_counter() - (t0 + arrivals[q]))  # creation and submission after arrival
        for t in tickets:
            if not srv.wait(t, 1200.0):
                raise RuntimeError("server request timed out")
        t_end = time.perf_counter()
        polls = [srv.poll(t) for t in tickets]
        lat = [delay[q] + polls[q]["latency_s"] for q in range(len(tickets))]
        res, on_dev = [], 0
        for t in tickets:
            inst = srv.take(t)
            res.append(inst.solution())
            on_dev += inst.plan_stats()[0]
            inst.close()
        launches = srv.stats()["kernel_launches"] - l0
        srv.close()
        return lat, t_end - t0, res, [p["status"] for p in polls], launches, on_dev

    def run_sequential():
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat, res, status = [], [], []
        for q, g in enumerate(ilps):
            d = t0 + arrivals[q] - time.perf_counter()
            if d > 0:
                time.sleep(d)
            inst = P.Instance.from_ilp(g, params).build(dev, stream)
            inst.iterate(max_iters)
            rc, _ = inst.primal_round()
            res.append(inst.solution())
            status.append(rc)
            inst.close()
            lat.append(time.perf_counter() - (t0 + arrivals[q]))
        return lat, time.perf_counter() - t0, res, status

    run_server()  # warm-up: specialised modules of the growing shape set, graphs
    lat_srv, t_srv, res_srv, st_srv, launches, on_dev = run_server()
    lat_seq, t_seq, res_seq, st_seq = run_sequential()
    same = all(np.array_equal(a[0], b[0]) and a[1] == b[1] for a, b in zip(res_srv, res_seq))
    same = same and st_srv == st_seq
    n_vars = sum(g.n_vars for g in ilps)
    kinds = [sp["kind"] for sp in specs]
    return {
        "workload": f"serving stream: first {n_req} of 10,000 seeded requests, Poisson 200/s, 50% MRF "
                    f"(side U{{16..256}}, labels U{{2..8}}), 50% QAP (left U{{50..1000}}, products of 10-NN "
                    f"neighbour matches), seed 4; {kinds.count('mrf')} MRF, {kinds.count('qap')} QAP, "
                    f"{n_vars} variables in all",
        "metric": "instances/s and latency from arrival to result (1e-4 LB-gap stopping rule + rounding)",
        "server_instances_per_s": n_req / t_srv, "sequential_instances_per_s": n_req / t_seq,
        "speedup": t_seq / t_srv,
        "server_latency_p50_s": pct(lat_srv, 50), "server_latency_p99_s": pct(lat_srv, 99),
        "sequential_latency_p50_s": pct(lat_seq, 50), "sequential_latency_p99_s": pct(lat_seq, 99),
        "results_identical": bool(same), "server_kernel_launches": launches,
        "rounding_noconverge": int(sum(1 for v in st_srv if v == P.FDOG_ENOCONVERGE)),
        "failed": int(sum(1 for v in st_srv if v not in (P.FDOG_OK, P.FDOG_ENOCONVERGE))),
        "feasible": int(sum(1 for r in res_srv if r[2])),
        "planned_on_device": int(on_dev),
        "scope": "requests created from host arrays at arrival and submitted unplanned: BDD construction on "
                 "the device, upload, solve and read-back inside the latency",
        "server_admission_budget_bytes": budget,
    }


def update_scheme_section(P, dev, stream):
    """Parallel deferred averaging (Alg. 1, Eq. 5) for several damping factors
    against the serial averaging of Eq. 4, same instance, no early stop:
    iterations each needs to come within 1e-3 / 1e-4 (relative) of the best
    bound any of them reaches, and the device time per iteration."""
    import ilpgen

    cases = [("MRF grid 256x256, 4 labels, Potts U(0,2), seed 5", ilpgen.mrf_grid(256, 256, 4, 5, potts_max=2.0),
              1500, 600),
             ("cell-tracking instance (first of the seed-3 batch)", ilpgen.cell_tracking(ilpgen._child_seeds(3, 1)[0]),
              1500, 300)]
    schemes = [("parallel", 0.3), ("parallel", 0.5), ("parallel", 0.7), ("parallel", 1.0), ("serial", None)]
    import torch

    out = []
    for name, g, it_par, it_ser in cases:
        traces, per_iter = {}, {}
        for kind, omega in schemes:
            kw = dict(tol=0.0, update=1) if kind == "serial" else dict(tol=0.0, omega=omega)
            inst = P.Instance.from_ilp(g, **kw).build(dev, stream)
            iters = it_ser if kind == "serial" else it_par
            tr = np.array([inst.iterate(1)[1] for _ in range(iters)])
            inst.reset()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            inst.iterate(iters)
            torch.cuda.synchronize()
            key = kind if kind == "serial" else f"parallel omega={omega}"
            traces[key] = tr
            per_iter[key] = (time.perf_counter() - t0) / iters * 1e3
            inst.close()
        best = max(float(t.max()) for t in traces.values())

        def first(tr, gap):
            hit = np.nonzero(tr >= best - gap * max(1.0, abs(best)))[0]
            return int(hit[0]) + 1 if len(hit) else None

        out.append({"instance": name, "best_bound": best,
                    "schemes": {k: {"iters_to_1e-3": first(t, 1e-3), "iters_to_1e-4": first(t, 1e-4),
                                    "final_bound": float(t[-1]), "ms_per_iter": per_iter[k],
                                    "bound_non_decreasing": bool(np.all(np.diff(t) >= -1e-6 * max(1.0, abs(best))))}
                                for k, t in traces.items()}})
    return out


def split_section(torch, P, dev, stream):
    """The 500x1000 QAP-shaped matching with its long at-most-one rows as
    given and split into chains of at most 8 or 5 variables
    (fdog_split_rows): dual iterations to the 1e-4 stopping rule and the bound
    there, the bound after 1500 iterations without early stop, the device
    time per iteration, and how many tiles the segmented (long-row) kernels
    still run."""
    import ilpgen

    g = ilpgen.qap(2, 500, 1000, 20, 10)
    cases = {}
    for max_len in (None, 8, 5):
        if max_len is None:
            s, key = g, "as given"
        else:
            nv, rp, col, coef, sense, rhs, _ = P.capi.split_rows(g.n_vars, g.row_ptr, g.col, g.coef, g.sense,
                                                                 g.rhs, max_len)
            s = ilpgen.ILP(nv, np.concatenate([g.cost, np.zeros(nv - g.n_vars)]), rp, col, coef, sense, rhs)
            key = f"split, rows of at most {max_len}"
        inst = P.Instance.from_ilp(s, tol=1e-4).build(dev, stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n_stop, lb_stop = inst.iterate(3000)
        torch.cuda.synchronize()
        t_stop = time.perf_counter() - t0
        seg_tiles = inst.kernel_plan()["static_tiles"]
        inst.close()
        inst = P.Instance.from_ilp(s, tol=0.0).build(dev, stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, lb_fixed = inst.iterate(1500)
        torch.cuda.synchronize()
        ms_iter = (time.perf_counter() - t0) / 1500 * 1e3
        inst.close()
        cases[key] = {"vars": int(s.n_vars), "rows": int(len(s.row_ptr) - 1),
                      "max_row": int(np.diff(s.row_ptr).max()), "iters_to_stop": int(n_stop),
                      "bound_at_stop": float(lb_stop), "seconds_to_stop": t_stop, "bound_after_1500": float(lb_fixed),
                      "ms_per_iter": ms_iter, "generic_kernel_tiles": int(seg_tiles)}
    return {"instance": "QAP-shaped matching 500x1000, 20 candidates, 10-NN AND products, seed 2", "cases": cases}


def iteration_bytes(kp, info):
    """Compulsory bytes of one dual iteration (two update sweeps, two
    deferred-sum passes): every array element counted once per launch (see
    the roofline block of main)."""
    tiles = kp["jit_tiles"] + kp["static_tiles"]
    sweep = 12 * info["n_slots"] + 4 * (kp["local_vars"] + kp["work_vars"]) + 40 * tiles + 8 * kp["local_vars"]
    reduce = 12 * kp["work_vars"] + 8 * kp["work_slots"]
    return sweep, reduce, 2 * (sweep + reduce)


def per_workload_section(torch, P, dev, stream, peak):
    """Dual-iteration throughput of the QAP-shaped matching and one
    cell-tracking instance solved alone: BDD arc-updates/s and device time per
    iteration over a fixed number of iterations (no early stop, iteration
    graphs on), then the same iterations with per-launch CUDA events for the
    dominant update sweep and the deferred-sum step; their compulsory bytes
    over those times, as fractions of the measured HBM bandwidth; and the
    full solve's rounding outcome (Alg. 2)."""
    import ilpgen

    out = {}
    for name in ("qap500", "qap500_dense", "cell1"):
        g, w = make_workload(name)
        iters = 200
        inst = P.Instance.from_ilp(g, tol=0.0).build(dev, stream)
        info, kp = inst.info(), inst.kernel_plan()
        inst.iterate(20)  # warm-up: graphs, modules
        inst.reset()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        inst.iterate(iters)
        ev1.record(stream)
        torch.cuda.synchronize()
        t_iter = ev0.elapsed_time(ev1) / 1e3 / iters
        inst.reset()
        inst.profile_read()
        inst.set_profiling(True)
        inst.iterate(iters)
        inst.set_profiling(False)
        prof = inst.profile_read()
        sweep_b, reduce_b, iter_b = iteration_bytes(kp, info)
        sw = prof["sweep_ms"] / max(prof["sweep_launches"], 1) / 1e3
        rd = prof["reduce_ms"] / max(prof["reduce_launches"], 1) / 1e3
        inst.close()
        # the full solve (stopping rule + rounding) of the same instance
        full = P.Instance.from_ilp(g, P.capi.default_params(tol=1e-4)).build(dev, stream)
        r = solve(full, w["max_iters"], full.params.rounding_dual_iters)
        full.close()
        out[name] = {
            "workload": w["desc"], "vars": info["n_vars"], "bdds": info["n_bdds"], "slots": info["n_slots"],
            "nodes": info["n_nodes"], "arc_updates_per_s": 4.0 * info["n_nodes"] / t_iter,
            "ms_per_iter": t_iter * 1e3, "iteration_bytes": iter_b,
            "iteration_gbs": iter_b / t_iter / 1e9, "iteration_frac": iter_b / t_iter / 1e9 / peak,
            "sweep": {"avg_launch_us": sw * 1e6, "alg_bytes_per_launch": sweep_b,
                      "achieved_gbs": sweep_b / sw / 1e9 if sw else None,
                      "frac": sweep_b / sw / 1e9 / peak if sw else None},
            "deferred_sums": {"avg_launch_us": rd * 1e6, "alg_bytes_per_launch": reduce_b,
                              "achieved_gbs": reduce_b / rd / 1e9 if rd else None,
                              "frac": reduce_b / rd / 1e9 / peak if rd else None},
            "full_solve": {"dual_iters": r["iters"], "rounds": r["rounds"], "status": r["rc"],
                           "feasible": r["feasible"], "lb": r["lb"], "ub": r["obj"]},
        }
    return out


LB_STAR_FILE = os.path.join(ROOT, "tests", "golden", "mrf512_lb_star.txt")


def lb_star_section(torch, P, g, dev, stream):
    """Dual iterations and device time the GPU needs to come within 1e-4
    (relative) of LB*, the FP64 oracle's bound after 2,000 iterations of the
    same schedule on the 512x512 grid (stored by
    tests/golden/make_mrf512_lb_star.py); no early stop."""
    if not os.path.exists(LB_STAR_FILE):
        return None
    rec = {}
    with open(LB_STAR_FILE) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                rec[k.strip()] = v.strip()
    lb_star, iters = float(rec["lb_star"]), int(rec["iterations"])
    inst = P.Instance.from_ilp(g, tol=0.0).build(dev, stream)
    tr = np.array([inst.iterate(1)[1] for _ in range(iters)])
    hit = np.nonzero(tr >= lb_star - 1e-4 * abs(lb_star))[0]
    k = int(hit[0]) + 1 if len(hit) else None
    # the first iteration at which Alg. 1's stopping rule (window 10, tol 1e-4, at least 20 iterations)
    # holds on this trajectory
    rule = [t + 1 for t in range(19, iters) if tr[t] - tr[t - 10] <= 1e-4 * max(abs(tr[t]), 1.0)]
    inst.reset()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    inst.iterate(k or iters)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    inst.close()
    rise = float(rec["lb_after_2000"]) - float(rec["lb_after_1500"]) if "lb_after_1500" in rec else None
    return {"lb_star": lb_star, "lb_star_source": f"FP64 oracle, {iters} iterations of Alg. 1 (omega 0.5), stored",
            "lb_star_converged": False, "lb_star_rise_last_500_iters": rise,
            "stop_rule_iter": rule[0] if rule else "not reached",
            "iters_to_1e-4": k, "seconds_to_1e-4": t if k else None,
            "gpu_bound_after_same_iters": float(tr[-1]),
            "gpu_vs_oracle_rel_diff": abs(float(tr[-1]) - lb_star) / max(1.0, abs(lb_star))}


def sweep_traffic(workload):
    """DRAM bytes per update-sweep launch from the committed ncu summary (of
    the 512x512 MRF), if the sweep's generator sources are unchanged since."""
    if workload != "mrf512":
        return None
    try:
        rec = {}
        with open(TRAFFIC_FILE) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    rec[k.strip()] = v.strip()
        h = hashlib.sha256()
        for f in SWEEP_SRCS:
            h.update(open(f, "rb").read())
        if rec.get("sweep_source_sha256") == h.hexdigest():
            return int(rec["dram_bytes_per_launch"])
    except (OSError, ValueError, KeyError):
        pass
    return None


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = local
    import paper_2111_10270_gb300 as P
    from paper_2111_10270_gb300 import build as libbuild

    libbuild.build()
    g, w = make_workload(args.workload)
    w = dict(w)
    if args.max_iters is not None:
        w["max_iters"] = args.max_iters
    params = P.capi.default_params(tol=1e-4)
    kr = params.rounding_dual_iters
    stream = torch.cuda.current_stream()
    inst = P.Instance.from_ilp(g, params).build(dev, stream)
    info = inst.info()
    nodes = info["n_nodes"]
    dev_bytes = inst.plan()  # device memory of the built instance

    for _ in range(args.warmup):
        solve(inst, w["max_iters"], kr, args.dual_only)

    # ---- device-timed steps -------------------------------------------------
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    sampler = ClockSampler(gpu_smi_id(torch, dev))
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    inst.profile_read()  # clear
    launches0 = inst.profile_read()["kernel_launches"]
    sampler.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    results = [solve(inst, w["max_iters"], kr, args.dual_only) for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches = inst.profile_read()["kernel_launches"] - launches0
    if world > 1:
        torch.distributed.barrier()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    # per-launch kernel timing for the roofline: CUDA events around every sweep and deferred-sum launch on
    # the instance's stream, over as many further solves identical to the timed ones (recording an event
    # per launch turns the iteration graphs off, so the timed solves above run without it)
    inst.set_profiling(True)
    ep0, ep1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ep0.record(stream)
    for _ in range(args.steps):
        solve(inst, w["max_iters"], kr, args.dual_only)
    ep1.record(stream)
    torch.cuda.synchronize()
    inst.set_profiling(False)
    prof = inst.profile_read()
    profiled_ms = ep0.elapsed_time(ep1) / args.steps
    dual_iters = sum(r["dual_iters"] for r in results)
    arcs = 4.0 * nodes * dual_iters
    if world > 1:
        elapsed, arcs = aggregate_ranks(elapsed, arcs, f"cuda:{dev}")
    value = arcs / elapsed

    # ---- roofline of the dominant kernel (update sweep) ----------------------
    kp = inst.kernel_plan()
    S = info["n_slots"]
    n_bdds = info["n_bdds"]
    tiles = kp["jit_tiles"] + kp["static_tiles"]
    n_row_vars = kp["local_vars"] + kp["work_vars"]  # variables inside some BDD
    # compulsory bytes of one sweep launch, every array element counted once: per slot lambda read + write
    # and its variable id (12 B); per variable in a row its deferred term T, read once (4 B; the per-slot
    # gathers of T beyond the first are re-reads the L2 serves); per tile its descriptor and bound partial
    # (40 B); per tile-local variable its target C and new deferred term (8 B)
    alg_bytes = 12 * S + 4 * n_row_vars + 40 * tiles + 8 * kp["local_vars"]
    # per deferred-sum launch: per listed variable its id, C and the new T (12 B); per copy its slot
    # position and the gathered multiplier (8 B)
    reduce_bytes = 12 * kp["work_vars"] + 8 * kp["work_slots"]
    sweep_avg_s = prof["sweep_ms"] / max(prof["sweep_launches"], 1) / 1e3
    reduce_avg_s = prof["reduce_ms"] / max(prof["reduce_launches"], 1) / 1e3
    achieved = alg_bytes / sweep_avg_s / 1e9 if sweep_avg_s > 0 else None
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    if not peak:
        peak = 6800.0
    kernel_name = ("fdog_jit_fwd / fdog_jit_bwd (shape-specialised update sweeps)" if kp["jit_tiles"] * 2 >= tiles
                   else "update sweeps of the dominant kernel class")
    traffic = sweep_traffic(args.workload)
    dram_gbs = traffic / sweep_avg_s / 1e9 if (traffic and sweep_avg_s > 0) else None
    roofline = {"bound": "hbm", "kernel": kernel_name,
                "achieved": achieved, "peak": peak, "peak_source": peak_src, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "traffic": traffic,
                "traffic_source": (f"{os.path.relpath(TRAFFIC_FILE, ROOT)} (ncu capture of this sweep source, "
                                   "not measured in this run)") if traffic else None,
                "dram_achieved": dram_gbs, "dram_frac": dram_gbs / peak if dram_gbs else None,
                "alg_bytes_per_launch": alg_bytes, "avg_launch_us": sweep_avg_s * 1e6,
                "launches": prof["sweep_launches"],
                "timing": (f"CUDA events around each launch over {args.steps} solves identical to the timed ones, "
                           f"right after them ({profiled_ms:.2f} ms per solve with the events, which turn the "
                           "iteration graphs off)"),
                "deferred_sum_kernel": {"avg_launch_us": reduce_avg_s * 1e6, "alg_bytes_per_launch": reduce_bytes,
                                        "achieved_gbs": reduce_bytes / reduce_avg_s / 1e9 if reduce_avg_s else None,
                                        "variables": kp["work_vars"]},
                "tile_local_variables": kp["local_vars"]}

    # ---- end to end through the public API from host buffers ------------------
    e2e = None
    if args.e2e_steps > 0:
        # one untimed end-to-end step first, as the resident measurement has its warm-up steps
        # (first-use costs: pages of host buffers of these sizes, stream and module set-up)
        if args.warmup > 0:
            solve(P.Instance.from_ilp(g, params).build(dev, stream), w["max_iters"], kr, args.dual_only)
            import gc
            gc.collect()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e_arcs, h2d, d2h = 0.0, 0, 0
        plan_dev, plan_s = [], []
        phases = {"create": 0.0, "build": 0.0, "solve": 0.0, "close": 0.0}
        for _ in range(args.e2e_steps):
            # host clock per call: each call below returns with its device work done
            # (build and the solve's read-back synchronise), so the phases add up
            t1 = time.perf_counter()
            e_inst = P.Instance.from_ilp(g, params)
            t2 = time.perf_counter()
            e_inst.build(dev, stream)
            t3 = time.perf_counter()
            od, ps = e_inst.plan_stats()
            plan_dev.append(od)
            plan_s.append(ps)
            r = solve(e_inst, w["max_iters"], kr, args.dual_only)
            t4 = time.perf_counter()
            hb, db = e_inst.transfer_bytes()
            h2d += hb
            d2h += db
            e_arcs += 4.0 * nodes * r["dual_iters"]
            e_inst.close()
            t5 = time.perf_counter()
            for k, a, b in (("create", t1, t2), ("build", t2, t3), ("solve", t3, t4), ("close", t4, t5)):
                phases[k] += (b - a) * 1e3 / args.e2e_steps
        torch.cuda.synchronize()
        e_t = time.perf_counter() - t0
        e2e = {"value": e_arcs / e_t, "unit": UNIT, "h2d_bytes_per_step": h2d // args.e2e_steps,
               "d2h_bytes_per_step": d2h // args.e2e_steps,
               "planned_on_device": all(plan_dev), "plan_s": float(np.median(plan_s)),
               "phases_ms_per_step": phases,
               "scope": "fdog_create from host CSR + upload of the rows + BDD construction and layout on the "
                        "device + solve + solution read-back + fdog_destroy, per step, after "
                        + ("one untimed warm-up step" if args.warmup > 0 else "no warm-up step")}

    # ---- CPU baseline (rank 0, N = 1) ------------------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rates, _ = oracle_rate(g, 1, 6 if args.workload == "mrf512" else 20)
        cpu = {"value": float(np.median(rates)), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"median of {len(rates)} single dual iterations of the full {args.workload} instance "
                         f"(FP64 single-threaded C oracle; its BDD construction not timed)"}

    # ---- batched and served instance mixes (rank 0, N = 1) ---------------------
    batched = served = schemes = split = lb_star = per_workload = None
    if rank == 0 and world == 1 and args.lb_star and args.workload == "mrf512":
        try:
            lb_star = lb_star_section(torch, P, g, dev, stream)
        except Exception as exc:  # a report section: its failure must not cost the bench line
            lb_star = {"error": f"{type(exc).__name__}: {exc}"}
    if rank == 0 and world == 1 and args.per_workload:
        per_workload = per_workload_section(torch, P, dev, stream, peak)
    if rank == 0 and world == 1 and args.schemes:
        schemes = update_scheme_section(P, dev, stream)
    if rank == 0 and world == 1 and args.split:
        split = split_section(torch, P, dev, stream)
    if rank == 0 and world == 1 and args.batch_instances > 0:
        batched = batched_section(torch, P, dev, stream, params, args.batch_instances, args.threads)
    if rank == 0 and world == 1 and args.serve_instances > 0:
        served = serving_section(torch, P, dev, stream, params, args.serve_instances, args.threads)

    if rank == 0:
        last = results[-1]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w["desc"], "vars": info["n_vars"], "bdds": n_bdds, "slots": S, "nodes": nodes,
                       "dual_iters_per_step": dual_iters / args.steps, "stop_iters": last["iters"],
                       "rounds": last["rounds"], "rounding_status": last["rc"], "lb": last["lb"], "ub": last["obj"],
                       "feasible": last["feasible"],
                       "l2": (f"inputs larger than L2 ({dev_bytes / 1e6:.0f} MB resident, L2 129 MB)" if dev_bytes > 129e6
                              else f"inputs fit in L2 ({dev_bytes / 1e6:.0f} MB resident); no flush between steps"),
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
            "per_workload": per_workload, "batched": batched, "serving": served, "update_schemes": schemes,
            "long_rows": split, "time_to_lb_star": lb_star,
        }
        print(json.dumps(line), flush=True)
    inst.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
