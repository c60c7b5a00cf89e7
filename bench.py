#!/usr/bin/env python
"""Benchmark: stress node-steps/s of the coupled EM/TM/IR aging run on the full chip.

Workload: the 2048 x 2048-stripe two-layer mesh at 5 um (4,096 stripes x
20,471 stress nodes = 83.8 M, 4.19 M IR nodes, 5 % lognormal sinks, 8
hotspots) with a batch of Monte Carlo samples (20 % CoV kappa / sigma_crit
per segment) held at once; per-node coefficients are rebuilt in windows of
samples.  One step = one aging step of every sample: 256 backward-Euler
steps of every stripe, nucleation, void growth, resistance write-back, IR
re-solve, drop.  The line also carries the plain-vs-chosen comparison
(whole-horizon TTF runs of one sample, FP64 plain against the FP32 path),
the roofline of the dominant kernel, the CPU oracle on a bounded sample and
an end-to-end number through the public API.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--samples S] [--window W]

Under torchrun (N > 1) every rank runs its own replica of the workload (the
trees and samples are independent; no collective on the data path) and
rank 0 prints the aggregate.  --impl reference times the CPU oracle on a
bounded sample of the same workload on this host's cores.
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "stress node-steps/s; full-chip TTF time at <=0.05% TTF error, plain vs chosen"
WORKLOAD = ("2048x2048-stripe two-layer Cu mesh at 5 um (the full chip): 4,096 trees x 20,471 stress nodes "
            "(83.8 M), 4.19 M IR nodes, a pad every 32 crossings, 5 %% lognormal sinks, 330 K + 8 hotspots; "
            "%d Monte Carlo samples (20 %% CoV kappa and sigma_crit per segment) held at once, coefficients "
            "rebuilt in windows of %d samples; one step = one aging step (256 BE steps, void update, IR re-solve) "
            "of every sample")


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(ms, dist, device):
    """The step time every rank reports is the slowest rank's (replicas: each
    rank times its own copy of the workload; one all-reduce on the timing,
    none on the data path)."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(node_steps_per_step, steps, world, ms):
    """Whole-job throughput: the node-steps of all ranks over the slowest
    rank's time (weak scaling: every rank runs the full workload)."""
    return node_steps_per_step * steps * world / (ms / 1e3)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1])); mx = max(mx, float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                pass
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _result_error(ref, run):
    """Largest relative difference of TTF (where the reference's is finite)
    and final IR drop between two TTF results; inf when the sets of failed
    samples differ."""
    import numpy as np
    fr, fx = np.isfinite(ref["ttf"]), np.isfinite(run["ttf"])
    if np.any(fr != fx):
        return math.inf
    e = float(np.max(np.abs(run["final_drop"] - ref["final_drop"]) / ref["final_drop"]))
    if fr.any():
        t = ref["ttf"][fr]
        e = max(e, float(np.max(np.abs(run["ttf"][fr] - t) / np.maximum(t, 1e-30))))
    return e


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def _finite(o):
    """JSON-safe copy: non-finite floats (a censored TTF is +inf) become null."""
    if isinstance(o, float):
        return o if math.isfinite(o) else None
    if isinstance(o, dict):
        return {k: _finite(v) for k, v in o.items()}
    if isinstance(o, (list, tuple)):
        return [_finite(v) for v in o]
    return o


def full_chip(n_samples, seed=5):
    """The 2048 x 2048 full chip with n_samples Monte Carlo factor sets."""
    import ems_synth as es
    return es.grid.large_grid(seed=seed, n_samples=n_samples)


def tuned_rules(p, prec, args):
    """Chain shapes of the full chip picked by the autotuner (ems_autotune),
    measured on a 2-sample copy of the workload: the chains and their launch
    groups are the same, the samples only multiply the launch size."""
    from paper_2604_10743_gb300.engine import Engine
    t0 = time.perf_counter()
    e = Engine(p, full_chip(2), precision=prec, max_voids=args.max_voids)
    e.ir_solve()
    table = e.autotune(n_steps=32, max_samples=2)
    log = e.autotune_log()
    e.close()
    for k, r in enumerate(table):
        r["candidates"] = [{"kernel": x["kernel"], "M": x["M"], "CL": x["CL"], "T": x["T"], "ms": round(x["ms"], 3)}
                           for x in log if x["group"] == k]
    return table, time.perf_counter() - t0


def source_sha1(files):
    """SHA-1 over the bytes of the named repository files, in order (None
    when one is missing): ties a stored profiler capture to the kernel
    source it was taken on."""
    h = hashlib.sha1()
    for f in files:
        try:
            with open(os.path.join(ROOT, f), "rb") as fh:
                h.update(fh.read())
        except OSError:
            return None
    return h.hexdigest() if files else None


def kernel_name(rule, prec_name):
    r = "float" if prec_name == "f32" else "double"
    if rule["kernel"] == "cluster":
        return "k_chain_cl<%s,%d,%d>" % (r, rule["M"], rule["CL"])
    if rule["kernel"] == "cluster_shared":
        return "k_chain_cl<%s,%d,%d,smem>" % (r, rule["M"], rule["CL"])
    if rule["kernel"] == "register":
        return "k_chain_reg<%d>" % rule["M"]
    return "k_chain<%s,%d,%s>" % (r, rule["M"], "shared" if rule["kernel"] == "shared" else "global")


def run_mine(args):
    import numpy as np
    import torch

    import ems_synth as es
    from paper_2604_10743_gb300 import EMS_F32, EMS_F64
    from paper_2604_10743_gb300.engine import Engine

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    S, W = args.samples, args.window
    p = es.default_params()
    prec = EMS_F32 if args.precision == "f32" else EMS_F64
    rules, tune_s = ([], 0.0) if args.no_tune else tuned_rules(p, prec, args)
    g = full_chip(S)
    t0 = time.perf_counter()
    eng = Engine(p, g, precision=prec, max_voids=args.max_voids, window=W, chain_rules=rules)
    torch.cuda.synchronize()
    t_load = time.perf_counter() - t0
    stream = torch.cuda.current_stream()

    # one step = one aging step (256 BE steps of every tree of every sample,
    # void update, IR re-solve, drop) of the whole Monte Carlo batch; steps
    # follow each other along the horizon (warm-up steps included)
    def one():
        return eng.ttf(n_outer=1)

    for _ in range(args.warmup):
        one()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    l0 = eng.launch_count()
    clk = ClockSampler(local)
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    stress_ms = ir_ms = 0.0
    res = None
    for _ in range(args.steps):
        res = one()
        stress_ms += res["stress_ms"]
        ir_ms += res["ir_ms"]
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    launches = eng.launch_count() - l0
    ms = e0.elapsed_time(e1)
    if world > 1:
        ms = max_over_ranks(ms, dist, "cuda")
        dist.barrier()
    node_steps = res["node_steps"]                      # per step: nodes x samples x 256
    value = job_value(node_steps, args.steps, world, ms)
    n_win = (S + W - 1) // W if 0 < W < S else 1
    voids = int(np.asarray(res["n_voids"]).sum())

    # dominant kernel: the cluster chain kernel (one launch = 256 BE steps of
    # every tree of one window of samples).  Algorithmic bytes per node-step:
    # state in + out (2w), plus the per-launch coefficient arrays.
    w = 4 if prec == EMS_F32 else 8
    n_inner = p["n_inner"]
    from paper_2604_10743_gb300 import _abi as A
    shape = rules[0] if rules else A.chain_candidates(int(eng.n_stress // eng.n_trees), prec)[0]
    kname = kernel_name(shape, args.precision)
    n_coef = 7 if prec == EMS_F32 else 6
    nodes_launch = eng.n_stress * (S / n_win)
    alg_bytes_launch = nodes_launch * (2 * w * n_inner + n_coef * w)
    per_launch_ms = stress_ms / (args.steps * n_win)
    peaks, src = _peaks()
    achieved = alg_bytes_launch / (per_launch_ms / 1e3) / 1e9
    traffic = None
    traffic_note = None
    issue = None
    tf = os.path.join(ROOT, "profiles", "chain_kernel_traffic.json")
    if os.path.exists(tf):
        try:
            for t in json.load(open(tf)).get("captures", []):
                if t.get("precision") == args.precision and t.get("kernel") == kname:
                    # counters of another build of the kernel do not count
                    if source_sha1(t.get("source_files", [])) != t.get("source_sha1"):
                        traffic_note = "kernel source changed since the ncu capture (%s)" % t.get("captured_at", "?")
                        break
                    traffic = t.get("bytes_per_launch")
                    if t.get("issue_active_pct") is not None:
                        issue = {"issue_active_frac": t["issue_active_pct"] / 100.0,
                                 "fma_pipe_active_frac": t["fma_pipe_active_pct"] / 100.0,
                                 "source": "ncu, " + t.get("command", "")}
        except (OSError, ValueError):
            pass
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": traffic,
            "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % src if src == "measured" else "fallback 6.8 TB/s",
            "kernel": "%s (stress advance, the autotuner's shape for the 20,471-node stripes; one launch = "
                      "256 BE steps of every stripe of %d samples)" % (kname, S // n_win),
            "alg_bytes_per_launch": int(alg_bytes_launch), "launch_ms": round(per_launch_ms, 3),
            "issue_roof": issue}
    if traffic_note:
        roof["traffic_note"] = traffic_note

    # end to end through the public API with host buffers: the netlist, the
    # map and the factor sets copied in, then aging steps with every step's
    # drops and TTF read back
    e2e = None
    if not args.no_e2e:
        eng.close()
        h2d = sum(np.asarray(g[k]).nbytes for k in ("node_x", "node_y", "seg_a", "seg_b", "seg_layer",
                                                      "seg_cells", "seg_R0", "seg_W", "seg_H", "seg_L",
                                                      "pad_node", "pad_V", "sink_node", "sink_I",
                                                      "kappa_factor", "sigc_factor"))
        h2d += g["thermal"]["T"].nbytes
        ke = 3
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e = Engine(p, g, precision=prec, max_voids=args.max_voids, window=W, chain_rules=rules)
        for _ in range(ke):
            r = e.ttf(n_outer=1)                      # results come back to the host
        torch.cuda.synchronize()
        dt_e = time.perf_counter() - t0
        e.close()
        d2h = S * (8 * 3 + 4 + 8 * 2)
        e2e = {"value": node_steps * ke * world / dt_e, "unit": "node-steps/s",
               "h2d_bytes_per_step": int(h2d / ke), "d2h_bytes_per_step": int(d2h),
               "s_total": round(dt_e, 2), "steps": ke,
               "note": "one context built from host arrays (netlist, map, %d factor sets), then %d aging steps "
                       "with results read back each step; the load is spread over the steps" % (S, ke)}
    else:
        eng.close()

    # plain vs chosen on the full chip: whole TTF runs of one Monte Carlo
    # sample (the batch's first factor set): plain = FP64 backward Euler;
    # chosen = the FP32 path timed above (cluster kernel, compensated sums)
    pvc = None
    if not args.no_plain:
        pvc = plain_vs_chosen(p, args, stream, rules, n_samples=args.mc_samples)

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(p)

    mc = None
    if not args.no_mc:
        mc = mc_leg(p, peaks, src, stream)

    surrogate = None
    sched = None
    if not args.no_surrogate:
        surrogate = surrogate_leg(peaks, src, stream, rows=args.surrogate_rows)
        # what the learned part buys: the trained surrogate's step schedule on
        # an unseen Monte Carlo workload, against the plain solver
        sched = schedule_leg(p, stream)

    line = {
        "metric": METRIC, "value": value, "unit": "node-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (stress, increment form, compensated sums) / f64 (IR PCG, nucleation time)"
                 if prec == EMS_F32 else "f64",
        "data": "synthetic (seeded generator; the paper's SAED32 netlists and maps are not available)",
        "config": {"workload": WORKLOAD % (S, W), "trees": eng.n_trees, "stress_nodes": eng.n_stress,
                   "samples": S, "window_samples": W, "node_steps_per_step": node_steps,
                   "precision": args.precision, "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "no flush: the per-step working set (%d samples x 83.8 M nodes of state, %d samples of "
                         "coefficients) is far larger than the 129 MB L2" % (S, S // n_win),
                   "workspace_gb": round(eng.ws_bytes / 1e9, 2), "load_s": round(t_load, 1)},
        "stress_node_steps_per_s": node_steps * args.steps / (stress_ms / 1e3),
        "stress_ms_per_step": round(stress_ms / args.steps, 1), "ir_ms_per_step": round(ir_ms / args.steps, 1),
        "voids_after_timed_steps": voids, "max_drop_after_timed_steps": float(np.max(res["final_drop"])),
        "plain_vs_chosen": pvc, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clocks, "surrogate": surrogate, "surrogate_schedule": sched, "monte_carlo": mc,
        "autotune": None if args.no_tune else {
            "table": rules, "tune_s": round(tune_s, 2),
            "how": "ems_autotune on a 2-sample copy of the full chip (after one IR solve): every valid shape of "
                   "each launch group timed over 32 BE steps after a factorising launch, on scratch copies; the "
                   "fastest applied by loading with ems_set_chain_rules (the load and tuning are not timed)"},
    }
    if rank == 0:
        print(json.dumps(_finite(line)))
    if world > 1:
        dist.destroy_process_group()


def chosen_scheduled(p, args, stream, rules, g, seeds=(6, 7)):
    """The chosen path plus the learned step schedule on the full chip: the
    surrogate trained on the plain solver's records of the full chip at
    another seed (one Monte Carlo sample: 4,096 (tree, sample) records), its
    skip bound validated end to end on a third seed, then the benchmark
    grid's TTF run with the schedule (CUDA events), with executed node-steps."""
    import torch
    from paper_2604_10743_gb300 import EMS_F32
    from paper_2604_10743_gb300 import surrogate as sg
    from paper_2604_10743_gb300.engine import Engine
    t0 = time.perf_counter()
    x, t = sg.generate_records(full_chip(1, seed=seeds[0]), p)
    m = sg.Mlp(n_hidden=4, seed=0)
    m.fit_norm(x, t)
    losses = m.train(x, t, batch=1024, epochs=60, lr=1e-3, seed=1)
    bound, log = sg.validate_bound(m, [full_chip(1, seed=seeds[1])], p, coarsen=16, guard=0.8,
                                   candidates=(-0.3, 0.0, 0.3, 0.6), max_voids=args.max_voids)
    t_prep = time.perf_counter() - t0
    res = {"train_seed": seeds[0], "validation_seed": seeds[1], "records": int(x.shape[0]),
           "final_loss_ratio": float(losses[-1] / losses[0]), "bound": bound, "validation": log,
           "prep_s": round(t_prep, 1)}
    if not math.isfinite(bound):
        res["note"] = "no candidate bound passed validation: the schedule is not used"
        return res
    eng = Engine(p, g, precision=EMS_F32, max_voids=args.max_voids, chain_rules=rules)
    eng.ir_solve()
    n_coarse, _ = eng.schedule(m, bound, 16, 0.8)
    a0 = torch.cuda.Event(enable_timing=True); a1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a0.record(stream)
    r = eng.ttf()
    a1.record(stream)
    torch.cuda.synchronize()
    tm = a0.elapsed_time(a1)
    res.update({"ttf_s": [float(v) for v in r["ttf"]], "final_drop": [float(v) for v in r["final_drop"]],
                "ttf_wall_ms": round(tm, 1), "stress_ms": round(r["stress_ms"], 1), "ir_ms": round(r["ir_ms"], 1),
                "coarse_trees": [int(v) for v in (n_coarse.cpu() if hasattr(n_coarse, "cpu") else n_coarse)],
                "node_steps_executed_ratio": r["node_steps_executed"] / r["node_steps"]})
    eng.close()
    return res


def plain_vs_chosen(p, args, stream, rules, n_samples=1, sched=True):
    """Full-chip TTF of the same sample(s), plain FP64 method (built-in
    shapes) against the chosen FP32 path (the autotuner's shapes): wall time
    (CUDA events), TTF, final IR drop, errors."""
    import numpy as np
    import torch
    from paper_2604_10743_gb300 import EMS_F32, EMS_F64
    from paper_2604_10743_gb300.engine import Engine
    g = full_chip(n_samples)
    out = {}
    for name, prec in (("chosen", EMS_F32), ("plain", EMS_F64)):
        eng = Engine(p, g, precision=prec, max_voids=args.max_voids, chain_rules=rules if prec == EMS_F32 else None)
        a0 = torch.cuda.Event(enable_timing=True); a1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a0.record(stream)
        r = eng.ttf()
        a1.record(stream)
        torch.cuda.synchronize()
        t = a0.elapsed_time(a1)
        out[name] = {"ttf_s": [float(v) for v in r["ttf"]], "final_drop": [float(v) for v in r["final_drop"]],
                     "ttf_wall_ms": round(t, 1), "stress_ms": round(r["stress_ms"], 1), "ir_ms": round(r["ir_ms"], 1),
                     "voids": [int(v) for v in r["n_voids"]],
                     "node_steps_per_s": r["node_steps"] / (t / 1e3),
                     "precision": "f32" if prec == EMS_F32 else "f64"}
        eng.close()
    rc, rp = out["chosen"], out["plain"]

    def rel_err(rc, rp):
        err = 0.0
        for a, b in zip(rc["final_drop"], rp["final_drop"]):
            err = max(err, abs(a - b) / b)
        for a, b in zip(rc["ttf_s"], rp["ttf_s"]):
            if math.isfinite(b):
                err = max(err, abs(a - b) / b if math.isfinite(a) else math.inf)
            elif math.isfinite(a):
                err = math.inf
        return err
    out["max_rel_err_ttf_and_final_drop"] = rel_err(rc, rp)
    out["speedup"] = round(rp["ttf_wall_ms"] / rc["ttf_wall_ms"], 3)
    if sched:
        out["chosen_scheduled"] = chosen_scheduled(p, args, stream, rules, g)
        rs = out["chosen_scheduled"]
        rs["max_rel_err_ttf_and_final_drop"] = rel_err(rs, rp)
        rs["speedup_vs_plain"] = round(rp["ttf_wall_ms"] / rs["ttf_wall_ms"], 3)
    out["samples"] = n_samples
    out["workload"] = "2048x2048 full chip, %d Monte Carlo sample(s), whole 10-year horizon (64 x 256 BE steps)" % \
        n_samples
    return out


def mid_grid_leg(args, stream):
    """The 256 x 256-stripe mesh (512 trees x 5,101 nodes): full TTF runs
    (64 x 256 BE steps) with inputs resident, FP32."""
    import torch
    import ems_synth as es
    from paper_2604_10743_gb300 import EMS_F32
    from paper_2604_10743_gb300.engine import Engine
    g, p = es.mid_grid(), es.default_params()
    eng = Engine(p, g, precision=EMS_F32)
    init = eng.state_export()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ms = []
    r = None
    for k in range(args.warmup + args.steps):
        eng.state_import(init)
        flush.fill_(1)
        a0 = torch.cuda.Event(enable_timing=True); a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        r = eng.ttf()
        a1.record(stream)
        torch.cuda.synchronize()
        if k >= args.warmup:
            ms.append(a0.elapsed_time(a1))
    t = sum(ms) / len(ms)
    eng.close()
    return {"workload": "256x256 mesh, 512 trees x 5,101 nodes, full TTF run", "ttf_wall_ms": round(t, 2),
            "node_steps_per_s": r["node_steps"] / (t / 1e3), "stress_ms": round(r["stress_ms"], 2),
            "ir_ms": round(r["ir_ms"], 2), "final_drop": float(r["final_drop"][0])}


def surrogate_leg(peaks, src, stream, rows=4096 * 1024, reps=10):
    """Inference throughput of the surrogate network (24 -> 4 x 256 -> 2,
    BF16 tensor cores, FP32 accumulate) on `rows` feature rows resident in
    HBM; roofline against the measured dense BF16 peak."""
    import numpy as np
    import torch
    from paper_2604_10743_gb300.surrogate import Mlp
    m = Mlp(n_hidden=4, seed=0)
    x = torch.randn(rows, 24, device="cuda", generator=torch.Generator(device="cuda").manual_seed(0))
    for _ in range(3):
        m.predict(x)
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        a0 = torch.cuda.Event(enable_timing=True); a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        m.predict(x)
        a1.record(stream)
        torch.cuda.synchronize()
        ms.append(a0.elapsed_time(a1))
    t = float(np.median(ms))
    flop_row = 2 * (24 * 256 + 3 * 256 * 256 + 256 * 2)        # algorithmic: 406,528 per row
    tflops = rows * flop_row / (t / 1e3) / 1e12
    m.close()
    return {"rows": rows, "ms_median": round(t, 4), "rows_per_s": rows / (t / 1e3),
            "flop_per_row": flop_row,
            "roofline": {"bound": "tensor", "achieved": round(tflops, 1), "peak": peaks["bf16_tflops"],
                         "unit": "TFLOP/s", "frac": round(tflops / peaks["bf16_tflops"], 4), "traffic": None,
                         "peak_source": ("measured (MEASURED_PEAKS.json bf16_tflops, burst)" if src == "measured"
                                         else "fallback 1.9 PFLOP/s"),
                         "kernel": "k_mlp_fused (all layers, 256 rows per CTA)"}}


def mc_leg(p, peaks, src, stream, n_samples=1024, reps=2):
    """Batched Monte Carlo: the 8 x 8 grid with uneven trees (32-1,024 cells
    per stripe) and n_samples lognormal kappa / sigma_crit samples, all
    advanced in one graph-captured TTF run; the oracle times one sample."""
    import torch
    import ems_synth as es
    from paper_2604_10743_gb300 import EMS_F32
    from paper_2604_10743_gb300.engine import Engine
    g = es.mc_grid(n_samples=n_samples)
    eng = Engine(p, g, precision=EMS_F32)
    init = eng.state_export()
    eng.ttf()                                        # warm-up (captures the graph)
    torch.cuda.synchronize()
    ms, r = [], None
    for _ in range(reps):
        eng.state_import(init)
        a0 = torch.cuda.Event(enable_timing=True); a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        r = eng.ttf()
        a1.record(stream)
        torch.cuda.synchronize()
        ms.append(a0.elapsed_time(a1))
    t = min(ms)
    out = {"workload": "8x8 grid, stripes of 32-1,024 FD cells, %d Monte Carlo samples (20 %% CoV kappa and "
                       "sigma_crit per segment), 64 x 256 BE steps" % n_samples,
           "samples": n_samples, "stress_nodes_per_sample": eng.n_stress, "ttf_wall_ms": round(t, 2),
           "node_steps_per_s": r["node_steps"] / (t / 1e3), "stress_ms": round(r["stress_ms"], 2),
           "ir_ms": round(r["ir_ms"], 2), "ttf_mean_s": r["ttf_mean"], "ttf_cov": r["ttf_cov"],
           "censored": r["n_censored"], "graph": r["graph"]}
    eng.close()
    from oracle import flow as F
    g1 = es.mc_grid(n_samples=n_samples)
    g1["trees"] = F.build_trees(g1)
    t0 = time.perf_counter()
    ro = F.run_ttf(g1, p, sample=0)
    dt = time.perf_counter() - t0
    out["cpu_baseline"] = {"value": ro["node_steps"] / dt, "unit": "node-steps/s", "cores": os.cpu_count(),
                           "kind": "oracle", "sample": "sample 0 of the same workload, full TTF run",
                           "seconds": round(dt, 2)}
    return out


def krylov_leg(g, p, stream, be, q=20, oracle=True):
    """The rational Krylov reduced models (method AUTO, order q, cached bases
    extended by the current starting block) on the bench workload: TTF wall
    time and the final-drop difference from the BE run (the paper's metric
    when no sample fails); the oracle times its Krylov stepper over one
    aging step of the same grid."""
    import torch
    from paper_2604_10743_gb300 import EMS_F32
    from paper_2604_10743_gb300 import _abi as A
    from paper_2604_10743_gb300.engine import Engine
    pk = dict(p, krylov_q=q)
    eng = Engine(pk, g, precision=EMS_F32, method=A.EMS_AUTO, max_voids=32)
    init = eng.state_export()
    eng.ttf()
    torch.cuda.synchronize()
    eng.state_import(init)
    a0 = torch.cuda.Event(enable_timing=True); a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    r = eng.ttf()
    a1.record(stream)
    torch.cuda.synchronize()
    t = a0.elapsed_time(a1)
    nv = int(r["n_voids"][0])
    eng.close()
    out = {"q": q, "ttf_wall_ms": round(t, 2), "stress_ms": round(r["stress_ms"], 2), "ir_ms": round(r["ir_ms"], 2),
           "node_steps_per_s": r["node_steps"] / (t / 1e3), "graph": r["graph"], "voids": nv,
           "final_drop_rel_diff_vs_be": abs(r["final_drop"][0] - be["final_drop"][0]) / be["final_drop"][0]}
    if not oracle:
        return out
    from oracle import flow as F, krylov as K
    g1 = dict(g)
    g1["trees"] = F.build_trees(g1)
    t0 = time.perf_counter()
    ro = F.run_ttf(g1, pk, n_outer=1, stepper=K.KrylovStepper(q=q, eta=1.0, n_threads=os.cpu_count()))
    dt = time.perf_counter() - t0
    out["cpu_baseline"] = {"value": ro["node_steps"] / dt, "unit": "node-steps/s (full-order equivalent)",
                           "cores": os.cpu_count(), "kind": "oracle",
                           "sample": "1 of 64 aging steps (bases built), all 512 trees, Krylov stepper",
                           "seconds": round(dt, 2)}
    return out


def schedule_leg(p, stream, n_train=24, n_valid=3, test_seed=3000, N=64, S=32):
    """What the learned part buys: the surrogate trained on the plain
    solver's records of n_train seeded N x N grids (S Monte Carlo samples
    each), its skip bound validated end to end on n_valid more, then the
    S-sample TTF run of an unseen grid with and without the step schedule:
    wall time, executed node-steps and the largest TTF / final-drop error."""
    import numpy as np
    import torch
    import ems_synth as es
    from paper_2604_10743_gb300 import EMS_F32
    from paper_2604_10743_gb300 import surrogate as sg
    from paper_2604_10743_gb300.engine import Engine

    def grid(seed):
        g = es.grid.surrogate_grid(seed=seed, N=N, n_samples=S)
        return sg.scale_to_drop(g, p, np.random.default_rng(seed + 7).uniform(0.07, 0.095))

    t0 = time.perf_counter()
    xs, ts = [], []
    for seed in range(1000, 1000 + n_train):
        x, t = sg.generate_records(grid(seed), p)
        xs.append(x); ts.append(t)
    X, T = torch.cat(xs), torch.cat(ts)
    m = sg.Mlp(n_hidden=4, seed=0)
    m.fit_norm(X, T)
    losses = m.train(X, T, batch=1024, epochs=30, lr=1e-3, seed=1)
    bound, _ = sg.validate_bound(m, [grid(2000 + k) for k in range(n_valid)], p, coarsen=16, guard=0.8,
                                 candidates=(-0.3, 0.0, 0.3, 0.6, 1.0))
    t_prep = time.perf_counter() - t0
    g = grid(test_seed)

    def run(scheduled):
        eng = Engine(p, g, precision=EMS_F32, max_voids=32)
        init = eng.state_export()
        ms, r = [], None
        for rep in range(3):
            eng.state_import(init)
            eng.ir_solve()
            n = None
            if scheduled:
                n, _ = eng.schedule(m, bound, 16, 0.8)
            torch.cuda.synchronize()
            a0 = torch.cuda.Event(enable_timing=True); a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            r = eng.ttf()
            a1.record(stream)
            torch.cuda.synchronize()
            if rep > 0:
                ms.append(a0.elapsed_time(a1))
        eng.close()
        return min(ms), r, n

    t_plain, r_plain, _ = run(False)
    t_sched, r_sched, n_coarse = run(True)
    return {"workload": "%d x %d stripes at 10 um, %d Monte Carlo samples, unseen test grid (seed %d); network "
                        "trained on %d grids, bound validated on %d" % (N, N, S, test_seed, n_train, n_valid),
            "records": int(X.shape[0]), "final_loss_ratio": float(losses[-1] / losses[0]),
            "bound": bound, "prep_s": round(t_prep, 1),
            "coarse_trees_frac": float(np.asarray(n_coarse.cpu() if hasattr(n_coarse, "cpu") else n_coarse).sum())
                                 / (S * 2 * N),
            "plain_ttf_ms": round(t_plain, 2), "scheduled_ttf_ms": round(t_sched, 2),
            "speedup": round(t_plain / t_sched, 3),
            "node_steps_executed_ratio": r_sched["node_steps_executed"] / r_plain["node_steps_executed"],
            "max_rel_err_ttf_or_final_drop": _result_error(r_plain, r_sched)}


def cluster_stripes_case(n_samples=20, cells=2924, shape=None):
    """Small case of the cluster chain kernel for a profiler capture: 16
    stripes of 7 x cells + 1 stress nodes (full-chip length for cells =
    2,924), the 8 x 8 grid's pads and sinks, a 33 x 33 hotspot map, n_samples
    factor sets; two aging steps of 256 BE steps, FP32.  shape "KIND:CL"
    (e.g. "cluster_shared:4") overrides the built-in chain shape."""
    import numpy as np
    import torch
    import ems_synth as es
    from paper_2604_10743_gb300 import EMS_F32
    from paper_2604_10743_gb300.engine import Engine
    g = es.stripe_mesh(8, 20e-6)
    g["seg_cells"][:] = cells
    t = es.tiny_grid()
    g["pad_node"], g["pad_V"], g["sink_node"], g["sink_I"] = t["pad_node"], t["pad_V"], t["sink_node"], t["sink_I"]
    g["thermal"] = es.hotspot_raster(np.random.default_rng(4), 140e-6, 2, 360.0, 20.0, 40.0, 0.2, nx=33, ny=33)
    g["kappa_factor"], g["sigc_factor"] = es.mc_factors(np.random.default_rng(3), n_samples, g["seg_a"].size)
    p = es.default_params(n_outer=4, n_inner=256)
    rules = None
    if shape:
        from paper_2604_10743_gb300 import _abi as A
        kind, cl = shape.split(":")
        kinds = {v: k for k, v in A.CHAIN_KINDS.items()}
        rules = [dict(n_lo=1, n_hi=10 ** 9, kind=kinds[kind], M=16, CL=int(cl))]
    eng = Engine(p, g, precision=EMS_F32, max_voids=64, chain_rules=rules)
    r = eng.ttf(n_outer=2)
    torch.cuda.synchronize()
    out = {"stress_ms": r["stress_ms"], "voids": int(r["n_voids"].sum()),
           "node_steps_per_s": r["node_steps"] / (r["stress_ms"] / 1e3)}
    eng.close()
    return out


def ir_mg_case(N=1024, n_samples=4):
    """Small case of the multigrid IR PCG for a profiler capture: the full
    chip's pitch, pads, sinks and map on an N x N mesh (N^2 IR nodes; 4
    samples are 0.5 GB of matrix and vectors, past the L2), one solve from
    zero."""
    import torch
    import ems_synth as es
    from paper_2604_10743_gb300 import EMS_F32
    from paper_2604_10743_gb300.engine import Engine
    g = es.grid.large_grid(N=N, n_samples=n_samples)
    eng = Engine(es.default_params(), g, precision=EMS_F32)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    eng.ir_solve()
    torch.cuda.synchronize()
    out = {"solve_ms": round((time.perf_counter() - t0) * 1e3, 2),
           "iterations": [int(v) for v in eng.ir_iterations()]}
    eng.close()
    return out


def corner_grid(n=256):
    """The n x n-crossing corner of the full chip: the same pitch, pads, sinks
    and thermal map, cut out of the 2048 x 2048 netlist (array selection
    only)."""
    import numpy as np
    g = full_chip(0)
    N = 2048
    ii, jj = np.divmod(np.arange(N * N), N)
    keep = (ii < n) & (jj < n)
    new_id = -np.ones(N * N, np.int64)
    new_id[keep] = ii[keep] * n + jj[keep]
    a, b = np.asarray(g["seg_a"]), np.asarray(g["seg_b"])
    sk = keep[a] & keep[b]
    out = dict(g)
    out.update(N=n, node_x=g["node_x"][keep], node_y=g["node_y"][keep],
               seg_a=new_id[a[sk]].astype(np.int32), seg_b=new_id[b[sk]].astype(np.int32))
    for k in ("seg_layer", "seg_cells", "seg_R0", "seg_W", "seg_H", "seg_L"):
        out[k] = np.asarray(g[k])[sk]
    pk = keep[g["pad_node"]]
    out["pad_node"] = new_id[g["pad_node"][pk]].astype(np.int32); out["pad_V"] = g["pad_V"][pk]
    sk2 = keep[g["sink_node"]]
    out["sink_node"] = new_id[g["sink_node"][sk2]].astype(np.int32); out["sink_I"] = g["sink_I"][sk2]
    return out


def cpu_baseline(p, n_outer=1):
    """The CPU oracle, as it stands, on a bounded sample of the workload: the
    256 x 256-crossing corner of the full chip (512 stripes x 2,551 nodes),
    one sample, n_outer aging steps including the IR solves."""
    from oracle import flow as F
    g = corner_grid()
    g["trees"] = F.build_trees(g)
    t0 = time.perf_counter()
    r = F.run_ttf(g, p, n_outer=n_outer, n_threads=os.cpu_count() or 0)
    dt = time.perf_counter() - t0
    return {"value": r["node_steps"] / dt, "unit": "node-steps/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "%d aging step(s) of the 256x256-crossing corner of the full chip (512 stripes x 2,551 "
                      "nodes, same pitch, sinks and map), one Monte Carlo sample, IR solves included" % n_outer,
            "seconds": round(dt, 2)}


def run_reference(args):
    rank, world, local = _dist()
    if rank != 0:
        return
    import ems_synth as es
    from oracle import flow as F
    g = corner_grid()
    p = es.default_params()
    g["trees"] = F.build_trees(g)
    nt = os.cpu_count() or 0
    for _ in range(args.warmup):
        F.run_ttf(g, p, n_outer=1, n_threads=nt)
    t0 = time.perf_counter()
    ns = 0
    for _ in range(args.steps):
        r = F.run_ttf(g, p, n_outer=1, n_threads=nt)
        ns += r["node_steps"]
    dt = time.perf_counter() - t0
    v = ns / dt
    cores = os.cpu_count()
    sample = ("1 aging step per step of the 256x256-crossing corner of the full chip (512 stripes x 2,551 nodes, "
              "same pitch, sinks and map), one Monte Carlo sample, IR solve included")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "node-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD % (args.samples, args.window), "sample": sample},
            "cpu_baseline": {"value": v, "unit": "node-steps/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "node-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-mc", action="store_true")
    ap.add_argument("--krylov", action="store_true", help="also time the Krylov reduced model (slow oracle leg)")
    ap.add_argument("--schedule-only", action="store_true",
                    help="train the surrogate and time a Monte Carlo TTF run with and without its step schedule")
    ap.add_argument("--krylov-only", action="store_true",
                    help="time only the Krylov TTF run and its BE reference (profiling); prints its own JSON line")
    ap.add_argument("--surrogate-only", action="store_true",
                    help="time only the surrogate inference (profiling); prints its own JSON line")
    ap.add_argument("--surrogate-rows", type=int, default=4096 * 1024)
    ap.add_argument("--samples", type=int, default=24, help="Monte Carlo samples of the full chip held at once")
    ap.add_argument("--window", type=int, default=8, help="samples whose coefficients are held at once")
    ap.add_argument("--max-voids", type=int, default=128)
    ap.add_argument("--no-tune", action="store_true", help="built-in chain shapes instead of the autotuner's")
    ap.add_argument("--mc-samples", type=int, default=1,
                    help="Monte Carlo samples of the full-chip plain vs chosen TTF comparison (plain FP64 takes "
                         "about 100 s per sample)")
    ap.add_argument("--profile-case", choices=["cluster-stripes", "ir-mg"],
                    help="run one small case of a kernel for an ncu capture: cluster-stripes = 16 stripes of "
                         "20,469 nodes x 20 Monte Carlo samples, two aging steps (k_chain_cl on 4-CTA clusters); "
                         "ir-mg = two IR solves of a 1024 x 1024 mesh (1.05 M unknowns) for 4 samples "
                         "(k_pcg_cluster_mg)")
    ap.add_argument("--profile-shape", default=None,
                    help="with --profile-case cluster-stripes: chain shape KIND:CL, e.g. cluster_shared:4")
    ap.add_argument("--mid-only", action="store_true",
                    help="time only full TTF runs of the 256 x 256 mesh; prints its own JSON line")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        import __graft_entry__ as ge
        ge.build()
        if args.profile_case == "cluster-stripes":
            print(json.dumps({"profile_case": cluster_stripes_case(shape=args.profile_shape)}))
        elif args.profile_case == "ir-mg":
            print(json.dumps({"profile_case": ir_mg_case()}))
        elif args.schedule_only:
            import torch
            import ems_synth as es
            print(json.dumps({"surrogate_schedule": schedule_leg(es.default_params(), torch.cuda.current_stream())}))
        elif args.mid_only:
            import torch
            print(json.dumps({"mid": mid_grid_leg(args, torch.cuda.current_stream())}))
        elif args.krylov_only:
            import torch
            import ems_synth as es
            from paper_2604_10743_gb300 import EMS_F32
            from paper_2604_10743_gb300.engine import Engine
            g, p = es.mid_grid(), es.default_params()
            e = Engine(p, g, precision=EMS_F32)
            be = e.ttf()
            e.close()
            print(json.dumps({"krylov": krylov_leg(g, p, torch.cuda.current_stream(), be, oracle=not args.no_cpu)}))
        elif args.surrogate_only:
            import torch
            peaks, src = _peaks()
            print(json.dumps({"surrogate": surrogate_leg(peaks, src, torch.cuda.current_stream(),
                                                         rows=args.surrogate_rows, reps=max(1, args.steps))}))
        else:
            run_mine(args)


if __name__ == "__main__":
    main()
