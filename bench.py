"""Benchmark of the GB300 UTIL-table library.

Headline workload: exact Bucket Elimination on the 12x12 grid WCSP (144
variables, domain 4, binary int32 tables U[0,1000], natural order, induced
width 12, largest bucket table 4^13 joint entries).  One step = the whole hot
path on device-resident tables: every bucket function (UTIL kernel, one
persistent launch per elimination-tree level, replayed from a CUDA graph),
the root reduction and the VALUE phase.  Metric: UTIL entries per second
(joint separator x eliminated-variable rows of every bucket).

Also reported on the same line: the HBM roofline of the UTIL kernel, the
end-to-end solve through the C ABI from host buffers (wcsp_load + be_solve,
uploads and result copy included), the oracle on the host cores, and the
secondary workloads (level-batched vs per-bucket MBE on the Erdos-Renyi
WCSP, MPE in the -log domain, sum-product -log Z on the grid shape, DCOP
serving latency).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Multi-GPU (torchrun): every rank solves its own instance (independent
replicas, weak scaling); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "UTIL entries/s"
UNIT = "entries/s"
WORKLOAD = "BE 12x12 grid WCSP, d=4, int32 U[0,1000], natural order (w*=12, max table 4^13)"
L2_FLUSH_BYTES = 512 << 20
# tuned launch shapes (CTA size, rows per item) per plan, kept beside the build
TUNE_CACHE = os.path.join(ROOT, "paper_1608_05288_gb300", "_build", "autotune.txt")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def max_over_ranks(seconds, device):
    """The slowest rank's time (every rank gets it); the local time when not
    distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(seconds)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step, world, steps, seconds):
    """Units processed by all ranks (independent replicas) per second of the
    slowest rank."""
    return units_per_rank_step * world * steps / seconds


def _traffic_per_launch(alg_bytes_per_launch):
    """DRAM bytes per UTIL launch of the headline step, from the committed ncu
    capture of full-size launches of the same grid (traffic taken as
    proportional to algorithmic bytes), or None when the kernel source changed
    since that capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        src = os.path.join(ROOT, "paper_1608_05288_gb300", "csrc", "util_kernel.cuh")
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        if t.get("source_sha256_16") != h:
            return None
        return t["full_launch_dram_bytes"] / t["full_launch_alg_bytes"] * alg_bytes_per_launch
    except Exception:
        return None


class Clocks:
    """nvidia-smi samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


CPU_ROWS = 4  # grid rows in the oracle's bounded sample (all host cores)
CPU_ROWS_1T = 2  # grid rows in the single-thread sample


def cpu_sample_instance(rows=CPU_ROWS):
    """The first `rows` rows of the headline grid (same tables, same natural
    order): a bounded piece of the same workload for the oracle."""
    import synth
    inst = synth.config_instance(1, 0)
    nv = 12 * rows
    keep = [j for j, s in enumerate(inst.scopes) if int(np.max(s)) < nv]
    return synth.Instance(f"grid12x12_rows0-{rows - 1}", inst.dom[:nv].copy(),
                          [inst.scopes[j] for j in keep], [inst.tables[j] for j in keep], "int",
                          inst.top_k)


def cpu_oracle_step(threads=0, rows=CPU_ROWS):
    """One oracle pass over the bounded sample, on `threads` host threads
    (0: all); returns (entries, seconds, threads)."""
    import oracle
    inst = cpu_sample_instance(rows)
    th = threads or oracle.max_threads()
    oracle.set_threads(th)
    t0 = time.perf_counter()
    run = oracle.eliminate(inst, np.arange(inst.n), "be", tables=False)
    dt = time.perf_counter() - t0
    entries = sum(int(t.rows) * int(inst.dom[t.var]) for t in run.tasks)
    return entries, dt, th


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        cpu_oracle_step()
    tot_e, tot_t, th = 0, 0.0, 1
    for _ in range(args.steps):
        e, t, th = cpu_oracle_step()
        tot_e += e
        tot_t += t
    v = tot_e / tot_t
    sample = f"oracle BE on rows 0-{CPU_ROWS - 1} of the 12x12 grid ({12 * CPU_ROWS} variables, natural order), every step"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": th, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def secondary(torch, gb, synth, steps):
    """Batched vs per-bucket MBE (Erdos-Renyi), MPE entries/s, sum-product
    -log Z on the grid shape, DCOP serving."""
    out = {}
    peak, _ = _peaks()
    # level-batched vs one launch per bucket, MBE log2 <= 16: each form with
    # direct launches and replayed from a CUDA graph (so graph replay and
    # batching are measured apart), the launch over all levels, and the
    # autotuned configuration
    inst = synth.config_instance(2, 0)
    times = {}
    for name, kw in (("batched", dict(batched=1, use_graph=True)),
                     ("batched_direct", dict(batched=1, use_graph=False)),
                     ("plain", dict(batched=0, use_graph=False)),
                     ("plain_graph", dict(batched=0, use_graph=True)),
                     ("fused", dict(batched=2, use_graph=True)),
                     ("tuned", dict(batched=1, use_graph=True, autotune_cache=TUNE_CACHE))):
        st = gb.UtilState(inst, "mbe", 16, ibound_mode="log2", **kw)
        st.bind()
        if name == "tuned":
            st.autotune()
            tuned_cfg = st.launch_config()
        ms = []
        for k in range(3 + steps):
            st.run()
            st.sync()
            if k >= 3:
                ms.append(st.times()[0])
        times[name] = statistics.median(ms)
        info = st.info()
        st.free()
    out["mbe_er500"] = {"workload": "MBE Erdos-Renyi n=500, 1500 ternary tables, log2 bound 16",
                        "tasks": info["n_tasks"], "levels": info["n_levels"],
                        "util_entries": info["util_entries"],
                        "batched_ms": times["batched"], "batched_direct_ms": times["batched_direct"],
                        "plain_ms": times["plain"], "plain_graph_ms": times["plain_graph"],
                        "fused_ms": times["fused"], "tuned_ms": times["tuned"], "tuned_config": tuned_cfg,
                        "batched_speedup": times["plain"] / times["batched"],
                        "batched_speedup_both_graph": times["plain_graph"] / times["batched"],
                        "batched_speedup_both_direct": times["plain"] / times["batched_direct"],
                        "tuned_speedup_vs_plain_graph": times["plain_graph"] / times["tuned"]}
    # MPE, -log p in fp32, MBE i = 20 (autotuned launch configuration)
    inst = synth.config_instance(3, 0)
    st = gb.UtilState(inst, "mbe", 20, ibound_mode="sep", use_graph=True, autotune_cache=TUNE_CACHE)
    st.bind()
    st.autotune()
    mpe_cfg = st.launch_config()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    ms = []
    for k in range(3 + steps):
        flush.fill_(k & 0xFF)
        st.run()
        st.sync()
        if k >= 3:
            ms.append(st.times()[0])
    info = st.info()
    st.free()
    del flush
    m = statistics.median(ms)
    out["mpe_bn200"] = {"workload": "MPE Bayesian network n=200, MBE i=20 (fp32 -log p)",
                        "util_entries": info["util_entries"], "util_ms": m,
                        "entries_per_s": info["util_entries"] / (m * 1e-3),
                        "gbs": info["alg_bytes"] / (m * 1e-3) / 1e9,
                        "hbm_frac": info["alg_bytes"] / (m * 1e-3) / 1e9 / peak, "config": mpe_cfg,
                        "argmin_tables": f'{info["n_argmin_tables"]} of {info["n_tasks"]} mini-buckets'}
    # repeated mini-bucket bounds under changing evidence (the bound inside a
    # search): one plan, util_condition + graph replay per bound, against
    # planning and binding a new state per bound (direct launches, the
    # cheaper choice for a single run); a large and a small bound
    inst = synth.config_instance(3, 0)
    rng = np.random.default_rng(0)
    ev_vars = sorted(int(v) for v in rng.choice(inst.n, size=16, replace=False))
    draws = [{int(v): int(rng.integers(-1, int(inst.dom[v]))) for v in rng.choice(ev_vars, size=3, replace=False)}
             for _ in range(3 + 10 * steps)]
    for z in (20, 10):
        st = gb.UtilState(inst, "mbe", z, ibound_mode="sep", use_graph=True, evidence_vars=ev_vars)
        st.bind()
        walls = []
        for k, ev in enumerate(draws):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st.condition(ev)
            st.run()
            st.value()
            t1 = time.perf_counter()
            if k >= 3:
                walls.append(t1 - t0)
        st.free()
        fresh = []
        for k, ev in enumerate(draws[: 3 + steps]):
            aug = synth.with_evidence(inst, {v: a for v, a in ev.items() if a >= 0})
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st2 = gb.UtilState(aug, "mbe", z, ibound_mode="sep")
            st2.bind()
            st2.run()
            st2.value()
            st2.free()
            t1 = time.perf_counter()
            if k >= 3:
                fresh.append(t1 - t0)
        out[f"conditioned_mbe_bn200_i{z}"] = {
            "workload": f"MBE i={z} bound of the n=200 Bayesian network under changing evidence "
                        "(16 evidence variables, 3 re-clamped per bound)",
            "bounds_per_s": 1.0 / statistics.median(walls), "ms_per_bound": 1e3 * statistics.median(walls),
            "replan_ms_per_bound": 1e3 * statistics.median(fresh),
            "speedup_vs_replan": statistics.median(fresh) / statistics.median(walls)}
    # sum-product (-log Z) on the 12x12 grid shape: a pairwise MRF, d = 4
    inst = synth.grid_mrf(12, 12, 4, seed=0, unary=False)
    st = gb.UtilState(inst, "sum", order="best", use_graph=True, autotune_cache=TUNE_CACHE)
    st.bind()
    st.autotune()
    sum_cfg = st.launch_config()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    ms = []
    for k in range(3 + steps):
        flush.fill_(k & 0xFF)
        st.run()
        st.sync()
        if k >= 3:
            ms.append(st.times()[0])
    logz = st.value().bound
    info = st.info()
    st.free()
    del flush
    m = statistics.median(ms)
    gbs = info["alg_bytes"] / (m * 1e-3) / 1e9
    out["logz_mrf12x12"] = {"workload": "sum-product -log Z, 12x12 grid MRF, d=4, 264 pairwise tables (fp32)",
                            "util_entries": info["util_entries"], "util_ms": m,
                            "entries_per_s": info["util_entries"] / (m * 1e-3), "gbs": gbs,
                            "hbm_frac": gbs / peak, "config": sum_cfg, "neg_log_z": logz}
    out["shapes"] = shape_lines(torch, gb, synth, steps)
    out["serving"] = serve_bench(torch, gb, synth, int(os.environ.get("GPUBE_SERVE_REQUESTS", "2000")))
    return out


def time_util(torch, st, steps, flush=None):
    """Median UTIL ms of a bound state over `steps` runs after 3 warm-up runs
    (L2 flushed before each run when a flush buffer is given)."""
    ms = []
    for k in range(3 + steps):
        if flush is not None:
            flush.fill_(k & 0xFF)
        st.run()
        st.sync()
        if k >= 3:
            ms.append(st.times()[0])
    return statistics.median(ms)


def shape_lines(torch, gb, synth, steps):
    """The other workload shapes, each autotuned: the 4x5 grid (exact BE,
    min-fill), exact BE on the 60-variable prefix of the Bayesian network
    (fp32), and the random-network, scale-free and grid generators of the
    paper's experiments (Section 8.1 shapes, exact BE in the best order)."""
    peak, _ = _peaks()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    cases = [("grid4x5_d4", synth.config_instance(0, 0), "minfill"),
             ("bn200_prefix60_be", synth.bn_prefix(synth.config_instance(3, 0), 60), "minfill")]
    for n, d, p1 in ((14, 8, 0.5), (12, 16, 0.3), (10, 32, 0.4), (8, 100, 0.4)):
        cases.append((f"random_n{n}_d{d}", synth.random_network_wcsp(n, d, p1, seed=1), "best"))
    for n, d in ((150, 4), (300, 2)):
        cases.append((f"scalefree_n{n}_d{d}", synth.scale_free_wcsp(n, d, seed=1), "best"))
    for r, c, d in ((20, 20, 2), (14, 14, 3), (9, 9, 6), (8, 8, 8), (6, 6, 16)):
        cases.append((f"grid{r}x{c}_d{d}", synth.grid_wcsp(r, c, d, seed=1, unary=False), "best"))
    out = {}
    for name, inst, order in cases:
        st = gb.UtilState(inst, "be", order=order, use_graph=True, autotune_cache=TUNE_CACHE)
        st.bind()
        st.autotune()
        m = time_util(torch, st, steps, flush)
        info = st.info()
        cfg = st.launch_config()
        st.free()
        out[name] = {"n": inst.n, "width": info["induced_width"], "levels": info["n_levels"],
                     "util_entries": info["util_entries"], "util_ms": m,
                     "entries_per_s": info["util_entries"] / (m * 1e-3),
                     "hbm_frac": info["alg_bytes"] / (m * 1e-3) / 1e9 / peak,
                     "mode": cfg["batched"], "lo_target": cfg["lo_target"]}
    del flush
    return out


def serve_bench(torch, gb, synth, n_req):
    """Poisson stream of DCOPs through the continuous-batching server."""
    insts = [synth.dcop_random(1000 + i) for i in range(n_req)]
    loaded = [gb.WCSP(x) for x in insts]
    budget = 8 << 30

    def run(arrivals):
        srv = gb.Server(budget, max_slots=64)
        ids = {}
        t0 = time.perf_counter()
        nxt = 0
        lag = {}
        while True:
            now = time.perf_counter() - t0
            while nxt < n_req and arrivals[nxt] <= now:
                rid = srv.submit(loaded[nxt], "dpop", parent=insts[nxt].parent)
                ids[nxt] = rid
                lag[nxt] = (time.perf_counter() - t0) - arrivals[nxt]
                nxt += 1
            left = srv.step()
            if nxt >= n_req and left == 0:
                break
        wall = time.perf_counter() - t0
        lat = []
        ent = 0
        alg = 0
        for i in range(n_req):
            ts, ta, td = srv.times(ids[i])
            lat.append(td - ts + lag[i])
            r = srv.result(ids[i])
            ent += r.util_entries
            alg += r.alg_bytes
        st = srv.stats()
        srv.close()
        st["alg_bytes"] = alg
        return wall, lat, ent, st

    # saturated: everything arrives at once
    wall, lat, ent, st = run(np.zeros(n_req))
    sat = n_req / wall
    rate = 0.8 * sat
    arrivals, _ = synth.dcop_stream(n_req, 7, rate)
    wall2, lat2, ent2, st2 = run(arrivals)
    return {"workload": f"{n_req} random DCOPs (20-200 agents, d 5-10, sep <= 8), DPOP UTIL+VALUE",
            "alg_bytes": st2["alg_bytes"], "saturated_instances_per_s": sat, "poisson_rate": rate,
            "instances_per_s": n_req / wall2, "p50_ms": 1e3 * float(np.percentile(lat2, 50)),
            "p99_ms": 1e3 * float(np.percentile(lat2, 99)), "entries_per_s": ent2 / wall2,
            "merged_launches": st2["launches"], "max_inflight": st2["max_inflight"]}


def serve_case(args):
    """The DCOP serving workload alone (GPUBE_SERVE_REQUESTS requests, default
    300, saturated and then as a Poisson stream at 0.8 x that rate), for
    launch lists of the merged level launches; prints the serving line."""
    import torch
    import synth
    import paper_1608_05288_gb300 as gb
    from paper_1608_05288_gb300 import _build
    _build.build()
    out = serve_bench(torch, gb, synth, int(os.environ.get("GPUBE_SERVE_REQUESTS", "300")))
    print(json.dumps({"case": "serve", **out}), flush=True)
    return 0


def mpe_bucket_case(args):
    """One mini-bucket of the MPE bound (Bayesian network n=200, MBE i=20) on
    its own through util_bucket: the same separator and input scopes as task
    --task of the plan, fp32 tables of random -log p values, the plan's
    default decomposition.  Times --steps launches (median) for kernel
    profiles of that bucket shape."""
    import torch
    import synth
    import paper_1608_05288_gb300 as gb
    from paper_1608_05288_gb300 import _build
    _build.build()
    inst = synth.config_instance(3, 0)
    st = gb.UtilState(inst, "mbe", 20, ibound_mode="sep")
    tasks = st.tasks()
    T = tasks[args.task]
    sep = [int(v) for v in T["sep"]]
    d = int(inst.dom[T["var"]])
    nf = inst.n_funcs
    g = torch.Generator(device="cuda").manual_seed(args.task)
    tabs, positions = [], []
    alg = 5 * int(T["rows"])
    for fid in (int(x) for x in T["inputs"]):
        scope = [int(v) for v in (inst.scopes[fid] if fid < nf else tasks[fid - nf]["sep"])]
        pos = sorted(sep.index(v) for v in scope if v != T["var"])
        size = int(np.prod([int(inst.dom[sep[p]]) for p in pos])) * d if pos else d
        tabs.append(torch.rand(size, generator=g, device="cuda") * 5.0)
        positions.append(pos)
        alg += 4 * size
    sep_dom = [int(inst.dom[v]) for v in sep]
    out = torch.empty(int(T["rows"]), dtype=torch.float32, device="cuda")
    arg = torch.empty(int(T["rows"]), dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        gb.util_bucket(sep_dom, d, tabs, positions, out, arg, "real")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for k in range(args.steps):
        ev[k][0].record()
        gb.util_bucket(sep_dom, d, tabs, positions, out, arg, "real")
        ev[k][1].record()
    torch.cuda.synchronize()
    ms = statistics.median(a.elapsed_time(b) for a, b in ev)
    peak, kind = _peaks()
    print(json.dumps({"case": "mpe_bucket", "task": args.task, "d": d, "rows": int(T["rows"]),
                      "inputs": [len(t) for t in tabs], "ms": ms, "alg_bytes": alg,
                      "gbs": alg / ms / 1e6, "frac": alg / ms / 1e6 / peak}), flush=True)
    return 0


def bucket_case(args):
    """The grid's largest bucket alone through util_bucket: separator of 12
    variables (d = 4), inputs = the previous bucket function (the 12 lowest
    joint digits), the edge to the next row (top digit, x) and the edge to the
    right neighbour (second-lowest digit, x); 4^13 joint entries.  Used for
    kernel profiles."""
    import torch
    import paper_1608_05288_gb300 as gb
    from paper_1608_05288_gb300 import _build
    _build.build()
    g = torch.Generator(device="cuda").manual_seed(0)
    m, d = 12, 4
    msg = torch.randint(0, 12000, (4 ** 12,), dtype=torch.int32, device="cuda", generator=g)
    f1 = torch.randint(0, 1000, (16,), dtype=torch.int32, device="cuda", generator=g)
    f2 = torch.randint(0, 1000, (16,), dtype=torch.int32, device="cuda", generator=g)
    out = torch.empty(4 ** 12, dtype=torch.int32, device="cuda")
    arg = torch.empty(4 ** 12, dtype=torch.uint8, device="cuda")
    pos = [list(range(1, 12)), [0], [11]]
    tabs = [msg, f1, f2]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for _ in range(args.warmup):
        gb.util_bucket([d] * m, d, tabs, pos, out, arg)
    torch.cuda.synchronize()
    for k in range(args.steps):
        ev[k][0].record()
        gb.util_bucket([d] * m, d, tabs, pos, out, arg)
        ev[k][1].record()
    torch.cuda.synchronize()
    ms = statistics.median(a.elapsed_time(b) for a, b in ev)
    alg = 4 * (4 ** 12 + 32) + 5 * 4 ** 12
    peak, kind = _peaks()
    print(json.dumps({"case": "bucket13", "ms": ms, "alg_bytes": alg, "gbs": alg / ms / 1e6,
                      "frac": alg / ms / 1e6 / peak, "peak_kind": kind}), flush=True)
    return 0


def sweep_case(args):
    """Throughput sweep over the paper's random-network, scale-free and grid
    workload shapes (Section 8.1 generators, exact BE in the best order,
    graph replay, autotuned launch shape); one JSON line per instance.
    Instances whose largest bucket exceeds 2^30 joint entries are skipped."""
    import torch
    import synth
    import paper_1608_05288_gb300 as gb
    from paper_1608_05288_gb300 import _build
    _build.build()
    os.makedirs(os.path.dirname(TUNE_CACHE), exist_ok=True)
    peak, kind = _peaks()
    cases = []
    for n, d, p1 in ((14, 8, 0.5), (12, 16, 0.3), (10, 32, 0.4), (8, 100, 0.4)):
        cases.append(synth.random_network_wcsp(n, d, p1, seed=1))
    for n, d in ((150, 4), (300, 2)):
        cases.append(synth.scale_free_wcsp(n, d, seed=1))
    for r, c, d in ((20, 20, 2), (14, 14, 3), (9, 9, 6), (8, 8, 8), (6, 6, 16)):
        cases.append(synth.grid_wcsp(r, c, d, seed=1, unary=False))
    for inst in cases:
        try:
            st = gb.UtilState(inst, "be", order="best", use_graph=True, autotune_cache=TUNE_CACHE)
        except gb.GpubeError:
            print(json.dumps({"case": inst.name, "skipped": "a bucket table over 2^31 entries"}), flush=True)
            continue
        info = st.info()
        big = max(t["rows"] * int(inst.dom[t["var"]]) for t in st.tasks())
        if big > (1 << 30):
            print(json.dumps({"case": inst.name, "skipped": f"largest bucket {big} joint entries"}), flush=True)
            st.free()
            continue
        st.bind()
        st.autotune()
        ms = []
        for k in range(args.warmup + args.steps):
            st.run()
            st.sync()
            if k >= args.warmup:
                ms.append(st.times()[0])
        m = statistics.median(ms)
        print(json.dumps({"case": inst.name, "n": inst.n, "d": int(max(inst.dom)), "width": info["induced_width"],
                          "buckets": info["n_tasks"], "levels": info["n_levels"],
                          "util_entries": info["util_entries"], "util_ms": m,
                          "entries_per_s": info["util_entries"] / (m * 1e-3),
                          "hbm_frac": info["alg_bytes"] / (m * 1e-3) / 1e9 / peak}), flush=True)
        st.free()
    return 0


def instance_case(args, which):
    """One instance for kernel profiles, no autotuning (launch shape from
    --threads / --rows): "wide100" = BE on a random network n=8, d=100
    (warp-per-row path, its first level holds 98% of the work); "er_mbe" =
    the Erdos-Renyi MBE (log2 bound 16), level-batched; "mpe_tasks" = the MPE
    bound of the n=200 Bayesian network (MBE i=20, fp32), one launch per
    mini-bucket in task order, no graph (a launch list then times each
    mini-bucket).  Prints the UTIL ms."""
    import torch
    import synth
    import paper_1608_05288_gb300 as gb
    from paper_1608_05288_gb300 import _build
    _build.build()
    kw = dict(use_graph=True)
    if args.threads:
        kw["block_threads"] = args.threads
    if args.rows:
        kw["rows_per_item"] = args.rows
    if which == "wide100":
        st = gb.UtilState(synth.random_network_wcsp(8, 100, 0.4, seed=1), "be", order="best", **kw)
    elif which == "mpe_tasks":
        kw.update(use_graph=False, batched=False)
        st = gb.UtilState(synth.config_instance(3, 0), "mbe", 20, ibound_mode="sep", **kw)
    else:
        st = gb.UtilState(synth.config_instance(2, 0), "mbe", 16, ibound_mode="log2", **kw)
    st.bind()
    info = st.info()
    ms = []
    for k in range(args.warmup + args.steps):
        st.run()
        st.sync()
        if k >= args.warmup:
            ms.append(st.times()[0])
    print(json.dumps({"case": which, "util_ms": statistics.median(ms), "util_entries": info["util_entries"],
                      "launches": info["n_tasks"] if which == "mpe_tasks" else info["n_levels"],
                      "alg_bytes": info["alg_bytes"]}), flush=True)
    return 0


def grid_rows_case(args, rows=3, sum_product=False):
    """BE on the first `rows` rows of the headline grid (same tables, natural
    order, every bucket of row 1 is a full 4^13-entry bucket), a few GB on
    the device: the case for kernel profiles of full-size launches.  With
    sum_product: -log Z of the same rows of the 12x12 MRF."""
    import torch
    import synth
    import paper_1608_05288_gb300 as gb
    from paper_1608_05288_gb300 import _build
    _build.build()
    inst = synth.grid_mrf(12, 12, 4, seed=0, unary=False) if sum_product else synth.config_instance(1, 0)
    nv = 12 * rows
    keep = [j for j, s in enumerate(inst.scopes) if int(np.max(s)) < nv]
    sub = synth.Instance("grid12x12_rows", inst.dom[:nv].copy(), [inst.scopes[j] for j in keep],
                         [inst.tables[j] for j in keep], inst.cost_type, inst.top_k)
    kw = {}
    if args.threads:
        kw["block_threads"] = args.threads
    if args.rows:
        kw["rows_per_item"] = args.rows
    os.makedirs(os.path.dirname(TUNE_CACHE), exist_ok=True)
    st = gb.UtilState(sub, "sum" if sum_product else "be", order="natural", use_graph=True,
                      autotune_cache=TUNE_CACHE, **kw)
    st.bind()
    if not kw:
        st.autotune()
    info = st.info()
    ms = []
    for k in range(args.warmup + args.steps):
        st.run()
        st.sync()
        if k >= args.warmup:
            ms.append(st.times()[0])
    m = statistics.median(ms)
    peak, kind = _peaks()
    print(json.dumps({"case": f"{'mrf' if sum_product else 'grid'}12x{rows}", "util_ms": m, "alg_bytes": info["alg_bytes"],
                      "gbs": info["alg_bytes"] / m / 1e6, "frac": info["alg_bytes"] / m / 1e6 / peak,
                      "launches": info["n_levels"], "arena_gb": info["arena_bytes"] / 1e9}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-secondary", action="store_true")
    ap.add_argument("--case", default="",
                    choices=["", "bucket13", "grid3", "grid12", "mrf3", "sweep", "wide100", "er_mbe", "mpe_tasks",
                             "serve", "mpe_bucket"])
    ap.add_argument("--task", type=int, default=165)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--rows", type=int, default=0)
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.case == "bucket13":
        return bucket_case(args)
    if args.case == "serve":
        return serve_case(args)
    if args.case == "mpe_bucket":
        return mpe_bucket_case(args)
    if args.case == "grid3":
        return grid_rows_case(args, 3)
    if args.case == "grid12":
        return grid_rows_case(args, 12)
    if args.case == "mrf3":
        return grid_rows_case(args, 3, sum_product=True)
    if args.case == "sweep":
        return sweep_case(args)
    if args.case in ("wide100", "er_mbe", "mpe_tasks"):
        return instance_case(args, args.case)

    import torch
    import torch.distributed as dist

    import synth
    import paper_1608_05288_gb300 as gb
    from paper_1608_05288_gb300 import _build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if rank == 0 or world == 1:
        _build.build()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
        dist.barrier()
        _build.build()
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")

    inst = synth.config_instance(1, seed=rank)  # one replica per rank
    st = gb.UtilState(inst, "be", order="best", use_graph=True, device=local, autotune_cache=TUNE_CACHE)
    st.bind(device=local)
    threads, rows = st.autotune()  # launch configuration measured on this instance (cached)
    tuned = st.launch_config()
    info = st.info()
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    for _ in range(args.warmup):
        st.run()
        st.value_launch()
    st.sync()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = Clocks(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)  # L2 flush between steps (outside the step's events)
        ev[k][0].record(stream)
        st.run()
        ev[k][1].record(stream)
        st.value_launch()
        ev[k][2].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    st.sync()
    util_ms = [a.elapsed_time(b) for a, b, _ in ev]
    step_ms = [a.elapsed_time(c) for a, _, c in ev]
    tot_s = max_over_ranks(sum(step_ms) * 1e-3, dev)
    value = whole_job_rate(info["util_entries"], world, args.steps, tot_s)
    res = st.value()
    # UTIL launches of one step (one per level, or one over all levels) + the VALUE kernel
    n_launch_step = (1 if tuned["batched"] == 2 else info["n_levels"]) + 1

    # roofline of the UTIL kernel: algorithmic bytes / its device time
    peak, peak_kind = _peaks()
    util_s = sum(util_ms) * 1e-3 / args.steps
    achieved = info["alg_bytes"] / util_s / 1e9
    # (the capture behind the traffic figure is of per-level launches)
    traffic = _traffic_per_launch(info["alg_bytes"] / info["n_levels"]) if tuned["batched"] == 1 else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
                "alg_bytes_per_launch": info["alg_bytes"] / (n_launch_step - 1),
                "alg_bytes_per_step": info["alg_bytes"], "launches_per_step": n_launch_step - 1}
    st.free()
    del flush

    # end to end through the C ABI from host buffers: load, plan, upload, UTIL,
    # VALUE, result copy, in every step
    arena = torch.empty(info["arena_bytes"] + 4096, dtype=torch.uint8, device=dev)
    e2e_s, plan_ms = [], []
    pk = gb.Packed(inst)  # the problem as wcsp_desc's flat host arrays
    for k in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        w = gb.WCSP(pk)
        r = gb.be_solve(w, order="best", arena=arena.data_ptr(), arena_bytes=arena.numel(),
                        stream=stream.cuda_stream, device=local, **tuned)
        t1 = time.perf_counter()
        if k >= args.warmup:
            e2e_s.append(t1 - t0)
            plan_ms.append(r.plan_ms)
        assert r.bound == res.bound
    e2e_tot = max_over_ranks(sum(e2e_s), dev)
    h2d = sum(len(t) for t in inst.tables) * 4
    e2e = {"value": whole_job_rate(info["util_entries"], world, args.steps, e2e_tot), "unit": UNIT,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 24 + 4 * inst.n,
           "ms_per_step": 1e3 * e2e_tot / args.steps,
           "host_plan_ms": statistics.median(plan_ms),  # ordering, buckets, levels (inside the step)
           "input": "wcsp_desc flat arrays in host memory; wcsp_load, plan, upload, UTIL, VALUE, result "
                    "copy every step"}
    del arena

    extra = {}
    cpu = None
    if rank == 0 and world == 1:
        if not args.no_secondary:
            extra = secondary(torch, gb, synth, max(3, min(args.steps, 10)))
        e, t, th = cpu_oracle_step()
        cpu = {"value": e / t, "unit": UNIT, "cores": th, "kind": "oracle",
               "sample": f"oracle BE on rows 0-{CPU_ROWS - 1} of the 12x12 grid ({12 * CPU_ROWS} variables, "
                         f"natural order, {e} joint entries, {t:.1f} s)"}
        # the sequential oracle (one host thread), the form of the paper's
        # CPU comparison, on a smaller piece of the same grid
        e1, t1, _ = cpu_oracle_step(threads=1, rows=CPU_ROWS_1T)
        cpu["single_thread"] = {"value": e1 / t1, "unit": UNIT, "cores": 1,
                                "sample": f"oracle BE on rows 0-{CPU_ROWS_1T - 1} of the 12x12 grid "
                                          f"({12 * CPU_ROWS_1T} variables, {e1} joint entries, {t1:.1f} s)"}
        cpu["sample"] += f"; on one host thread: {e1 / t1:.3g} entries/s (rows 0-{CPU_ROWS_1T - 1})"

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "buckets": info["n_tasks"], "levels": info["n_levels"],
                           "block_threads": threads, "rows_per_item": rows, "launch": tuned,
                           "util_entries_per_step": info["util_entries"],
                           "l2": "flushed between steps (512 MB write)",
                           "parallelism": f"replicas x{world}", "bound": res.bound},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": n_launch_step * args.steps, "clocks": clk,
                "util_ms_per_step": 1e3 * util_s, "secondary": extra}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
