#!/usr/bin/env python3
"""Throughput of the fused GTMP planner on one B300 (or N, one process each).

Workload (default): 7-DoF DH arm, 20 sphere + 10 box obstacles in a 1.5 m
cube, M = 1024 samples per layer, L = 8 layers, H = 32 waypoints per edge,
float32.  One step = one complete plan through the C ABI: Philox layer
sampling, vertex labels, the L+1 fused edge + min-plus transitions and path
extraction, i.e. H * (2M + (L-1) M^2) = 234,946,560 nominal waypoint checks.
Every step plans a different sample set (seed = step); under torchrun every
rank plans its own seeds (independent problems, weak scaling, no collective
on the data path).

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle
instead, on a bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "edge-waypoint checks/sec and solves/sec (7-DoF, M=1024, L=8), surrogate/batched vs plain"


def flops_per_waypoint(dof, spl, n_s, n_b, arm=True):
    """FP32 arithmetic of one interior waypoint check as the kernel performs it.

    add/sub/mul/div/sqrt count 1, fma counts 2; compares, min/max and the
    sincosf calls count 0.  Waypoint: dof fma + 1 div.  FK per link: angle add
    (1), new x and pre-twist y axes (2 x (3 mul + 3 fma) = 18), origin (6 fma =
    12), twisted y and z axes (18), and spl sphere centres (9 fma = 18 each).
    Per robot sphere: sphere obstacle 3 sub + 1 mul + 2 fma = 8, box 3 sub +
    3 sub + 1 mul + 2 fma = 11.
    """
    interp = 2 * dof + 1
    if arm:
        fk = dof * (1 + 18 + 12 + 18 + 18 * spl)
        spheres = dof * spl
    else:
        fk, spheres = 0, 1
    return interp + fk + spheres * (8 * n_s + 11 * n_b)


def rank_seed_base(rank: int) -> int:
    """First Philox seed of a rank: ranks plan disjoint seed ranges (independent problems)."""
    return 1 + rank * 1_000_003


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Max of a host float over all ranks (identity for one rank)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def oracle_rows(sc, wl, budget_s, seed=0, max_rows=None):
    """Run the oracle's edge realisation on whole rows of the layer-to-layer
    transitions (row i of transition 1, 2, ..., L-1, then row i+1, ...) until
    budget_s has passed; return (edges, seconds, rows)."""
    import oracle
    M, L, H = wl["M"], wl["L"], wl["H"]
    Q = oracle.sample_uniform(seed, 0, L, M, sc.robot.q_lo, sc.robot.q_hi)
    verts = oracle.layer_vertices(Q, sc.q_start, sc.q_goal)
    mids = list(range(1, L)) or [0]
    t0 = time.perf_counter()
    rows = 0
    while True:
        layer = mids[rows % len(mids)]
        i = (rows // len(mids)) % len(verts[layer])
        oracle.edge_block(sc, verts[layer][i:i + 1], verts[layer + 1], H)
        rows += 1
        el = time.perf_counter() - t0
        if el >= budget_s or (max_rows and rows >= max_rows):
            return rows * len(verts[layer + 1]), el, rows


L2_POLICY = "flushed between GPU steps"


def workload_config(args, wl, world, n_s, n_b):
    """The workload description both arms print (the reference arm runs the same workload on host cores)."""
    M, L, H = wl["M"], wl["L"], wl["H"]
    return {"workload": args.workload, "M": M, "L": L, "H": H, "dof": wl.get("dof", 2), "obstacles": [n_s, n_b],
            "eval_mode": "early_exit", "parallelism": f"replicas x{world}", "l2": L2_POLICY,
            "checks_per_solve": H * (2 * M + (L - 1) * M * M)}


def cpu_baseline(sc, wl, budget_s, seed0):
    """The oracle on whole rows of the layer-to-layer transitions: all host threads for budget_s, then one
    thread for a third of it; checks/s extrapolated per nominal check."""
    import oracle
    M, H = wl["M"], wl["H"]
    n_all = oracle.set_threads(0)
    edges, secs, rows = oracle_rows(sc, wl, budget_s, seed=seed0)
    oracle.set_threads(1)
    e1, s1, r1 = oracle_rows(sc, wl, budget_s / 3, seed=seed0)
    oracle.set_threads(n_all)
    return {"value": edges * H / secs, "unit": "checks/s", "cores": n_all, "kind": "oracle",
            "value_1thread": e1 * H / s1,
            "sample": f"{rows} rows x {M} edges of the layer-to-layer transitions (H={H}) in {secs:.1f} s on "
                      f"{n_all} threads, {r1} rows in {s1:.1f} s on 1 thread; extrapolated per nominal check"}


def oracle_free_fn(sc):
    import oracle
    return lambda q: oracle.config_free(sc, q)


def run_reference(args, wl):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2608_25830_b300 import scenes
    if wl["kind"] == "point2d":
        sc = scenes.point2d_scene(wl["seed"], wl["n_obs"])
    else:
        base = scenes.arm_scene(wl["seed"], wl["dof"], wl["n_obs"])
        sc = scenes.pick_endpoints(base, oracle_free_fn(base))
    import oracle
    per_step = args.ref_budget
    for _ in range(args.warmup):
        oracle_rows(sc, wl, per_step / 4, max_rows=1)
    edges = 0
    secs = 0.0
    rows = 0
    seed0 = rank_seed_base(0)                    # the GPU arm's seeds: step s plans seed seed0 + s
    for s in range(args.steps):
        e, t, r = oracle_rows(sc, wl, per_step, seed=seed0 + s)
        edges += e
        secs += t
        rows += r
    checks = edges * wl["H"]
    nominal_edges = 2 * wl["M"] + (wl["L"] - 1) * wl["M"] ** 2
    cores = oracle.set_threads(0)
    value = checks / secs
    sample = (f"{rows} rows x {wl['M']} edges of the layer-to-layer transitions (H={wl['H']}), "
              f"{args.steps} steps of ~{per_step:.0f} s on {cores} threads, extrapolated per nominal check")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "checks/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "solves_per_s": edges / secs / nominal_edges,
        "config": workload_config(args, wl, world, sc.spheres.shape[0], sc.boxes.shape[0]),
        "cpu_baseline": {"value": value, "unit": "checks/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "checks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9 or not f[1].isdigit():
                    continue
                sm.append(int(f[1]))
                mx.append(int(f[2]))
                for n, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        except OSError:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# DRAM bytes (read + write) of one full-evaluation launch of the fused kernel on a 1024 x 1024
# transition of this workload, from the ncu capture summarised in
# profiles/fused_transition_arm7_m1024_l8_h32.md (set back to None whenever the kernel changes); the
# algorithmic bytes per launch are reported beside it
FULL_MODE_DRAM_BYTES_PER_LAUNCH = 189696


def measured_peaks():
    """HBM copy bandwidth and bf16 GEMM rate measured on this GPU model (file beside this script), else the
    fallback figures of an earlier B300 measurement."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        d["source"] = "measured"
        return d
    except (OSError, ValueError):
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "source": "fallback"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args, wl):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2608_25830_b300 import binding, scenes

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    M, L, H = wl["M"], wl["L"], wl["H"]
    # scene: endpoints chosen by the GPU's own exact checker
    if wl["kind"] == "point2d":
        sc = scenes.point2d_scene(wl["seed"], wl["n_obs"])
    else:
        base = scenes.arm_scene(wl["seed"], wl["dof"], wl["n_obs"])
        probe = binding.Planner(base.robot, 8, 1, 2, max_obstacles=64)
        binding.gtmp_set_obstacles(probe.ctx, base.spheres, base.boxes)

        def free_fn(q):
            return (probe.label_configs(torch.from_numpy(np.ascontiguousarray(q)).cuda()).cpu().numpy() == 0)

        sc = scenes.pick_endpoints(base, free_fn)
        probe.close()
    dof = sc.robot.dof
    n_s, n_b = sc.spheres.shape[0], sc.boxes.shape[0]
    nominal_edges = 2 * M + (L - 1) * M * M
    nominal_checks = H * nominal_edges

    p = binding.Planner(sc.robot, M, L, H, max_obstacles=64, eval_mode=binding.EVAL_EARLY_EXIT)
    p.set_scene(sc)
    path = torch.empty(L, dtype=torch.int32, device="cuda")
    cost = torch.empty(1, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > 126 MB L2

    def step(seed):
        binding.gtmp_sample_layers(p.ctx, seed, M)
        binding.gtmp_solve(p.ctx, path, cost)

    seed0 = rank_seed_base(rank)
    for s in range(args.warmup):
        step(seed0 + 10_000 + s)
    p.synchronize()

    # --- device-resident timed region: K plans, L2 flushed between them
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    costs = []
    binding.gtmp_profile_read(p.ctx)                 # reset counters
    binding.gtmp_profile_enable(p.ctx, True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        gpu_id = str(local)
    with ClockSampler(gpu_id) as clk:
        for s in range(args.steps):
            flush.zero_()
            evs[s][0].record(stream)
            step(seed0 + s)
            evs[s][1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    prof = binding.gtmp_profile_read(p.ctx)
    binding.gtmp_profile_enable(p.ctx, False)
    p.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_s = max_over_ranks(sum(step_ms) / 1e3, world, "cuda")
    solves = args.steps * world
    value = nominal_checks * solves / total_s
    clocks = clk.summary()
    last_cost = float(cost.cpu()[0])

    # --- end to end through the public API, host buffers, copies inside the region
    host_path = torch.empty(L, dtype=torch.int32, pin_memory=True)
    host_cost = torch.empty(1, dtype=torch.float32, pin_memory=True)
    h2d = (sc.spheres.size + sc.boxes.size + 2 * dof) * 4 + 8
    d2h = L * 4 + 4

    def e2e_step(seed):
        binding.gtmp_set_obstacles(p.ctx, sc.spheres, sc.boxes)
        binding.gtmp_set_endpoints(p.ctx, sc.q_start, sc.q_goal)
        step(seed)
        host_path.copy_(path, non_blocking=True)
        host_cost.copy_(cost, non_blocking=True)
        torch.cuda.current_stream().synchronize()

    e2e_step(seed0 + 20_000)
    e2e_s = 0.0
    for s in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step(seed0 + s)
        e2e_s += time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, world, "cuda")
    e2e_value = nominal_checks * solves / e2e_s

    # --- the same plans in lazy mode (exact: identical values and paths, most edges never realised)
    plz = binding.Planner(sc.robot, M, L, H, max_obstacles=64, eval_mode=binding.EVAL_LAZY)
    plz.set_scene(sc)
    lz_path = torch.empty(L, dtype=torch.int32, device="cuda")
    lz_cost = torch.empty(1, dtype=torch.float32, device="cuda")
    ref_path = torch.empty(L, dtype=torch.int32, device="cuda")
    ref_cost = torch.empty(1, dtype=torch.float32, device="cuda")
    for s in range(args.warmup):
        binding.gtmp_sample_layers(plz.ctx, seed0 + 10_000 + s, M)
        binding.gtmp_solve(plz.ctx, lz_path, lz_cost)
    plz.synchronize()
    lz_ms = []
    lz_same = True
    for s in range(args.steps):
        flush.zero_()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        binding.gtmp_sample_layers(plz.ctx, seed0 + s, M)
        binding.gtmp_solve(plz.ctx, lz_path, lz_cost)
        a1.record(stream)
        binding.gtmp_sample_layers(p.ctx, seed0 + s, M)
        binding.gtmp_solve(p.ctx, ref_path, ref_cost)
        torch.cuda.synchronize()
        lz_ms.append(a0.elapsed_time(a1))
        lz_same = lz_same and bool(torch.equal(lz_path, ref_path)) and (
            float(lz_cost.cpu()[0]) == float(ref_cost.cpu()[0]) or math.isinf(float(ref_cost.cpu()[0])))
    plz.close()
    lazy_s = max_over_ranks(sum(lz_ms) / 1e3, world, "cuda")

    # --- path-level lazy evaluation: optimistic sweeps, the winning chain checked exactly, repeated
    ppl = binding.Planner(sc.robot, M, L, H, max_obstacles=64)
    ppl.set_scene(sc)
    for s in range(args.warmup):
        binding.gtmp_sample_layers(ppl.ctx, seed0 + 10_000 + s, M)
        binding.gtmp_solve_lazy_path(ppl.ctx, lz_path, lz_cost)
    ppl.synchronize()
    lp_ms, lp_iters, lp_same = [], [], True
    for s in range(args.steps):
        flush.zero_()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        binding.gtmp_sample_layers(ppl.ctx, seed0 + s, M)
        st_lp = binding.gtmp_solve_lazy_path(ppl.ctx, lz_path, lz_cost)
        a1.record(stream)
        binding.gtmp_sample_layers(p.ctx, seed0 + s, M)
        binding.gtmp_solve(p.ctx, ref_path, ref_cost)
        torch.cuda.synchronize()
        lp_ms.append(a0.elapsed_time(a1))
        lp_iters.append(st_lp["iterations"])
        lp_same = lp_same and (float(lz_cost.cpu()[0]) == float(ref_cost.cpu()[0]) or
                               math.isinf(float(ref_cost.cpu()[0])))
    ppl.close()
    lazy_path_s = max_over_ranks(sum(lp_ms) / 1e3, world, "cuda")

    # --- the same seeds with layer samples drawn on C_free (rejection, Sec. III's pi_m): quality and speed
    pfree = binding.Planner(sc.robot, M, L, H, max_obstacles=64)
    pfree.set_scene(sc)
    binding.gtmp_set_sampler(pfree.ctx, binding.SAMPLER_FREE, 64)
    for s in range(args.warmup):
        binding.gtmp_sample_layers(pfree.ctx, seed0 + 10_000 + s, M)
        binding.gtmp_solve(pfree.ctx, lz_path, lz_cost)
    pfree.synchronize()
    fr_ms, fr_costs, un_costs = [], [], []
    for s in range(args.steps):
        flush.zero_()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        binding.gtmp_sample_layers(pfree.ctx, seed0 + s, M)
        binding.gtmp_solve(pfree.ctx, lz_path, lz_cost)
        a1.record(stream)
        binding.gtmp_sample_layers(p.ctx, seed0 + s, M)
        binding.gtmp_solve(p.ctx, ref_path, ref_cost)
        torch.cuda.synchronize()
        fr_ms.append(a0.elapsed_time(a1))
        fr_costs.append(float(lz_cost.cpu()[0]))
        un_costs.append(float(ref_cost.cpu()[0]))
    pfree.close()
    fin = [(a, b) for a, b in zip(fr_costs, un_costs) if math.isfinite(a) and math.isfinite(b)]
    free_sampling = {"solves_per_s": args.steps / (sum(fr_ms) / 1e3), "ms_per_step": sum(fr_ms) / len(fr_ms),
                     "feasible": sum(math.isfinite(c) for c in fr_costs), "feasible_uniform": sum(math.isfinite(c) for c in un_costs),
                     "mean_cost_ratio_free_over_uniform": (sum(a / b for a, b in fin) / len(fin)) if fin else None,
                     "note": "same seeds; samples redrawn on C_free (first free of up to 64 attempts)"}

    # --- the same seeds with weighted-length edge costs (App. "General Costs"): speed and cost
    pw = binding.Planner(sc.robot, M, L, H, max_obstacles=64)
    pw.set_scene(sc)
    bumps = scenes.weight_bumps(sc, wl["seed"])
    pw.set_cost_weight(bumps)
    for s in range(args.warmup):
        binding.gtmp_sample_layers(pw.ctx, seed0 + 10_000 + s, M)
        binding.gtmp_solve(pw.ctx, lz_path, lz_cost)
    pw.synchronize()
    w_ms, w_costs = [], []
    for s in range(args.steps):
        flush.zero_()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        binding.gtmp_sample_layers(pw.ctx, seed0 + s, M)
        binding.gtmp_solve(pw.ctx, lz_path, lz_cost)
        a1.record(stream)
        torch.cuda.synchronize()
        w_ms.append(a0.elapsed_time(a1))
        w_costs.append(float(lz_cost.cpu()[0]))
    pw.close()
    finw = [(a, b) for a, b in zip(w_costs, un_costs) if math.isfinite(a) and math.isfinite(b)]
    weighted = {"solves_per_s": args.steps / (sum(w_ms) / 1e3), "ms_per_step": sum(w_ms) / len(w_ms),
                "bumps": int(bumps.shape[0]), "w_max": float(1.0 + bumps[:, -1].astype(np.float64).sum()),
                "mean_cost_ratio_weighted_over_length": (sum(a / b for a, b in finw) / len(finw)) if finw else None,
                "note": "same seeds as the timed plans; edge cost = trapezoid rule of the weight on the H waypoints"}

    # --- roofline of the fused kernel in full-evaluation mode (data-independent FP32 work)
    pf = binding.Planner(sc.robot, M, L, H, max_obstacles=64, eval_mode=binding.EVAL_FULL)
    pf.set_scene(sc)
    binding.gtmp_sample_layers(pf.ctx, seed0, M)
    binding.gtmp_solve(pf.ctx, path, cost)
    pf.synchronize()
    binding.gtmp_profile_read(pf.ctx)
    binding.gtmp_profile_enable(pf.ctx, True)
    full_steps = max(1, min(3, args.steps))
    for s in range(full_steps):
        flush.zero_()
        binding.gtmp_sample_layers(pf.ctx, seed0 + s, M)
        binding.gtmp_solve(pf.ctx, path, cost)
    fprof = binding.gtmp_profile_read(pf.ctx)
    pf.close()
    fpw = flops_per_waypoint(dof, sc.robot.spheres_per_link, n_s, n_b, wl["kind"] == "arm")
    n_sp, n_bp = (n_s + 1) // 2, (n_b + 1) // 2
    full_alg_bytes = 2 * M * 8 * 4 + 2 * M * 8 + (5 * n_sp + 6 * n_bp + (n_s + n_b + 1) // 2 * 2) * 16
    full_flops = fprof["fused_edges"] * (H - 2) * fpw
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak_tflops = sms * 128 * 2 * 2.032e9 / 1e12
    achieved = full_flops / (fprof["fused_ms"] / 1e3) / 1e12
    ffma_tflops = binding.gtmp_fp32_fma_peak(torch.cuda.current_stream().cuda_stream)

    # --- unfused variant: the min-plus sweep over stored cost matrices, at M = 4096 (C = 470 MB >> L2)
    unfused = None
    if wl["kind"] == "arm" and not args.no_unfused:
        Mu = 4096
        pu = binding.Planner(sc.robot, Mu, L, H, max_obstacles=64)
        pu.set_scene(sc)
        upath = torch.empty(L, dtype=torch.int32, device="cuda")
        ucost = torch.empty(1, dtype=torch.float32, device="cuda")
        binding.gtmp_sample_layers(pu.ctx, seed0, Mu)
        binding.gtmp_solve_unfused(pu.ctx, upath, ucost)
        pu.synchronize()
        binding.gtmp_profile_read(pu.ctx)
        binding.gtmp_profile_enable(pu.ctx, True)
        for s in range(2):
            flush.zero_()
            binding.gtmp_sample_layers(pu.ctx, seed0 + s, Mu)
            binding.gtmp_solve_unfused(pu.ctx, upath, ucost)
        uprof = binding.gtmp_profile_read(pu.ctx)
        pu.close()
        peaks = measured_peaks()
        hbm = peaks.get("hbm_gbs")
        gbs = uprof["minplus_bytes"] / (uprof["minplus_ms"] / 1e3) / 1e9
        unfused = {"bound": "hbm", "kernel": "minplus_kernel (unfused value iteration, M=4096, L=8)",
                   "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm if hbm else None,
                   "traffic": None, "peak_basis": f"copy bandwidth (hbm_gbs, {peaks['source']})",
                   "bytes_per_solve": uprof["minplus_bytes"] / 2, "ms_per_solve": uprof["minplus_ms"] / 2,
                   "launches_per_solve": uprof["minplus_launches"] // 2,
                   "note": "4 B per stored edge cost + 8 B per cost-to-go read and written; the cost matrices are "
                           "written last-layer first, so most of each sweep's reads come from HBM"}

    # --- the metric's comparisons: batched (512 uneven problems) and surrogate-pruned (M = 4096) against the
    # plain solver on the same problems and samples, and the anytime / AO forms; each with its own clock record
    extras = {}
    if not args.no_extras:
        from paper_2608_25830_b300 import scenes as _sc
        extras["batched"] = measure_batched(args, _sc.WORKLOADS["batched512_h32"], flush, 2, 1)
        extras["surrogate"] = measure_surrogate(args, _sc.WORKLOADS["arm7_m4096_l8_h32_n40"], flush, 3, 1)
        extras["anytime"] = measure_anytime(args, _sc.WORKLOADS["arm6_anytime_r64_m256_l6_h32"], flush, 20, 3)
        extras["ao"] = measure_ao(args, _sc.WORKLOADS["arm6_ao_m64to4096_l6_h32"], 5, 1)

    out = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline(sc, wl, args.cpu_budget, seed0)
        out = {
            "metric": METRIC, "value": value, "unit": "checks/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sum(step_ms) / len(step_ms), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded scene and samples)",
            "solves_per_s": solves / total_s,
            "config": workload_config(args, wl, world, n_s, n_b),
            "last_cost": last_cost,
            "e2e": {"value": e2e_value, "unit": "checks/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(prof["launches"]),
            "roofline": {"bound": "alu", "kernel": "fused_transition_kernel (full-evaluation mode)",
                         "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                         "traffic": FULL_MODE_DRAM_BYTES_PER_LAUNCH,
                         "traffic_note": "dram__bytes_read.sum + dram__bytes_write.sum of one 1024 x 1024 transition "
                                         "launch (ncu --set full capture of the current kernel); the staged block "
                                         "also carries the 64 KB cull grid, and the unrolled link loop's code is "
                                         "fetched too: the algorithmic bytes plus the grid plus code, each byte "
                                         "read once",
                         "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 x 2032 MHz (max clock)",
                         "ffma_measured": ffma_tflops, "frac_of_ffma_measured": achieved / ffma_tflops,
                         "ffma_note": "gtmp_fp32_fma_peak: independent FMA chains on every SM, best of 6 launches",
                         "flops_per_waypoint": fpw,
                         "algorithmic_bytes_per_launch": full_alg_bytes,
                         "algorithmic_bytes_note": "rows' and columns' samples (M x 8 floats each), the columns' "
                                                   "cost-to-go keys read and the rows' keys written (8 B each), the "
                                                   "exact-test obstacle tables; the staged block also carries the "
                                                   "early-exit cull grid (up to 64 KB), which full evaluation does "
                                                   "not use",
                         "fused_ms_per_solve": fprof["fused_ms"] / full_steps},
            "fused_ms_per_solve_early_exit": prof["fused_ms"] / args.steps,
            "roofline_unfused_minplus": unfused,
            "free_sampling": free_sampling,
            "weighted_length": weighted,
            "lazy": {"solves_per_s": solves / lazy_s, "ms_per_step": sum(lz_ms) / len(lz_ms),
                     "same_paths_and_costs_as_early_exit": lz_same,
                     "note": "exact mode GTMP_EVAL_LAZY: an edge is realised only if c(u,v)+J(v) beats its row's "
                             "best so far; value above counts the nominal checks of the early-exit mode"},
            "lazy_path": {"solves_per_s": solves / lazy_path_s, "ms_per_step": sum(lp_ms) / len(lp_ms),
                          "iterations_mean": sum(lp_iters) / len(lp_iters), "iterations_max": max(lp_iters),
                          "same_costs_as_early_exit": lp_same,
                          "note": "gtmp_solve_lazy_path: min-plus sweeps over optimistic (unchecked) edge costs, "
                                  "the winning chain checked exactly and its colliding edges left out, until a "
                                  "chain is free; iterations enqueued eight at a time with the loop state on "
                                  "the device"},
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        out.update(extras)
        print(json.dumps(out), flush=True)
    p.close()
    if world > 1:
        dist.destroy_process_group()
    return out


def gpu_endpoints(binding, scenes, base):
    """Arm scene with start and goal picked by the GPU's own exact checker (first free candidate pair)."""
    import numpy as np
    import torch
    probe = binding.Planner(base.robot, 8, 1, 2, max_obstacles=64)
    binding.gtmp_set_obstacles(probe.ctx, base.spheres, base.boxes)
    sc = scenes.pick_endpoints(base, lambda q: probe.label_configs(
        torch.from_numpy(np.ascontiguousarray(q)).cuda()).cpu().numpy() == 0)
    probe.close()
    return sc


def gpu_uuid(local):
    import torch
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        return str(local)


def _timed_passes(fn, steps, flush, stream):
    """Device time (ms) of `steps` calls of fn, L2 flushed before each; one event pair per call."""
    import torch
    ms = []
    for _ in range(steps):
        flush.zero_()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        fn()
        a1.record(stream)
        torch.cuda.synchronize()
        ms.append(a0.elapsed_time(a1))
    return ms


def measure_batched(args, wl, flush, steps, warmup, lazy=True, breakdown=False):
    """512 uneven problems (2D point robots and 7-DoF arms): one persistent launch per robot variant against the plain
    single-problem solver running the same problems one after another, early exit and lazy."""
    import numpy as np
    import torch

    from paper_2608_25830_b300 import binding, scenes

    rank, world, local = dist_env()
    H = wl["H"]
    base = scenes.batch_problems(wl["seed"] + rank, wl["n"], H=H)
    problems = []
    for bp in base:
        sc = bp.scene
        if sc.candidates is not None:
            sc = gpu_endpoints(binding, scenes, sc)
        problems.append((sc, bp.M, bp.L, bp.seed))
    stream = torch.cuda.current_stream()

    def batched_form(mode):
        b = binding.Batch(problems, H, eval_mode=mode)
        b.autotune(repeats=1)                                   # per-kind tile autotuning on the batch, untimed
        tiling = binding.gtmp_batch_get_tilings(b.handle)
        for _ in range(warmup):
            b.solve()
        b.synchronize()
        return b, tiling

    def plain_form(mode):
        planners = []
        for sc, M, L, seed in problems:
            pl = binding.Planner(sc.robot, M, L, H, max_obstacles=64, eval_mode=mode)
            pl.set_scene(sc)
            planners.append((pl, M, L, seed, torch.empty(L, dtype=torch.int32, device="cuda"),
                             torch.empty(1, dtype=torch.float32, device="cuda")))

        def run():
            for pl, M, L, seed, pa, co in planners:
                binding.gtmp_sample_layers(pl.ctx, seed, M)
                binding.gtmp_solve(pl.ctx, pa, co)
        run()
        torch.cuda.synchronize()
        return planners, run

    out = {"problems": wl["n"], "H": H}
    modes = [("early_exit", binding.EVAL_EARLY_EXIT)] + ([("lazy", binding.EVAL_LAZY)] if lazy else [])
    ref_costs = None
    with ClockSampler(gpu_uuid(local)) as clk:
        for name, mode in modes:
            b, tiling = batched_form(mode)
            b_ms = _timed_passes(b.solve, steps, flush, stream)
            b.synchronize()
            costs = b.costs.cpu().numpy()
            nominal = b.nominal_checks
            items = b.work_items
            kernels = b.kernels_per_solve
            b.close()
            planners, run = plain_form(mode)
            p_ms = _timed_passes(run, steps, flush, stream)
            plain_costs = np.array([float(co.cpu()[0]) for *_, co in planners], np.float32)
            for pl, *_ in planners:
                pl.close()
            if ref_costs is None:
                ref_costs = costs
            b_s = max_over_ranks(sum(b_ms) / 1e3, world, "cuda")
            p_s = max_over_ranks(sum(p_ms) / 1e3, world, "cuda")
            out[name] = {
                "batched_solves_per_s": wl["n"] * steps * world / b_s,
                "plain_solves_per_s": wl["n"] * steps * world / p_s,
                "batched_over_plain": p_s / b_s,
                "batched_checks_per_s": nominal * steps * world / b_s,
                "batched_ms_per_batch": sum(b_ms) / len(b_ms), "plain_ms_per_batch": sum(p_ms) / len(p_ms),
                "tiling": {"point": list(tiling[binding.ROBOT_POINT]), "arm": list(tiling[binding.ROBOT_DH_ARM])},
                "work_items": items, "checks_per_batch": nominal,
                "feasible": int(np.isfinite(costs).sum()),
                "same_costs_batched_plain": bool(np.array_equal(costs, plain_costs)),
                "same_costs_as_early_exit": bool(np.array_equal(costs, ref_costs)),
                "gpu_launches_per_batch": kernels,
            }
    out["clocks"] = clk.summary()
    out["steps"], out["warmup"] = steps, warmup
    out["l2"] = "flushed before every batch and every plain pass"
    out["note"] = ("plain = gtmp_sample_layers + gtmp_solve per problem, one after another on one stream; "
                   "batched = gtmp_batch_solve (one persistent launch per robot variant, tilings autotuned "
                   "per robot kind before timing); same problems and seeds")
    if breakdown:
        out["breakdown"] = {}
        t = out["early_exit"]["tiling"]
        tiling = {binding.ROBOT_POINT: t["point"], binding.ROBOT_DH_ARM: t["arm"]}
        for name, keep in (("arm", lambda sc: sc.robot.dof > 3), ("point2d", lambda sc: sc.robot.dof <= 3)):
            sub = [p for p in problems if keep(p[0])]
            sb = binding.Batch(sub, H)
            binding.gtmp_batch_set_tilings(sb.handle, tiling)
            sb.solve()
            torch.cuda.synchronize()
            t_b = _timed_passes(sb.solve, 1, flush, stream)[0] / 1e3
            sb.close()
            pls = []
            for sc, M, L, seed in sub:
                pl = binding.Planner(sc.robot, M, L, H, max_obstacles=64)
                pl.set_scene(sc)
                pls.append((pl, M, L, seed, torch.empty(L, dtype=torch.int32, device="cuda"),
                            torch.empty(1, dtype=torch.float32, device="cuda")))

            def run_sub():
                for pl, M, L, seed, pa, co in pls:
                    binding.gtmp_sample_layers(pl.ctx, seed, M)
                    binding.gtmp_solve(pl.ctx, pa, co)
            run_sub()
            t_p = _timed_passes(run_sub, 1, flush, stream)[0] / 1e3
            out["breakdown"][name] = {"problems": len(sub), "batched_s": t_b, "plain_s": t_p}
            for pl, *_ in pls:
                pl.close()
    return out


def run_batched(args, wl):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    r = measure_batched(args, wl, flush, args.steps, args.warmup, lazy=args.lazy, breakdown=args.breakdown)
    if rank == 0:
        ee = r["early_exit"]
        print(json.dumps({
            "metric": METRIC, "value": ee["batched_checks_per_s"], "unit": "checks/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ee["batched_ms_per_batch"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded scenes and samples)", "solves_per_s": ee["batched_solves_per_s"],
            "config": {"workload": args.workload, "problems": wl["n"], "H": wl["H"], "l2": r["l2"]},
            "gpu_launches": ee["gpu_launches_per_batch"] * args.steps, "clocks": r["clocks"], "batched": r}),
              flush=True)


def measure_surrogate(args, wl, flush, steps, warmup, n_train=None, epochs=None):
    """Surrogate-pruned solves against plain solves of the same samples, early exit and lazy."""
    import numpy as np
    import torch

    from paper_2608_25830_b300 import binding, scenes

    rank, world, local = dist_env()
    M, L, H = wl["M"], wl["L"], wl["H"]
    sc = gpu_endpoints(binding, scenes, scenes.arm_scene(wl["seed"], wl["dof"], wl["n_obs"]))
    planners = {}
    for name, mode in (("early_exit", binding.EVAL_EARLY_EXIT), ("lazy", binding.EVAL_LAZY)):
        planners[name] = binding.Planner(sc.robot, M, L, H, max_obstacles=64, eval_mode=mode)
        planners[name].set_scene(sc)
    n_train = n_train or wl["n_train"]
    train = binding.gtmp_surrogate_train(planners["early_exit"].ctx, n_train=n_train, n_holdout=1 << 16,
                                         epochs=epochs or wl["epochs"], batch=1024, lr=1e-3, seed=1,
                                         fourier_sigma=wl["sigma"])
    binding.gtmp_surrogate_set_params(planners["lazy"].ctx,
                                      binding.gtmp_surrogate_get_params(planners["early_exit"].ctx, sc.robot.dof))
    thr, kw = wl["threshold"], wl["score_waypoints"]
    band = wl.get("protect", 0.0)   # edges within (1 + band) x their row's best bound stay exact
    for pl in planners.values():
        binding.gtmp_surrogate_set_protect(pl.ctx, band)
    stream = torch.cuda.current_stream()
    path = torch.empty(L, dtype=torch.int32, device="cuda")
    cost = torch.empty(1, dtype=torch.float32, device="cuda")
    seed0 = rank_seed_base(rank)
    times = {k: [] for k in ("early_exit", "early_exit_pruned", "lazy", "lazy_pruned")}
    band_only_ms, band_only_ratios, band_only_lost = [], [], 0
    ratios, pruned_frac, colliding_waypoints, checked = [], [], 0, 0
    score_ms, live_edges, band_ms, lists_ms = [], [], [], []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        flush.zero_()
        torch.cuda.synchronize()
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), r

    def recheck(pl, pa):
        """Every waypoint of a returned chain through the exact checker (GPU)."""
        Q = pl.get_layers().double().cpu().numpy()
        verts = [sc.q_start.astype(np.float64)] + [Q[l, pa[l]] for l in range(L)] + [sc.q_goal.astype(np.float64)]
        t = np.arange(H, dtype=np.float64)[:, None] / (H - 1)
        wps = np.concatenate([u + t * (v - u) for u, v in zip(verts[:-1], verts[1:])]).astype(np.float32)
        return int(pl.label_configs(torch.from_numpy(wps).cuda()).sum()), len(wps)

    with ClockSampler(gpu_uuid(local)) as clk:
        for s in range(-warmup, steps):
            seed = seed0 + (10_000 + s if s < 0 else s)
            row = {}
            for name, pl in planners.items():
                pl.sample_layers(seed, M)
                ms, _ = timed(lambda: binding.gtmp_solve(pl.ctx, path, cost))
                c_plain = float(cost.cpu()[0])
                msp, st = timed(lambda: binding.gtmp_solve_pruned(pl.ctx, thr, path, cost, score_waypoints=kw))
                c_pruned = float(cost.cpu()[0])
                row[name] = (ms, msp, c_plain, c_pruned, st)
                if name == "early_exit" and band > 0 and s >= 0:
                    # the band without the model: every live edge outside it pruned (threshold ~0)
                    msb, _ = timed(lambda: binding.gtmp_solve_pruned(pl.ctx, 1e-6, path, cost, score_waypoints=kw))
                    c_band = float(cost.cpu()[0])
                    band_only_ms.append(msb)
                    if math.isfinite(c_plain):
                        if math.isinf(c_band):
                            band_only_lost += 1
                        else:
                            band_only_ratios.append(c_band / c_plain)
                if s >= 0 and math.isfinite(c_pruned):
                    bad, n = recheck(pl, path.cpu().numpy())
                    colliding_waypoints += bad
                    checked += n
            if s < 0:
                continue
            for name in planners:
                ms, msp, c_plain, c_pruned, st = row[name]
                times[name].append(ms)
                times[name + "_pruned"].append(msp)
            ms, msp, c_plain, c_pruned, st = row["early_exit"]
            assert row["lazy"][2] == c_plain or (math.isinf(c_plain) and math.isinf(row["lazy"][2]))
            pruned_frac.append(st["pruned"] / st["edges"])
            score_ms.append(st["score_ms"])
            band_ms.append(st["band_ms"])
            lists_ms.append(st["lists_ms"])
            live_edges.append(st["scored"])
            if math.isfinite(c_plain):
                ratios.append(c_pruned / c_plain if math.isfinite(c_pruned) else math.inf)
    for pl in planners.values():
        pl.close()
    # tensor-core roofline of the fused scoring kernel: 164 096 MAC per scored waypoint (128x256 + 2x256x256
    # + 256), one scored waypoint per live edge; the live-edge count is measured from the same solves.  The
    # kernel runs inside a solve, so the sustained bf16 rate is its peak.
    peaks = measured_peaks()
    tfl = 2.0 * 164096 * kw * (sum(live_edges) / len(live_edges)) / (sum(score_ms) / len(score_ms) / 1e3) / 1e12
    pk = peaks.get("bf16_tflops_sustained")
    roof = {"bound": "tensor", "kernel": "score_edges_kernel (BF16 MLP, tcgen05)", "achieved": tfl,
            "peak": pk, "unit": "TFLOP/s", "frac": tfl / pk if pk else None, "traffic": None,
            "peak_basis": f"cuBLAS bf16 GEMM sustained (bf16_tflops_sustained, {peaks['source']})",
            "frac_of_burst": tfl / peaks["bf16_tflops"] if peaks.get("bf16_tflops") else None,
            "score_ms_per_solve": sum(score_ms) / len(score_ms),
            "band_ms_per_solve": sum(band_ms) / len(band_ms),
            "live_edges_per_solve": sum(live_edges) / len(live_edges),
            "lists_ms_per_solve": sum(lists_ms) / len(lists_ms),
            "note": "score_ms: the scoring kernel alone (CUDA events on its stream); the live lists it reads are "
                    "lists_ms and the protection-band pass band_ms"}
    tot = {k: max_over_ranks(sum(v) / 1e3, world, "cuda") for k, v in times.items()}
    sps = {k: steps * world / v for k, v in tot.items()}
    fin = [r for r in ratios if math.isfinite(r)]
    return {
        "workload": "7-DoF arm, 40 obstacles, M=4096, L=8, H=32; MLP Fourier(64)-256-256-256-1, bf16",
        "M": M, "L": L, "H": H, "dof": wl["dof"], "obstacles": wl["n_obs"], "threshold": thr,
        "protection_band": band, "score_waypoints": kw, "train_configs": n_train, "steps": steps,
        "warmup": warmup,
        "solves_per_s": sps,
        "ms_per_solve": {k: 1e3 / v for k, v in sps.items()},
        "surrogate_over_plain": {"early_exit": sps["early_exit_pruned"] / sps["early_exit"],
                                 "lazy": sps["lazy_pruned"] / sps["lazy"]},
        "cost_ratio_pruned_over_plain": {"mean": float(np.mean(fin)) if fin else None,
                                         "max": float(np.max(fin)) if fin else None,
                                         "lost_feasibility": len(ratios) - len(fin), "solves": len(ratios)},
        "roofline": roof,
        "band_only": ({"early_exit_solves_per_s": len(band_only_ms) / (sum(band_only_ms) / 1e3),
                       "over_plain": (len(band_only_ms) / (sum(band_only_ms) / 1e3)) / sps["early_exit"],
                       "cost_ratio_mean": float(np.mean(band_only_ratios)) if band_only_ratios else None,
                       "cost_ratio_max": float(np.max(band_only_ratios)) if band_only_ratios else None,
                       "lost_feasibility": band_only_lost,
                       "note": "the protection band alone (every live edge outside it pruned, no model decision): a "
                               "bound heuristic shown for comparison"} if band_only_ms else None),
        "pruned_edge_fraction": float(np.mean(pruned_frac)),
        "returned_paths_recheck": {"waypoints": checked, "colliding": colliding_waypoints},
        "training": train,
        "clocks": clk.summary(),
        "l2": "flushed before every solve",
        "note": "plain and pruned solve the same samples (seed = step) in each mode; an edge is pruned when its "
                "midpoint's collision probability exceeds the threshold and its bound |v - u| + J(v) lies above "
                "(1 + protection_band) x its row's best bound; every returned chain is re-checked at all H "
                "waypoints of every edge by the exact checker",
    }


def run_surrogate(args, wl):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    r = measure_surrogate(args, wl, flush, args.steps, args.warmup,
                          n_train=args.sur_train or None, epochs=1 if args.sur_train else None)
    if rank == 0:
        print(json.dumps({
            "metric": "solves/s, surrogate-pruned vs plain (7-DoF, M=4096, L=8, H=32, 40 obstacles)",
            "value": r["solves_per_s"]["early_exit_pruned"], "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_solve"]["early_exit_pruned"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 surrogate, f32 checker",
            "data": "synthetic (seeded scene and samples)",
            "config": {"workload": args.workload, "M": wl["M"], "L": wl["L"], "H": wl["H"], "l2": r["l2"]},
            "clocks": r["clocks"], "roofline": r["roofline"], "surrogate": r}), flush=True)


def run_classes(args, wl):
    """Class-augmented value iteration (Prop. 1) on a planar scene: each step samples one layered graph and
    returns a minimum-cost chain in every realised class; then Alg. 1's anytime-gtmp class archive over R
    restarts.  The oracle's class sweep of the same graphs is the CPU baseline."""
    import numpy as np
    import torch

    from paper_2608_25830_b300 import binding, scenes

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    M, L, H, K, R = wl["M"], wl["L"], wl["H"], wl["K"], wl["R"]
    sc = scenes.point2d_scene(wl["seed"], wl["n_obs"])
    p = binding.Planner(sc.robot, M, L, H, max_obstacles=64)
    p.set_scene(sc)
    paths = torch.empty((K, L), dtype=torch.int32, device="cuda")
    costs = torch.empty(K, dtype=torch.float32, device="cuda")
    labels = torch.empty((K, 16), dtype=torch.int8, device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    seed0 = rank_seed_base(rank)
    for s in range(args.warmup):
        binding.gtmp_sample_layers(p.ctx, seed0 + 10_000 + s, M)
        binding.gtmp_solve_classes(p.ctx, K, K, paths, costs, labels)
    torch.cuda.synchronize()
    binding.gtmp_profile_read(p.ctx)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms, n_cls = [], []
    for s in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0.record(stream)
        binding.gtmp_sample_layers(p.ctx, seed0 + s, M)
        n_cls.append(binding.gtmp_solve_classes(p.ctx, K, K, paths, costs, labels))
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    launches = binding.gtmp_profile_read(p.ctx)["launches"]
    total_s = max_over_ranks(sum(ms) / 1e3, world, "cuda")
    t0 = time.perf_counter()
    archive = p.anytime_classes(seed0 + 20_000, R, K, K)
    torch.cuda.synchronize()
    archive_ms = (time.perf_counter() - t0) * 1e3
    p.close()
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            import oracle
            done, t0 = 0, time.perf_counter()
            while time.perf_counter() - t0 < args.cpu_budget:
                Q = oracle.sample_uniform(seed0 + done, 0, L, M, sc.robot.q_lo, sc.robot.q_hi)
                verts = oracle.layer_vertices(Q, sc.q_start, sc.q_goal)
                oracle.class_value_iteration(oracle.realize_edges(sc, verts, H), verts, oracle.obstacle_centres_2d(sc))
                done += 1
            secs = time.perf_counter() - t0
            cpu = {"value": done / secs, "unit": "solves/s", "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count())),
                   "kind": "oracle", "sample": f"{done} whole graphs (edges in C with OpenMP, class sweep in Python) "
                                               f"in {secs:.1f} s"}
        print(json.dumps({
            "metric": "class-augmented solves/s (every realised class of one layered graph)",
            "value": args.steps * world / total_s, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sum(ms) / len(ms), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 costs, exact f64 orientation labels",
            "data": "synthetic (seeded planar scene and samples)",
            "config": {"workload": args.workload, "M": M, "L": L, "H": H, "obstacles": wl["n_obs"], "max_labels": K,
                       "l2": "flushed between steps"},
            "classes_per_solve": sum(n_cls) / len(n_cls), "gpu_launches": int(launches),
            "anytime_archive": {"restarts": R, "classes": len(archive), "ms": archive_ms,
                                "best_cost": min(c for c, _, _ in archive.values()) if archive else None},
            "cpu_baseline": cpu,
        }), flush=True)


def measure_anytime(args, wl, flush, steps, warmup, lazy=False):
    """Anytime-GTMP: R restarts of one problem, all in one batch of launches (restart = grid.y)."""
    import numpy as np
    import torch

    from paper_2608_25830_b300 import binding, scenes

    rank, world, local = dist_env()
    M, L, H, R = wl["M"], wl["L"], wl["H"], wl["R"]
    sc = gpu_endpoints(binding, scenes, scenes.arm_scene(wl["seed"], wl["dof"], wl["n_obs"]))
    p = binding.Planner(sc.robot, M, L, H, R=R, max_obstacles=64,
                        eval_mode=binding.EVAL_LAZY if lazy else binding.EVAL_EARLY_EXIT)
    p.set_scene(sc)
    paths = torch.empty((R, L), dtype=torch.int32, device="cuda")
    costs = torch.empty(R, dtype=torch.float32, device="cuda")
    best = torch.empty(1, dtype=torch.int32, device="cuda")
    seed0 = rank_seed_base(rank)
    for s in range(warmup):
        binding.gtmp_anytime(p.ctx, seed0 + 10_000 + s, R, paths, costs, best)
    p.synchronize()
    stream = torch.cuda.current_stream()
    it = iter(range(steps))
    with ClockSampler(gpu_uuid(local)) as clk:
        ms = _timed_passes(lambda: binding.gtmp_anytime(p.ctx, seed0 + next(it), R, paths, costs, best),
                           steps, flush, stream)
    p.synchronize()
    p.close()
    total_s = max_over_ranks(sum(ms) / 1e3, world, "cuda")
    checks = R * H * (2 * M + (L - 1) * M * M)
    c = costs.cpu().numpy()
    b = int(best.cpu()[0])
    return {"workload": f"{wl['dof']}-DoF arm, {wl['n_obs']} obstacles, {R} restarts, M={M}, L={L}, H={H}",
            "restarts": R, "M": M, "L": L, "H": H, "dof": wl["dof"], "eval_mode": "lazy" if lazy else "early_exit",
            "steps": steps, "warmup": warmup,
            "solves_per_s": R * steps * world / total_s, "checks_per_s": checks * steps * world / total_s,
            "ms_per_launch_batch": sum(ms) / len(ms), "checks_per_launch_batch": checks,
            "feasible_restarts": int(np.isfinite(c).sum()), "best_cost": float(c[b]) if b >= 0 else None,
            "clocks": clk.summary(), "l2": "flushed before every launch batch"}


def run_anytime(args, wl):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    r = measure_anytime(args, wl, flush, args.steps, args.warmup, lazy=args.lazy)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": r["checks_per_s"], "unit": "checks/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_launch_batch"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "solves_per_s": r["solves_per_s"], "config": {"workload": args.workload, "l2": r["l2"]},
            "clocks": r["clocks"], "anytime": r}), flush=True)


def measure_ao(args, wl, steps, warmup, lazy=False, epochs=True):
    """AO-GTMP: M doubles from M0 to M1 (L fixed), best cost against device time; then the epoch schedule."""
    import torch

    from paper_2608_25830_b300 import binding, scenes

    rank, world, local = dist_env()
    L, H = wl["L"], wl["H"]
    sizes = []
    m = wl["M0"]
    while m <= wl["M1"]:
        sizes.append(m)
        m *= 2
    sc = gpu_endpoints(binding, scenes, scenes.arm_scene(wl["seed"], wl["dof"], wl["n_obs"]))
    stream = torch.cuda.current_stream()
    mode = binding.EVAL_LAZY if lazy else binding.EVAL_EARLY_EXIT

    def run_schedule(seed):
        """One schedule from an empty graph (a fresh context; its creation is outside the events)."""
        p = binding.Planner(sc.robot, sizes[-1], L, H, max_obstacles=64, eval_mode=mode)
        p.set_scene(sc)
        sp = torch.empty(L, dtype=torch.int32, device="cuda")
        scost = torch.empty(1, dtype=torch.float32, device="cuda")
        bp = torch.full((L,), -1, dtype=torch.int32, device="cuda")
        bc = torch.full((1,), math.inf, dtype=torch.float32, device="cuda")
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(sizes) + 1)]
        best = []
        torch.cuda.synchronize()
        evs[0].record(stream)
        for k, M in enumerate(sizes):
            binding.aogtmp_expand(p.ctx, seed, M, sp, scost, bp, bc)
            evs[k + 1].record(stream)
            best.append(bc.clone())
        torch.cuda.synchronize()
        p.synchronize()
        p.close()
        return [(evs[0].elapsed_time(evs[k + 1]), float(best[k].cpu()[0])) for k in range(len(sizes))]

    for s in range(warmup):
        run_schedule(rank_seed_base(rank) + 50_000 + s)
    with ClockSampler(gpu_uuid(local)) as clk:
        curves = [run_schedule(rank_seed_base(rank) + s) for s in range(steps)]
    total_s = max_over_ranks(sum(c[-1][0] for c in curves) / 1e3, world, "cuda")
    checks = sum(H * (2 * M + (L - 1) * M * M) for M in sizes)
    out = {"workload": f"{wl['dof']}-DoF arm, {wl['n_obs']} obstacles, AO-GTMP M {sizes[0]} -> {sizes[-1]} "
                       f"(x2 per stage), L={L}, H={H}",
           "M_stages": sizes, "L": L, "H": H, "dof": wl["dof"], "eval_mode": "lazy" if lazy else "early_exit",
           "steps": steps, "warmup": warmup,
           "ms_per_schedule": total_s * 1e3 / steps, "checks_per_s": checks * steps * world / total_s,
           "checks_per_schedule": checks,
           "best_cost_vs_time_ms": [[round(t, 3), c] for t, c in curves[0]],
           "final_best_cost_per_schedule": [c[-1][1] for c in curves],
           "clocks": clk.summary(), "l2": "not flushed inside a schedule (stages are sequential)"}
    ep = wl.get("epochs")
    if epochs and ep is not None:
        # epochs (Sec. IV-D): layer count grown by the layer rule and by saturation, edge limit l_M(r)
        pe = binding.Planner(sc.robot, ep["M_max"], ep["L_cap"], H, max_obstacles=64, eval_mode=mode)
        pe.set_scene(sc)
        kw = {k: ep[k] for k in ("L0", "M0", "M_max", "stages", "reach", "r", "varsigma", "limit_edges")}
        pe.ao_run(rank_seed_base(rank) + 50_000, **kw)          # warm-up
        pe.synchronize()
        runs = []
        for s in range(min(3, steps)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, cost_e, log, best_layers = pe.ao_run(rank_seed_base(rank) + s, **kw)
            pe.synchronize()
            runs.append((time.perf_counter() - t0, log, best_layers))
        pe.close()
        wall, log, best_layers = runs[0]
        out["epochs"] = {"schedule": ep, "wall_ms_per_run": [round(r[0] * 1e3, 3) for r in runs],
                         "best_cost_per_run": [r[1][-1]["best_cost"] for r in runs],
                         "best_chain_layers": best_layers,
                         "stages": [[r["epoch"], r["L"], r["M"], round(r["edge_limit"], 5), r["stage_cost"],
                                     r["best_cost"]] for r in log],
                         "note": "host wall time (the driver reads the best cost back after every stage); stages = "
                                 "[epoch, L, M, edge limit, stage cost, best cost]"}
    return out


def run_ao(args, wl):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    r = measure_ao(args, wl, args.steps, args.warmup, lazy=args.lazy)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": r["checks_per_s"], "unit": "checks/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_schedule"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "l2": r["l2"]}, "clocks": r["clocks"], "ao": r}), flush=True)


def main():
    from paper_2608_25830_b300 import scenes
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="arm7_m1024_l8_h32", choices=sorted(scenes.WORKLOADS))
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--ref-budget", type=float, default=6.0, help="seconds of oracle work per reference step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-unfused", action="store_true", help="skip the unfused min-plus roofline (M=4096)")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload: skip the batched, surrogate, anytime and AO comparisons")
    ap.add_argument("--lazy", action="store_true",
                    help="batched workload: also time the lazy mode, both forms; anytime / AO workloads: lazy mode")
    ap.add_argument("--sur-train", type=int, default=0,
                    help="surrogate workload: train on this many configurations for one epoch (short runs for profiling)")
    ap.add_argument("--breakdown", action="store_true", help="batched workload: time arm and 2D subsets separately")
    args = ap.parse_args()
    wl = dict(scenes.WORKLOADS[args.workload])
    if wl["kind"] == "classes":
        if args.impl == "reference":
            raise SystemExit("the reference arm times the single-solve workload")
        run_classes(args, wl)
        return
    if wl["kind"] == "batched" or "R" in wl or "M0" in wl:
        if args.impl == "reference":
            raise SystemExit("the reference arm times the single-solve workload")
        {"batched": run_batched}.get(wl["kind"], run_anytime if "R" in wl else run_ao)(args, wl)
        return
    if "n_train" in wl:
        if args.impl == "reference":
            raise SystemExit("the reference arm times the single-solve workload")
        run_surrogate(args, wl)
        return
    if "M" not in wl:
        raise SystemExit(f"{args.workload} is not a single-solve workload")
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
