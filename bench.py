"""Benchmark: Lamarckian-GA docking of the drug-size workload on GB300.

One step = one full docking (every step of the hot path: pose build, grid
and pair energies, analytic gradient, ADADELTA and the genetic operators) of
a 40-atom / 10-torsion ligand against 64^3 x 9 receptor maps built from a
3000-atom receptor: 50 runs x 2.5M evaluations, population 150, ADADELTA
300 iterations on 6% of each generation.  Inputs are seeded synthetic data
shaped like the paper's workloads.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  With N > 1 (launched by torchrun) every rank
docks its own replica (its own seed); there is no exchange step, so the only
collectives are the timing barrier and the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "score+grad evals/s (docking, all evaluations counted)"
UNIT = "evals/s"
L2_FLUSH_BYTES = 256 << 20

# ---------------------------------------------------------------------------
# algorithmic work per evaluation: the FP32 operations the method needs,
# counted from its formulas (an FMA counts as 2; a 3x4 transform of a point
# is 9 FMA + 3 adds = 21, a lerp is 3), not from the instructions issued.


def flops_score_grad(n_atoms: int, n_tors: int, n_pairs: int, n_pairs_in: float) -> float:
    """Per score+gradient evaluation: torsion rotations and forward kinematics
    153 per torsion; per atom 165 (pose 24, three trilinear reads with
    gradient 108, combine 18, force/torque sums 15); per pair inside the 8 A
    cutoff 77 (distance 8, energy terms 28, dE/dr 23, force gather 18), per
    pair beyond it 8 (distance only); root transform 37."""
    return 37.0 + 153.0 * n_tors + 165.0 * n_atoms + 77.0 * n_pairs_in + 8.0 * (n_pairs - n_pairs_in)


def grid_bytes_per_eval(n_atoms: int) -> int:
    """Algorithmic L2->SM bytes: 3 maps x 8 corners x 4 B per atom."""
    return 96 * n_atoms


# ---------------------------------------------------------------------------
# distributed helpers (host logic, tested with gloo on CPU)

def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def replica_seed(base_seed: int, rank: int) -> int:
    """Each rank docks an independent replica of the workload."""
    return base_seed + 1_000_003 * rank


def max_over_ranks(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ---------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9 and f[1].replace(".", "").isdigit():
                    rows.append(f)
        finally:
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = np.array([float(r[1]) for r in rows])
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(float(r[2]) for r in rows)),
                "reasons": reasons, "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows)}


# ---------------------------------------------------------------------------
# synthetic ligands in parallel (spawned worker processes, which touch no GPU)

def _ligand_worker(spec):
    from paper_2203_02096_gb300 import synth
    n, t, seed = spec
    return synth.make_ligand(n, t, seed=seed)


def make_ligands(specs):
    """synth.make_ligand(n, t, seed=seed) for each (n, t, seed), in order."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    specs = list(specs)
    workers = min(len(specs), os.cpu_count() or 1)
    if workers <= 1:
        return [_ligand_worker(sp) for sp in specs]
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_ligand_worker, specs, chunksize=max(1, len(specs) // (4 * workers))))


# ---------------------------------------------------------------------------
# the workload

def workload():
    from paper_2203_02096_gb300 import synth
    return synth.drug_ligand_workload()


def config_dict(w, l2_note: str):
    return {"workload": "plain docking, drug-size ligand", "ligand_atoms": w.ligand.n_atoms,
            "torsions": w.ligand.n_torsions, "grid": f"{w.box.dims[0]}^3 x {w.box.n_maps} maps FP32",
            "receptor_atoms": len(w.receptor.types), "nruns": w.nruns, "max_evals_per_run": w.max_evals,
            "pop_size": w.pop_size, "local_search": f"ADADELTA {w.ls_iters} iterations on {w.ls_rate_pct}%",
            "l2": l2_note}


_ORACLE_INPUTS = {}


def cpu_sample(w, target_s: float, seed: int = 0):
    """The FP64 oracle as it stands, on this host's cores: one docking run per
    core with a budget sized to about target_s of CPU work.  Returns (evals/s,
    cores, sample description, wall seconds).  The oracle builds its own maps
    (untimed, once)."""
    import oracle
    cores = os.cpu_count() or 1
    if w.name not in _ORACLE_INPUTS:
        maps = oracle.build_maps(w.receptor, w.box, nthreads=cores).astype(np.float32)
        _ORACLE_INPUTS[w.name] = (oracle.OracleGrid(maps, w.box), oracle.OracleLigand(w.ligand))
    grid, lig = _ORACLE_INPUTS[w.name]
    # calibration: score+grad throughput on all cores
    from paper_2203_02096_gb300 import synth
    g = synth.make_genotypes(4 * cores * 50, lig.n_torsions, w.box, seed=1)
    t0 = time.perf_counter()
    lig.score_batch(grid, g, with_grad=True, nthreads=cores)
    rate = len(g) / (time.perf_counter() - t0)
    per_gen = (w.pop_size - 1) + ((w.ls_rate_pct * w.pop_size + 99) // 100) * w.ls_iters
    budget = max(w.pop_size + per_gen, int(rate * target_s / cores))
    P = oracle.make_params(pop_size=w.pop_size, nruns=cores, max_evals=budget, ls_iters=w.ls_iters,
                           ls_rate_pct=w.ls_rate_pct)
    t0 = time.perf_counter()
    _, best_E, evals = oracle.dock(lig, grid, P, seed, nthreads=cores)
    dt = time.perf_counter() - t0
    desc = (f"{cores} docking runs x {int(evals[0])} evaluations of the drug-size workload (50 runs x 2.5M "
            f"in full), FP64 oracle, one run per thread")
    _ORACLE_INPUTS["last_sample"] = {"runs": cores, "budget_per_run": budget, "seed": seed, "best_E": best_E,
                                     "evals": evals}
    return float(evals.sum() / dt), cores, desc, dt


def cpu_other_workloads(head):
    """The FP64 oracle as it stands on the other workloads, on this host's
    cores (maps built by the oracle, untimed):
    - small-ligand docking (16 atoms / 4 torsions, 40^3 x 7 maps, 10 runs x
      100k evaluations) in full;
    - score+grad of the 65536-genotype batch of a 64-atom / 16-torsion ligand
      in the drug-size grids, in full;
    - the batching mix (10-108 atoms, 0-32 torsions, 80^3 x 9 maps) and the
      serving mix (10-128 atoms log-uniform, 0-32 torsions; on the same
      80^3 maps, the serving workload's 96^3 maps not being built here):
      16 of the workload's own ligands spread over the size range, one
      docking of `cores` runs x ~3300 evaluations each (three generations),
      extrapolated to 20 runs x 1M (batching) and 20 runs x 500k (serving)
      evaluations per ligand."""
    import oracle

    from paper_2203_02096_gb300 import synth
    cores = os.cpu_count() or 1
    out = {"cores": cores, "kind": "oracle"}
    w1 = synth.small_ligand_workload()
    g1 = oracle.OracleGrid(oracle.build_maps(w1.receptor, w1.box, nthreads=cores).astype(np.float32), w1.box)
    P = oracle.make_params(pop_size=w1.pop_size, nruns=w1.nruns, max_evals=w1.max_evals, ls_iters=w1.ls_iters,
                           ls_rate_pct=w1.ls_rate_pct)
    t0 = time.perf_counter()
    _, _, ev = oracle.dock(oracle.OracleLigand(w1.ligand), g1, P, w1.seed, nthreads=cores)
    dt = time.perf_counter() - t0
    out["small_ligand_docking"] = {"workload": w1.name, "in_full": True, "seconds": dt,
                                   "evals_per_s": float(ev.sum()) / dt, "ligands_per_hour": 3600.0 / dt,
                                   "threads": min(cores, w1.nruns)}
    grid = _ORACLE_INPUTS[head.name][0]
    lig = synth.make_ligand(64, 16, seed=0)
    X = synth.make_genotypes(65536, lig.n_torsions, head.box, seed=0)
    t0 = time.perf_counter()
    oracle.OracleLigand(lig).score_batch(grid, X, with_grad=True, nthreads=cores)
    dt = time.perf_counter() - t0
    out["score_grad_batch"] = {"workload": "65536 genotypes, 64 atoms / 16 torsions, 64^3 x 9 maps", "in_full": True,
                               "seconds": dt, "evals_per_s": 65536 / dt}
    box = synth.make_box(80)
    g3 = oracle.OracleGrid(oracle.build_maps(synth.make_receptor(3000, seed=4), box,
                                             nthreads=cores).astype(np.float32), box)
    mixes = {"batching": (_batching_specs(1024), 1_000_000), "serving": (_serving_specs(1024), 500_000)}
    P = oracle.make_params(pop_size=150, nruns=cores, max_evals=3000, ls_iters=100)
    for name, (specs, full_budget) in mixes.items():
        order = np.argsort([n for n, _, _ in specs], kind="stable")
        pick = order[np.linspace(0, len(specs) - 1, 16).round().astype(int)]
        ligs = [oracle.OracleLigand(synth.make_ligand(*specs[k][:2], seed=specs[k][2])) for k in pick]
        evals = 0
        t0 = time.perf_counter()
        for k, ol in zip(pick, ligs):
            _, _, ev = oracle.dock(ol, g3, P, int(k), nthreads=cores)
            evals += int(ev.sum())
        dt = time.perf_counter() - t0
        rate = evals / dt
        out[name] = {"workload": f"{name} ligand mix, 80^3 x 9 maps", "in_full": False,
                     "sample": f"16 of its ligands ({specs[pick[0]][0]}-{specs[pick[-1]][0]} atoms, every "
                               f"64th by size) x {cores} runs x {int(evals / 16 / cores)} evaluations",
                     "seconds": dt, "evals_per_s": rate,
                     "ligands_per_hour_extrapolated": 3600.0 * rate / (20 * full_budget),
                     "extrapolated_to": f"20 runs x {full_budget} evaluations per ligand"}
    return out


def _ks(a, b):
    a, b = np.sort(a), np.sort(b)
    xs = np.concatenate([a, b])
    return float(np.max(np.abs(np.searchsorted(a, xs, side="right") / len(a)
                               - np.searchsorted(b, xs, side="right") / len(b))))


def quality_vs_oracle(ctx, G, L, w):
    """The GPU docking at the oracle sample's budget, runs and seed: both
    forms' best energies (the same search, FP32 against FP64), as medians and
    a two-sample Kolmogorov-Smirnov distance."""
    from paper_2203_02096_gb300 import capi
    smp = _ORACLE_INPUTS.get("last_sample")
    if smp is None:
        return None
    P = capi.default_params(pop_size=w.pop_size, nruns=smp["runs"], max_evals=smp["budget_per_run"],
                            ls_iters=w.ls_iters)
    _, gE, gev = capi.dock(ctx, G, L, P, smp["seed"])
    oE = smp["best_E"]
    return {"runs": smp["runs"], "budget_per_run": smp["budget_per_run"], "seed": smp["seed"],
            "same_evaluation_counts": bool(np.array_equal(gev, smp["evals"])),
            "best_E_median": {"gpu": float(np.median(gE)), "oracle": float(np.median(oE))},
            "best_E_min": {"gpu": float(gE.min()), "oracle": float(oE.min())}, "ks": _ks(gE, oE)}


# ---------------------------------------------------------------------------

def run_reference(args):
    """The oracle arm: the FP64 CPU oracle timed on the host cores."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = workload()
    per_step = max(3.0, min(10.0, 150.0 / max(1, args.steps + args.warmup)))
    vals, cores, desc, total = [], 1, "", 0.0
    for k in range(args.warmup + args.steps):
        v, cores, desc, dt = cpu_sample(w, per_step if k >= args.warmup else 1.0, seed=k)
        if k >= args.warmup:
            vals.append(v)
            total += dt
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(w, "n/a (CPU)"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run(args):
    import torch
    import torch.distributed as dist

    from paper_2203_02096_gb300 import autotune, capi

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    w = workload()
    ctx = capi.Context(local)
    # setup (untimed): receptor maps on the device, ligand resident
    G = capi.grids_from_receptor(ctx, w.receptor, w.box)
    L = capi.ligand_from(ctx, w.ligand)
    P = capi.default_params(pop_size=w.pop_size, nruns=w.nruns, max_evals=w.max_evals, ls_iters=w.ls_iters,
                            ls_threads=max(args.ls_threads, 0))
    tune_dir = tempfile.mkdtemp(prefix="dock_tune_")
    tuner = autotune.Tuner(ctx, path=os.path.join(tune_dir, "tune.json"))
    if args.ls_threads < 0:      # the autotuner picks the threads per local-search chain (untimed)
        P = tuner.tuned(G, L, P)
    seed = replica_seed(w.seed, rank)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    out = None
    for k in range(args.warmup):
        out = capi.dock_async(ctx, G, L, P, seed + k, out=out)
    torch.cuda.synchronize(dev)

    # ---- timed region: K full dockings, L2 flushed between them
    ctx.reset_timing()
    ctx.set_timing(True)
    launches0 = ctx.launch_count()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize(dev)
        for k in range(args.steps):
            flush.fill_(float(k))
            starts[k].record(stream)
            out = capi.dock_async(ctx, G, L, P, seed + 100 + k, out=out)
            ends[k].record(stream)
        torch.cuda.synchronize(dev)
        barrier()
    ctx.set_timing(False)
    launches = ctx.launch_count() - launches0
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    evals_per_step = int(out["evals"].sum().item())
    my_s = sum(step_ms) / 1e3
    t_max = max_over_ranks(my_s, dev)
    total_evals = sum_over_ranks(float(evals_per_step * args.steps), dev)
    value = total_evals / t_max
    ligands_per_hour = 3600.0 * sum_over_ranks(float(args.steps), dev) / t_max
    ls_ms, ls_n = ctx.kernel_time("dock_ls")
    ga_ms, ga_n = ctx.kernel_time("dock_ga")
    clocks = clk.summary()

    # algorithmic work of the dominant kernel (the ADADELTA local search)
    nls = (w.ls_rate_pct * w.pop_size + 99) // 100
    evals_per_ls_launch = w.nruns * nls * w.ls_iters
    xyz = capi.pose_batch(ctx, L, out["best_geno"]).cpu().numpy()
    pij = pair_list(w.ligand)
    d = np.linalg.norm(xyz[:, pij[:, 0]] - xyz[:, pij[:, 1]], axis=2)
    p_in = float((d < 8.0).sum(axis=1).mean())
    f_eval = flops_score_grad(w.ligand.n_atoms, w.ligand.n_torsions, len(pij), p_in)
    ls_avg_s = ls_ms / max(ls_n, 1) / 1e3
    achieved = f_eval * evals_per_ls_launch / ls_avg_s / 1e12
    peak = peak_fp32_tflops()
    # measured device rates (microbenchmarks, untimed): context for the roofline
    measured = {"ffma_tflops": capi.microbench(ctx, capi.PEAK_FFMA),
                "ex2_gops": capi.microbench(ctx, capi.PEAK_EX2),
                "l2_read_gbs": capi.microbench(ctx, capi.PEAK_L2_READ)}

    # ---- end to end through the public API with host buffers
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize(dev)
    barrier()
    t0 = time.perf_counter()
    h2d = d2h = 0
    e2e_evals = 0
    for k in range(e2e_steps):
        Lk = capi.ligand_from(ctx, w.ligand)
        bg, bE, ev = capi.dock(ctx, G, Lk, P, seed + 200 + k)
        e2e_evals += int(ev.sum())
        Lk.free()
        h2d = w.ligand.nbytes()
        d2h = bg.nbytes + bE.nbytes + ev.nbytes
    torch.cuda.synchronize(dev)
    e2e_s = max_over_ranks(time.perf_counter() - t0, dev)
    e2e_value = sum_over_ranks(float(e2e_evals), dev) / e2e_s

    section_s = {}

    # the side studies and the CPU baseline are single-GPU measurements: a
    # multi-GPU run (replicas) times the headline only
    def side(name, fn):
        # a failing side study is reported in its section, not fatal to the
        # headline line
        t = time.perf_counter()
        r = None
        if not args.no_batch and world == 1:
            try:
                r = fn()
            except Exception as exc:  # noqa: BLE001
                torch.cuda.synchronize(dev)
                r = {"error": f"{type(exc).__name__}: {exc}"}
        section_s[name] = round(time.perf_counter() - t, 1)
        print(f"[bench] {name}: {section_s[name]} s", file=sys.stderr, flush=True)
        return r

    batch = side("score_grad_batch", lambda: score_grad_throughput(ctx, G, w.box, dev))
    multi = side("batched_docking", lambda: batched_docking(ctx, dev, full=not args.quick))
    serving = side("serving", lambda: serving_sweep(ctx, dev, full=not args.quick))
    solis = side("solis_wets", lambda: solis_wets_vs_adadelta(ctx, G, L, w, dev, out, value))
    graphs = side("cuda_graph", lambda: graph_vs_direct(ctx, G, L, P, dev))
    tuning = side("tuning", lambda: tuning_curves(ctx, G, w, tuner, P))

    cpu = quality = None
    if rank == 0 and world == 1 and not args.no_cpu:
        t = time.perf_counter()
        v, cores, desc, _ = cpu_sample(w, args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}
        section_s["cpu_baseline"] = round(time.perf_counter() - t, 1)
        quality = quality_vs_oracle(ctx, G, L, w)
        if not args.no_batch:
            t = time.perf_counter()
            cpu["other_workloads"] = cpu_other_workloads(w)
            section_s["cpu_other_workloads"] = round(time.perf_counter() - t, 1)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": float(np.mean(step_ms)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(config_dict(w, "flushed between steps (256 MB write, outside the step events)"),
                           ls_threads=f"{P.ls_threads} (autotuned)" if args.ls_threads < 0 else
                           (args.ls_threads or "library default")),
            "ligands_per_hour": ligands_per_hour,
            "roofline": {"bound": "alu", "kernel": "dock_ls (ADADELTA local search)", "achieved": achieved,
                         "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": LS_TRAFFIC_BYTES if sources_digest() == LS_TRAFFIC_SOURCES else None,
                         "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 FLOP x 2070 MHz (recipe unit counts, "
                                        "max SM clock of measured)",
                         "flops_per_eval": f_eval, "evals_per_launch": evals_per_ls_launch,
                         "launch_ms": ls_avg_s * 1e3, "launches": ls_n,
                         "l2_bytes_per_eval": grid_bytes_per_eval(w.ligand.n_atoms),
                         "l2_achieved_gbs": grid_bytes_per_eval(w.ligand.n_atoms) * evals_per_ls_launch / ls_avg_s / 1e9,
                         "measured_rates": measured,
                         "frac_of_measured_ffma": achieved / measured["ffma_tflops"],
                         "l2_frac_of_measured": grid_bytes_per_eval(w.ligand.n_atoms) * evals_per_ls_launch / ls_avg_s
                         / 1e9 / measured["l2_read_gbs"]},
            "kernel_share": {"dock_ls": ls_ms / sum(step_ms), "dock_ga": ga_ms / sum(step_ms)},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches),
            "clocks": {k: clocks[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
            "cpu_baseline": cpu,
            "quality_vs_oracle": quality,
            "score_grad_batch": batch,
            "batched_docking": multi,
            "serving": serving,
            "solis_wets": solis,
            "cuda_graph": graphs,
            "tuning": tuning,
            "best_energy_median": float(np.median(out["best_E"].cpu().numpy())),
            "side_section_seconds": section_s,
        }
        print(json.dumps(line), flush=True)
    for h in (L, G):
        h.free()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def score_grad_throughput(ctx, G, box, dev, reps: int = 5, score_blocks: int = 0):
    """score_grad_batch over 65536 random genotypes of a 64-atom / 16-torsion
    ligand in the same grids (the differentiation workload): evals/s and the
    FP32 roofline of that kernel (inputs resident, L2 flushed between calls).
    score_blocks > 0 fixes the scorer's register cap instead of tuning it."""
    import torch

    from paper_2203_02096_gb300 import autotune, capi, synth
    lig = synth.make_ligand(64, 16, seed=0)
    L = capi.ligand_from(ctx, lig)
    # register cap of the scorer by the autotuner (untimed), unless fixed
    tuner = autotune.Tuner(ctx, path=os.path.join(tempfile.mkdtemp(prefix="dock_tune_"), "tune.json"))
    if score_blocks > 0:
        blocks = score_blocks
        capi.set_option(ctx, capi.OPT_SCORE_BLOCKS, blocks)
    else:
        blocks = tuner.score_blocks(G, L)
    genos = torch.from_numpy(synth.make_genotypes(65536, lig.n_torsions, box, seed=0)).to(dev)
    E = torch.empty(65536, device=dev)
    grad = torch.empty_like(genos)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(3):
        capi.score_grad_batch(ctx, G, L, genos, E, grad)
    ms = []
    for k in range(reps):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        capi.score_grad_batch(ctx, G, L, genos, E, grad)
        b.record()
        torch.cuda.synchronize(dev)
        ms.append(a.elapsed_time(b))
    xyz = capi.pose_batch(ctx, L, genos[:1024]).cpu().numpy()
    pij = pair_list(lig)
    d = np.linalg.norm(xyz[:, pij[:, 0]] - xyz[:, pij[:, 1]], axis=2)
    p_in = float((d < 8.0).sum(axis=1).mean())
    f = flops_score_grad(lig.n_atoms, lig.n_torsions, len(pij), p_in)
    t = float(np.mean(ms)) / 1e3
    L.free()
    capi.set_option(ctx, capi.OPT_SCORE_BLOCKS, 1)
    achieved = f * 65536 / t / 1e12
    ffma, l2 = capi.microbench(ctx, capi.PEAK_FFMA), capi.microbench(ctx, capi.PEAK_L2_READ)
    return {"workload": "65536 genotypes, 64 atoms / 16 torsions, 64^3 x 9 maps", "evals_per_s": 65536 / t,
            "launch_ms": t * 1e3, "flops_per_eval": f, "achieved_tflops": achieved,
            "frac_fp32_peak": achieved / peak_fp32_tflops(),
            "l2_achieved_gbs": grid_bytes_per_eval(lig.n_atoms) * 65536 / t / 1e9,
            "frac_of_measured_ffma": achieved / ffma, "measured_ffma_tflops": ffma,
            "l2_frac_of_measured": grid_bytes_per_eval(lig.n_atoms) * 65536 / t / 1e9 / l2,
            "measured_l2_read_gbs": l2,
            "autotuned_score_blocks": blocks if score_blocks <= 0 else None, "score_blocks": blocks,
            "score_blocks_ms": tuner.curve("|score|")}


def run_score_grad_only(score_blocks: int = 0) -> int:
    """The score_grad_batch measurement alone (drug-size grids built on the GPU);
    score_blocks > 0 fixes the register cap (for profiling one cap)."""
    import torch

    from paper_2203_02096_gb300 import capi
    dev = torch.device("cuda", 0)
    w = workload()
    ctx = capi.Context(0)
    G = capi.grids_from_receptor(ctx, w.receptor, w.box)
    print(json.dumps(score_grad_throughput(ctx, G, w.box, dev, score_blocks=score_blocks)), flush=True)
    G.free()
    ctx.close()
    return 0


def run_batch_small() -> int:
    """A small batched docking alone, for profiling the persistent kernel:
    256 of the batching workload's ligands (10-108 atoms, 0-32 torsions), 8
    runs x 5000 evaluations, 80^3 x 9 maps; two dock_batch calls."""
    import torch

    from paper_2203_02096_gb300 import capi, synth
    dev = torch.device("cuda", 0)
    ctx = capi.Context(0)
    rng = np.random.default_rng(3)
    ligs = [synth.make_ligand(int(rng.integers(10, 109)), int(rng.integers(0, 33)), seed=5000 + k) for k in range(256)]
    G = capi.grids_from_receptor(ctx, synth.make_receptor(3000, seed=4), synth.make_box(80))
    L = [capi.ligand_from(ctx, l) for l in ligs]
    P = capi.default_params(pop_size=150, nruns=8, max_evals=5000, ls_iters=100)
    for k in range(2):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        out = capi.dock_batch(ctx, G, L, P, np.arange(256, dtype=np.uint64))
        b.record()
        torch.cuda.synchronize(dev)
    ev = int(out["evals"].sum().item())
    print(json.dumps({"workload": "256 ligands x 8 runs x 5000 evaluations", "evals_per_s": ev / (a.elapsed_time(b) / 1e3),
                      "seconds": a.elapsed_time(b) / 1e3}), flush=True)
    for h in L + [G]:
        h.free()
    ctx.close()
    return 0


def _serving_specs(n, seed=17):
    """(atoms, torsions, seed) of the first n ligands of the serving
    workload's request stream: atoms log-uniform in [10, 128]."""
    rng = np.random.default_rng(seed)
    specs = []
    for k in range(n):
        a = int(np.exp(rng.uniform(np.log(10), np.log(128.999))))
        specs.append((a, int(rng.integers(0, 33)), 9000 + k))
    return specs


def _serving_ligands(n, seed=17):
    """The first n ligands of the serving workload's request stream."""
    return make_ligands(_serving_specs(n, seed))


def _batching_specs(n):
    """(atoms, torsions, seed) of the batching workload's ligands: 10-108
    atoms and 0-32 torsions, uniform."""
    rng = np.random.default_rng(3)
    return [(int(rng.integers(10, 109)), int(rng.integers(0, 33)), 5000 + k) for k in range(n)]


def run_batch_96() -> int:
    """The persistent docking kernel on one 96^3 x 9 receptor of the serving
    workload (125 MB of z-column quads, about the size of L2): 608 of the
    serving workload's ligands x 4 runs x 4000 evaluations, two dock_batch
    calls (for an ncu capture of the second)."""
    import torch

    from paper_2203_02096_gb300 import capi, synth
    ctx = capi.Context(0)
    c = (12.5, -3.25, 7.0)
    G = capi.grids_from_receptor(ctx, synth.make_receptor(3000, center=c, seed=11), synth.make_box(96, center=c))
    L = [capi.ligand_from(ctx, l) for l in _serving_ligands(608)]
    P = capi.default_params(pop_size=150, nruns=4, max_evals=4000, ls_iters=100)
    for _ in range(2):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        out = capi.dock_batch(ctx, G, L, P, np.arange(len(L), dtype=np.uint64))
        b.record()
        torch.cuda.synchronize()
    ev = int(out["evals"].sum().item())
    print(json.dumps({"workload": "608 serving ligands x 4 runs x 4000 evaluations, one 96^3 x 9 receptor",
                      "evals": ev, "seconds": a.elapsed_time(b) / 1e3, "evals_per_s": ev / (a.elapsed_time(b) / 1e3)}),
          flush=True)
    for h in L + [G]:
        h.free()
    ctx.close()
    return 0


def run_serve_l2() -> int:
    """Served throughput with every request on one 96^3 x 9 receptor against
    requests alternating between two (2 x 125 MB of grid copies, twice the
    L2): 240 of the serving workload's ligands, 20 runs x 60 000 evaluations,
    all arriving at once, twice each."""
    from paper_2203_02096_gb300 import capi, serve, synth
    ctx = capi.Context(0)
    centers = [(12.5, -3.25, 7.0), (-30.0, 18.0, 4.0)]
    grids = [capi.grids_from_receptor(ctx, synth.make_receptor(3000, center=c, seed=11 + i), synth.make_box(96, center=c))
             for i, c in enumerate(centers)]
    ligs = _serving_ligands(240)
    server = capi.Server(ctx, capacity=1 << 16, max_atoms=128, pop_max=150)
    P = capi.default_params(pop_size=150, nruns=20, max_evals=60_000, ls_iters=100)
    serve.run(ctx, server, grids, [serve.Request(ligs[0], 0, seed=0)], P)
    out = []
    for rep in range(2):
        for name, gi in (("one receptor", lambda k: 0), ("two receptors, alternating", lambda k: k % 2)):
            reqs = [serve.Request(ligs[k], gi(k), seed=k, arrival=0.0) for k in range(len(ligs))]
            r = serve.run(ctx, server, grids, reqs, P)
            ev = sum(int(d.evals.sum()) for d in r.done)
            out.append({"case": name, "wall_s": r.wall, "evals_per_s": ev / r.wall})
    server.close()
    for g in grids:
        g.free()
    ctx.close()
    print(json.dumps({"workload": "240 serving requests x 20 runs x 60k evaluations, all at t = 0", "runs": out}),
          flush=True)
    return 0


def batched_docking(ctx, dev, n_ligs: int = 1024, nruns: int = 20, full_budget: int = 1_000_000,
                    probe_budget: int = 20_000, n_plain: int = 32, full: bool = True):
    """The batching workload: 1024 ligands with 10-108 atoms and 0-32
    torsions, 20 runs each, 80^3 x 9 maps, docked in one persistent launch
    (dock_batch), against the plain per-ligand form (dock, one launch
    sequence per ligand) on the same GPU.
    - packing: both packing modes (one largest-first launch; one launch per
      atom-count class) at the default and the autotuned launch shape, on
      the whole batch at probe_budget evaluations per run;
    - full budget (1M evaluations per run): the whole batch in one launch,
      and the plain form on n_plain ligands spread evenly over the size
      range, with the best energies of those ligands' runs in both forms
      (equal budget, same seeds): throughput and quality, not extrapolated."""
    import torch

    from paper_2203_02096_gb300 import autotune, capi, synth
    ligs = make_ligands(_batching_specs(n_ligs))
    box = synth.make_box(80)
    G = capi.grids_from_receptor(ctx, synth.make_receptor(3000, seed=4), box)
    L = [capi.ligand_from(ctx, l) for l in ligs]
    seeds = np.arange(n_ligs, dtype=np.uint64)
    P = capi.default_params(pop_size=150, nruns=nruns, max_evals=probe_budget, ls_iters=100)
    # warps per block and register cap of the persistent kernel by the autotuner (one-generation probes)
    tuner = autotune.Tuner(ctx, path=os.path.join(tempfile.mkdtemp(prefix="dock_tune_"), "tune.json"))
    tuned_warps = tuner.batch_warps(G, L, P, probe_generations=1)
    Pt = capi.DockParams.from_buffer_copy(P)
    Pt.batch_warps = tuned_warps
    tuned_blocks = tuner.batch_blocks(G, L, Pt, probe_generations=1)

    def timed_batch(params, blocks):
        capi.set_option(ctx, capi.OPT_BATCH_BLOCKS, blocks)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        out = capi.dock_batch(ctx, G, L, params, seeds)
        b.record()
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / 1e3, out

    capi.dock_batch(ctx, G, L[:8], Pt, seeds[:8])          # warm-up
    torch.cuda.synchronize(dev)
    packing = []
    for shape, warps, blocks in (("default", 4, 4), ("autotuned", tuned_warps, tuned_blocks)):
        for pack in (0, 1):
            Pp = capi.DockParams.from_buffer_copy(P)
            Pp.batch_warps, Pp.batch_pack = warps, pack
            t, out = timed_batch(Pp, blocks)
            packing.append({"shape": shape, "batch_warps": int(warps), "batch_blocks": int(blocks),
                            "pack": "by atom count" if pack else "one launch, largest first",
                            "seconds": t, "evals_per_s": float(out["evals"].sum().item()) / t})
    best = min(packing, key=lambda r: r["seconds"])
    res = {"workload": f"{n_ligs} ligands (10-108 atoms, 0-32 torsions), {nruns} runs, pop 150, 80^3 x 9 maps",
           "packing": {"budget_per_run": probe_budget, "runs": packing},
           "autotuned": {"batch_warps": int(tuned_warps), "batch_warps_ms": tuner.curve("|batch|"),
                         "batch_blocks": int(tuned_blocks), "batch_blocks_ms": tuner.curve("|batchregs|")}}
    if full:
        Pf = capi.DockParams.from_buffer_copy(P)
        Pf.max_evals = full_budget
        Pf.batch_warps = best["batch_warps"]
        Pf.batch_pack = 1 if best["pack"] == "by atom count" else 0
        t_batch, out = timed_batch(Pf, best["batch_blocks"])
        ev_batch = int(out["evals"].sum().item())
        bE = out["best_E"].cpu().numpy()
        # plain form: n_plain ligands spread over the size range, one docking at a time
        by_size = np.argsort([l.n_atoms for l in ligs], kind="stable")
        pick = by_size[np.linspace(0, n_ligs - 1, n_plain).round().astype(int)]
        # 128 threads per local-search chain: the autotuner's choice for the
        # 21-, 43- and 108-atom ligands of the tuning curves
        Pplain = capi.DockParams.from_buffer_copy(Pf)
        Pplain.ls_threads = 128
        Pw = capi.DockParams.from_buffer_copy(Pplain)
        Pw.max_evals = 20_000
        capi.dock(ctx, G, L[pick[0]], Pw, 0)           # untimed: loads the plain form's kernels
        torch.cuda.synchronize(dev)
        ev_plain, pE = 0, []
        t0 = time.perf_counter()
        for k in pick:
            _, e, ev = capi.dock(ctx, G, L[k], Pplain, int(seeds[k]))
            ev_plain += int(ev.sum())
            pE.append(e)
        torch.cuda.synchronize(dev)
        t_plain = time.perf_counter() - t0
        pE = np.array(pE)
        t_batch_pick = t_batch * ev_plain / ev_batch   # the batch's time share of those ligands' evaluations
        res["full_budget"] = {
            "budget_per_run": full_budget, "shape": {k: best[k] for k in ("batch_warps", "batch_blocks", "pack")},
            "batch_seconds": t_batch, "batched_evals_per_s": ev_batch / t_batch,
            "batched_ligands_per_hour": 3600.0 * n_ligs / t_batch,
            "plain_ligands": int(n_plain), "plain_seconds": t_plain, "plain_evals_per_s": ev_plain / t_plain,
            "plain_ligands_per_hour": 3600.0 * n_plain / t_plain,
            "speedup_evals_per_s": (ev_batch / t_batch) / (ev_plain / t_plain),
            "best_E_median": {"batched": float(np.median(bE[pick])), "plain": float(np.median(pE))},
            "best_E_median_all_1024": float(np.median(bE)),
            "per_ligand_median_diff": float(np.median(np.median(bE[pick], axis=1) - np.median(pE, axis=1))),
            "plain_ls_threads": 128,
            "note": f"plain form timed on {n_plain} of the ligands (every {n_ligs // n_plain}th by atom count); "
                    f"equal budget and seeds in both forms; batched time share of those ligands ~{t_batch_pick:.1f} s"}
    for h in L + [G]:
        h.free()
    capi.set_option(ctx, capi.OPT_BATCH_BLOCKS, 4)
    return res


def serving_sweep(ctx, dev, full_budget: int = 500_000, full_rates=((10, 30.0), (30, 8.0)),
                  probe_rates=(10, 30, 100, 300, 1000), probe_budget: int = 5_000, probe_seconds: float = 2.0,
                  nruns: int = 20, n_plain: int = 16, full: bool = True, light_seconds: float = 8.0):
    """The serving workload: Poisson arrivals of ligands with 10-128 atoms
    (log-uniform) and 0-32 torsions against two receptors with 96^3 x 9
    maps, 20 runs per request, through the continuous-batching server
    (server_* + serve.run).
    - full budget (500k evaluations per run): arrival rates 10 and 30 per
      second for the stated seconds of arrivals; p50/p99 latency (arrival to
      all runs done), throughput, ligands/hour, and whether the rate is past
      saturation (served rate while requests still arrive below 80% of the
      arrival rate); the plain
      form (one dock() per request, in order) on the first n_plain requests
      of the rate-10 stream, with the best energies of the same requests in
      both forms; light load (2 per second for light_seconds) served only
      and with serve.run's idle_plain route;
    - the knee at a reduced budget: every probe rate for probe_seconds."""
    import torch

    from paper_2203_02096_gb300 import capi, serve, synth
    centers = [(12.5, -3.25, 7.0), (-30.0, 18.0, 4.0)]
    grids = [capi.grids_from_receptor(ctx, synth.make_receptor(3000, center=c, seed=11 + i), synth.make_box(96, center=c))
             for i, c in enumerate(centers)]
    server = capi.Server(ctx, capacity=1 << 16, max_atoms=128, pop_max=150)
    # request k of every stream: the same ligand (sizes from one seeded draw)
    n_req = max([max(8, int(r * t)) for r, t in full_rates] + [max(8, int(r * probe_seconds)) for r in probe_rates])
    req_ligs = _serving_ligands(n_req)

    def stream(rate, seconds, budget, seed):
        n = max(8, int(rate * seconds))
        reqs = [serve.Request(req_ligs[k], k % 2, seed=k) for k in range(n)]
        for r, t in zip(reqs, serve.poisson_arrivals(n, rate, seed=seed)):
            r.arrival = float(t)
        return reqs

    res = {"workload": "ligands 10-128 atoms (log-uniform), 0-32 torsions, 20 runs, 2 receptors x 96^3 x 9 maps"}
    # warm-up: one request through the server
    Pw = capi.default_params(pop_size=150, nruns=nruns, max_evals=probe_budget, ls_iters=100)
    serve.run(ctx, server, grids, stream(10, 0.1, probe_budget, 0)[:1], Pw)
    if full:
        P = capi.default_params(pop_size=150, nruns=nruns, max_evals=full_budget, ls_iters=100)
        sweep, first = [], None
        for rate, seconds in full_rates:
            reqs = stream(rate, seconds, full_budget, int(rate))
            rep = serve.run(ctx, server, grids, reqs, P, timeout=900.0)
            sm = rep.summary()
            st = sm["steady_throughput_per_s"]
            sm["saturated"] = None if st is None else bool(st < 0.8 * rate)
            sweep.append(dict(rate_per_s=rate, arrival_seconds=seconds, **sm))
            if first is None:
                first = {d.request.seed: d for d in rep.done}
                first_reqs = reqs
        # plain form on the first requests of the first stream (one untimed
        # docking first: the plain form's first call loads its kernels)
        r0 = first_reqs[0]
        L0 = capi.ligand_from(ctx, r0.ligand)
        capi.dock(ctx, grids[r0.grid_index], L0, P, r0.seed)
        L0.free()
        lat, pE, sE = [], [], []
        t0 = time.perf_counter()
        for r in first_reqs[:n_plain]:
            ts = time.perf_counter()
            Lr = capi.ligand_from(ctx, r.ligand)
            _, e, _ = capi.dock(ctx, grids[r.grid_index], Lr, P, r.seed)
            Lr.free()
            lat.append(time.perf_counter() - ts)
            pE.append(e)
            sE.append(first[r.seed].best_E)
        t_plain = time.perf_counter() - t0
        # light load: 2 requests/s, served only and with the plain route for
        # requests that find the GPU idle (the library's team width; the
        # plain form's kernels are loaded by the dockings above)
        light = {}
        for mode, idle in (("served_only", False), ("idle_plain", True)):
            rep = serve.run(ctx, server, grids, stream(2, light_seconds, full_budget, 2), P, timeout=900.0,
                            idle_plain=idle)
            light[mode] = rep.summary()
        res["full_budget"] = {
            "budget_per_run": full_budget, "sweep": sweep,
            "plain": {"requests": n_plain, "requests_per_s": n_plain / t_plain,
                      "ligands_per_hour": 3600.0 * n_plain / t_plain, "latency_s_median": float(np.median(lat))},
            "best_E_median_same_requests": {"served": float(np.median(sE)), "plain": float(np.median(pE))},
            "light_load": {"rate_per_s": 2, "arrival_seconds": light_seconds, **light}}
    # the knee at a reduced budget
    Pp = capi.default_params(pop_size=150, nruns=nruns, max_evals=probe_budget, ls_iters=100)
    knee = []
    for rate in probe_rates:
        rep = serve.run(ctx, server, grids, stream(rate, probe_seconds, probe_budget, int(rate) + 1), Pp)
        sm = rep.summary()
        st = sm["steady_throughput_per_s"]
        sm["saturated"] = None if st is None else bool(st < 0.8 * rate)
        knee.append(dict(rate_per_s=rate, **sm))
    res["reduced_budget"] = {"budget_per_run": probe_budget, "arrival_seconds": probe_seconds, "sweep": knee}
    server.close()
    for g in grids:
        g.free()
    torch.cuda.synchronize(dev)
    return res


def tuning_curves(ctx, G, w, tuner, P_head):
    """The paper's tuning study (Section V-B: threads per block) on GB300:
    device time of the drug-size workload's local-search launch (50 runs x 9
    chains, 50 ADADELTA iterations) at 32..256 threads per chain, for ligands
    of the paper's three sizes (21/2, 43/15, 108/31 atoms/torsions, synthetic
    stand-ins), and the width the autotuner chose for the headline."""
    from paper_2203_02096_gb300 import autotune, capi, synth
    out = {}
    for name, (na, nt) in {"21 atoms / 2 torsions": (21, 2), "43 atoms / 15 torsions": (43, 15),
                           "108 atoms / 31 torsions": (108, 31)}.items():
        lig = capi.ligand_from(ctx, synth.make_ligand(na, nt, seed=77))
        P = capi.default_params(pop_size=w.pop_size, nruns=w.nruns, max_evals=w.max_evals, ls_iters=w.ls_iters)
        out[name] = {str(k): v for k, v in autotune.ls_curve(ctx, G, lig, P).items()}
        lig.free()
    return {"ls_threads_curve": out, "headline_ls_threads": int(P_head.ls_threads),
            "headline_tuning_ms": tuner.curve("|ls|")}


def graph_vs_direct(ctx, G, L, P_head, dev, reps: int = 3):
    """The plain docking replayed as a CUDA graph against direct launches.
    dock_async_noalloc (no allocation, no host synchronisation) is captured
    once per workload and replayed; both forms run the same seed, so they do
    the same work.  Milliseconds per docking (CUDA events, no L2 flush), for
    the drug-size workload and the small-ligand one (shorter kernels, where
    the gaps between launches weigh more)."""
    import torch

    from paper_2203_02096_gb300 import capi, synth

    def outputs(R, Gn):
        return dict(best_geno=torch.empty((R, Gn), dtype=torch.float32, device=dev),
                    best_E32=torch.empty(R, dtype=torch.float32, device=dev),
                    best_E=torch.empty(R, dtype=torch.float64, device=dev),
                    evals=torch.empty(R, dtype=torch.int64, device=dev))

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / reps

    def one(Gr, Lg, P):
        out = outputs(P.nruns, Lg.n_genes)
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            capi.dock_async_noalloc(ctx, Gr, Lg, P, 123, out)
        torch.cuda.current_stream(dev).wait_stream(side)
        torch.cuda.synchronize(dev)
        n0 = ctx.launch_count()
        direct = timed(lambda: capi.dock_async_noalloc(ctx, Gr, Lg, P, 123, out))
        launches = (ctx.launch_count() - n0) // reps
        ref = {k: v.clone() for k, v in out.items()}
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            capi.dock_async_noalloc(ctx, Gr, Lg, P, 123, out)
        graph.replay()
        torch.cuda.synchronize(dev)
        same = all(torch.equal(out[k], ref[k]) for k in ref)
        replay = timed(graph.replay)
        del graph
        return {"direct_ms": direct, "graph_ms": replay, "launches_per_docking": int(launches),
                "graph_same_results": bool(same)}

    res = {"note": "same seed in both forms; no L2 flush; ms per docking"}
    res["drug_size"] = one(G, L, P_head)
    w1 = synth.small_ligand_workload()
    G1 = capi.grids_from_receptor(ctx, w1.receptor, w1.box)
    L1 = capi.ligand_from(ctx, w1.ligand)
    P1 = capi.default_params(pop_size=w1.pop_size, nruns=w1.nruns, max_evals=w1.max_evals, ls_iters=w1.ls_iters)
    capi.dock(ctx, G1, L1, P1, 0)       # loads the kernels at this ligand's shapes
    res["small_ligand"] = one(G1, L1, P1)
    L1.free()
    G1.free()
    return res


def solis_wets_vs_adadelta(ctx, G, L, w, dev, ada_out, ada_value):
    """The paper's own local search (Solis-Wets, energies only) against
    ADADELTA (score+gradient) on the same drug-size docking at the same
    evaluation budget: evaluations/s and the best energies reached (FP64
    re-scores of each run's best pose), one timed docking after one warm-up."""
    import torch

    from paper_2203_02096_gb300 import capi
    P = capi.default_params(pop_size=w.pop_size, nruns=w.nruns, max_evals=w.max_evals, ls_iters=w.ls_iters,
                            ls_method=1)
    stream = torch.cuda.current_stream(dev)
    out = capi.dock_async(ctx, G, L, P, w.seed + 7)
    torch.cuda.synchronize(dev)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    out = capi.dock_async(ctx, G, L, P, w.seed + 8, out=out)
    t1.record(stream)
    torch.cuda.synchronize(dev)
    s = t0.elapsed_time(t1) / 1e3
    sw_E = out["best_E"].cpu().numpy()
    ada_E = ada_out["best_E"].cpu().numpy()
    return {"workload": "drug-size ligand, 50 runs x 2.5M evaluations, pop 150, local search on 6% "
                        "(ADADELTA 300 iterations / Solis-Wets at most 300 iterations)",
            "solis_wets_evals_per_s": float(out["evals"].sum().item()) / s, "solis_wets_seconds": s,
            "adadelta_evals_per_s": ada_value,
            "best_E_median": {"solis_wets": float(np.median(sw_E)), "adadelta": float(np.median(ada_E))},
            "best_E_min": {"solis_wets": float(sw_E.min()), "adadelta": float(ada_E.min())}}


def pair_list(lig):
    """Pairs of the ligand's intramolecular list (different rigid fragments,
    >= 4 bonds apart), from the bond graph -- used to count how many pairs of
    the docked poses fall inside the cutoff."""
    n = lig.n_atoms
    adj = [[] for _ in range(n)]
    for (a, b), r in zip(lig.bonds, lig.rotatable):
        adj[a].append((b, r))
        adj[b].append((a, r))
    frag = -np.ones(n, int)
    for s in range(n):
        if frag[s] >= 0:
            continue
        stack = [s]
        frag[s] = s
        while stack:
            a = stack.pop()
            for b, r in adj[a]:
                if not r and frag[b] < 0:
                    frag[b] = s
                    stack.append(b)
    out = []
    for s in range(n):
        dist = -np.ones(n, int)
        dist[s] = 0
        q = [s]
        for a in q:
            for b, _ in adj[a]:
                if dist[b] < 0:
                    dist[b] = dist[a] + 1
                    q.append(b)
        out += [(s, t) for t in range(s + 1, n) if frag[s] != frag[t] and dist[t] >= 4]
    return np.asarray(out, dtype=int).reshape(-1, 2)


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one ls_kernel
# launch on the drug-size workload, from one ncu capture (cold caches), and a
# digest of the kernel sources and input generator it was taken on: the figure
# is reported only while they are unchanged.
LS_TRAFFIC_BYTES = 31.04e6
LS_TRAFFIC_SOURCES = "1b8015fede9db610"


# the files that define the local-search kernel and the ligand it runs on
LS_SOURCES = ("csrc/eval.cuh", "csrc/ga.cuh", "csrc/search.cu", "csrc/internal.h", "csrc/forcefield.h",
              "csrc/host.cpp", "synth.py")


def sources_digest() -> str:
    import hashlib
    pkg = os.path.join(ROOT, "paper_2203_02096_gb300")
    h = hashlib.sha256()
    for rel in LS_SOURCES:
        h.update(os.path.basename(rel).encode())
        with open(os.path.join(pkg, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def peak_fp32_tflops() -> float:
    mhz = 2070.0
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        mhz = float(mp.get("sm_max_mhz", mhz))
    except (OSError, ValueError):
        pass
    return 152 * 128 * 2 * mhz * 1e6 / 1e12


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the side measurements")
    ap.add_argument("--quick", action="store_true",
                    help="side measurements without the full-budget batching and serving runs")
    ap.add_argument("--ls-threads", type=int, default=-1,
                    help="threads per local-search chain (-1 = autotuned, 0 = library default)")
    ap.add_argument("--only", choices=["score_grad", "batch_small", "batch_96", "serve_l2"], default=None,
                    help="run one side measurement alone and print its JSON (for profiling)")
    ap.add_argument("--score-blocks", type=int, default=0, choices=[0, 1, 6, 8],
                    help="with --only score_grad: fixed register cap of the scorer (0 = autotuned)")
    args = ap.parse_args(argv)
    if args.only == "score_grad":
        return run_score_grad_only(args.score_blocks)
    if args.only == "batch_small":
        return run_batch_small()
    if args.only == "batch_96":
        return run_batch_96()
    if args.only == "serve_l2":
        return run_serve_l2()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run(args)


if __name__ == "__main__":
    sys.exit(main())
