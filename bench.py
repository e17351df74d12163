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
    _, _, evals = oracle.dock(lig, grid, P, seed, nthreads=cores)
    dt = time.perf_counter() - t0
    desc = (f"{cores} docking runs x {int(evals[0])} evaluations of the drug-size workload (50 runs x 2.5M "
            f"in full), FP64 oracle, one run per thread")
    return float(evals.sum() / dt), cores, desc, dt


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

    batch = score_grad_throughput(ctx, G, w.box, dev) if not args.no_batch else None
    multi = batched_docking(ctx, dev) if not args.no_batch else None
    serving = serving_sweep(ctx, dev) if not args.no_batch else None
    solis = solis_wets_vs_adadelta(ctx, G, L, w, dev, out, value) if not args.no_batch else None
    tuning = tuning_curves(ctx, G, w, tuner, P) if not args.no_batch else None

    cpu = None
    if rank == 0 and not args.no_cpu:
        v, cores, desc, _ = cpu_sample(w, args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}

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
            "score_grad_batch": batch,
            "batched_docking": multi,
            "serving": serving,
            "solis_wets": solis,
            "tuning": tuning,
            "best_energy_median": float(np.median(out["best_E"].cpu().numpy())),
        }
        print(json.dumps(line), flush=True)
    for h in (L, G):
        h.free()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def score_grad_throughput(ctx, G, box, dev, reps: int = 5):
    """score_grad_batch over 65536 random genotypes of a 64-atom / 16-torsion
    ligand in the same grids (the differentiation workload): evals/s and the
    FP32 roofline of that kernel (inputs resident, L2 flushed between calls)."""
    import torch

    from paper_2203_02096_gb300 import autotune, capi, synth
    lig = synth.make_ligand(64, 16, seed=0)
    L = capi.ligand_from(ctx, lig)
    # register cap of the scorer by the autotuner (untimed)
    tuner = autotune.Tuner(ctx, path=os.path.join(tempfile.mkdtemp(prefix="dock_tune_"), "tune.json"))
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
            "autotuned_score_blocks": blocks, "score_blocks_ms": tuner.curve("|score|")}


def run_score_grad_only() -> int:
    """The score_grad_batch measurement alone (drug-size grids built on the GPU)."""
    import torch

    from paper_2203_02096_gb300 import capi
    dev = torch.device("cuda", 0)
    w = workload()
    ctx = capi.Context(0)
    G = capi.grids_from_receptor(ctx, w.receptor, w.box)
    print(json.dumps(score_grad_throughput(ctx, G, w.box, dev)), flush=True)
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


def batched_docking(ctx, dev, n_ligs: int = 1024, nruns: int = 20, evals_per_run: int = 20_000,
                    full_budget: int = 1_000_000, n_plain: int = 12):
    """Many-ligand docking in one persistent launch (dock_batch) against the
    plain per-ligand form (dock, one launch sequence per ligand): 1024
    ligands with 10-108 atoms and 0-32 torsions, 20 runs each, 80^3 x 9 maps.
    Both run each docking run with a reduced budget; ligands/hour at the full
    1M-evaluation budget is extrapolated from evals/s (the cost per
    evaluation does not depend on the budget)."""
    import torch

    from paper_2203_02096_gb300 import autotune, capi, synth
    rng = np.random.default_rng(3)
    ligs = [synth.make_ligand(int(rng.integers(10, 109)), int(rng.integers(0, 33)), seed=5000 + k)
            for k in range(n_ligs)]
    box = synth.make_box(80)
    G = capi.grids_from_receptor(ctx, synth.make_receptor(3000, seed=4), box)
    L = [capi.ligand_from(ctx, l) for l in ligs]
    P = capi.default_params(pop_size=150, nruns=nruns, max_evals=evals_per_run, ls_iters=100)
    seeds = np.arange(n_ligs, dtype=np.uint64)
    # warps per block of the persistent kernel by the autotuner (one-generation probes)
    tuner = autotune.Tuner(ctx, path=os.path.join(tempfile.mkdtemp(prefix="dock_tune_"), "tune.json"))
    Pb = capi.DockParams.from_buffer_copy(P)
    Pb.batch_warps = tuner.batch_warps(G, L, P, probe_generations=1)
    batch_blocks = tuner.batch_blocks(G, L, Pb, probe_generations=1)   # register cap, set on the context
    capi.dock_batch(ctx, G, L[:8], Pb, seeds[:8])          # warm-up
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    out = capi.dock_batch(ctx, G, L, Pb, seeds)
    b.record()
    torch.cuda.synchronize(dev)
    t_batch = a.elapsed_time(b) / 1e3
    ev_batch = int(out["evals"].sum().item())
    # plain form on a sample of the same ligands, one docking at a time
    ev_plain = 0
    plain_params = [tuner.tuned(G, L[k], P) for k in range(n_plain)]   # threads per chain, per ligand
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for k in range(n_plain):
        _, _, ev = capi.dock(ctx, G, L[k], plain_params[k], int(seeds[k]))
        ev_plain += int(ev.sum())
    torch.cuda.synchronize(dev)
    t_plain = time.perf_counter() - t0
    for h in L + [G]:
        h.free()
    capi.set_option(ctx, capi.OPT_BATCH_BLOCKS, 4)
    rate_b, rate_p = ev_batch / t_batch, ev_plain / t_plain
    per_lig_full = nruns * full_budget
    return {"workload": f"{n_ligs} ligands (10-108 atoms, 0-32 torsions), {nruns} runs, pop 150, 80^3 x 9 maps",
            "sample": f"{evals_per_run} evaluations per run (full budget {full_budget}); plain form timed on "
                      f"{n_plain} of the ligands",
            "batched_evals_per_s": rate_b, "plain_evals_per_s": rate_p, "speedup": rate_b / rate_p,
            "batched_ligands_per_hour_extrapolated": 3600.0 * rate_b / per_lig_full,
            "plain_ligands_per_hour_extrapolated": 3600.0 * rate_p / per_lig_full,
            "batch_seconds": t_batch, "launches": 1,
            "autotuned": {"batch_warps": int(Pb.batch_warps), "batch_warps_ms": tuner.curve("|batch|"),
                          "batch_blocks": int(batch_blocks), "batch_blocks_ms": tuner.curve("|batchregs|"),
                          "plain_ls_threads": [int(p.ls_threads) for p in plain_params]}}


def serving_sweep(ctx, dev, rates=(10, 30, 100, 300, 1000), seconds: float = 2.0, nruns: int = 20,
                  evals_per_run: int = 5_000, full_budget: int = 500_000, n_plain: int = 8):
    """Continuous-batching service (server_* + serve.run): Poisson arrivals
    of ligands with 10-128 atoms (log-uniform) and 0-32 torsions against two
    receptors with 96^3 x 9 maps, 20 runs per request; p50/p99 latency and
    throughput per arrival rate, beside the plain form (one dock() call per
    request, in arrival order).  Each run gets evals_per_run evaluations
    (full budget 500k: latencies scale with it, the ordering does not)."""
    import torch

    from paper_2203_02096_gb300 import capi, serve, synth
    centers = [(12.5, -3.25, 7.0), (-30.0, 18.0, 4.0)]
    grids = [capi.grids_from_receptor(ctx, synth.make_receptor(3000, center=c, seed=11 + i), synth.make_box(96, center=c))
             for i, c in enumerate(centers)]
    P = capi.default_params(pop_size=150, nruns=nruns, max_evals=evals_per_run, ls_iters=100)
    server = capi.Server(ctx, capacity=1 << 16, max_atoms=128, pop_max=150)
    rng = np.random.default_rng(17)

    def request(k):
        n = int(np.exp(rng.uniform(np.log(10), np.log(128.999))))
        return serve.Request(synth.make_ligand(n, int(rng.integers(0, 33)), seed=9000 + k), k % 2, seed=k)

    # warm-up: one request through the server
    serve.run(ctx, server, grids, [request(0)], P)
    out = []
    for rate in rates:
        n = max(8, int(rate * seconds))
        reqs = [request(k) for k in range(n)]
        for r, t in zip(reqs, serve.poisson_arrivals(n, rate, seed=int(rate))):
            r.arrival = float(t)
        rep = serve.run(ctx, server, grids, reqs, P)
        out.append(dict(rate_per_s=rate, **rep.summary()))
    # the plain form: one docking at a time
    reqs = [request(k) for k in range(n_plain)]
    t0 = time.perf_counter()
    lat = []
    for r in reqs:
        ts = time.perf_counter()
        L = capi.ligand_from(ctx, r.ligand)
        capi.dock(ctx, grids[r.grid_index], L, P, r.seed)
        L.free()
        lat.append(time.perf_counter() - ts)
    t_plain = time.perf_counter() - t0
    server.close()
    for g in grids:
        g.free()
    torch.cuda.synchronize(dev)
    return {"workload": "ligands 10-128 atoms (log-uniform), 0-32 torsions, 20 runs, 2 receptors x 96^3 x 9 maps",
            "sample": f"{evals_per_run} evaluations per run (full budget {full_budget}); {seconds} s of arrivals per rate",
            "sweep": out,
            "plain": {"requests_per_s": n_plain / t_plain, "ligands_per_hour": 3600.0 * n_plain / t_plain,
                      "latency_s_median": float(np.median(lat))}}


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
LS_TRAFFIC_SOURCES = "34859c32270eda0e"


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
    ap.add_argument("--no-batch", action="store_true", help="skip the score_grad_batch side measurement")
    ap.add_argument("--ls-threads", type=int, default=-1,
                    help="threads per local-search chain (-1 = autotuned, 0 = library default)")
    ap.add_argument("--only", choices=["score_grad", "batch_small"], default=None,
                    help="run one side measurement alone and print its JSON (for profiling)")
    args = ap.parse_args(argv)
    if args.only == "score_grad":
        return run_score_grad_only()
    if args.only == "batch_small":
        return run_batch_small()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run(args)


if __name__ == "__main__":
    sys.exit(main())
