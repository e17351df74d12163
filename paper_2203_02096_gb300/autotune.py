"""Autotuner for the docking kernels' launch shapes.

The paper tunes threads per block and register use per GPU (Section V-B);
here the knobs are the threads that evaluate one local-search chain of a
docking (``dock_params.ls_threads``: 32..256, one to eight warps per chain),
the warps per block of the persistent batch kernel
(``dock_params.batch_warps``) and the register cap of the batched scorers
(context option ``DOCK_OPT_SCORE_BLOCKS``: 1, 6 or 8 blocks per SM) and
of the persistent docking kernel (``DOCK_OPT_BATCH_BLOCKS``: 4 or 3).  The tuner times every candidate on the
device through ``dock_tune`` (CUDA events inside the library, one untimed
launch first), keeps the fastest, and caches the choice in a JSON file keyed
by device name and workload shape, so a shape is timed once per machine.

Choices and reproducibility: the batch kernel's warps per block never change
a result.  The local-search team width does change the last bits of a
docking (the team's reductions run in a different fixed order), so a tuned
docking is reproducible for a given cache entry; pass ``ls_threads``
explicitly to pin it.
"""
from __future__ import annotations

import json
import os
import threading

from . import capi

LS_CANDIDATES = (32, 64, 128, 256)
BATCH_CANDIDATES = (1, 2, 4)
SCORE_BLOCK_CANDIDATES = (1, 6, 8)
BATCH_BLOCK_CANDIDATES = (4, 3)
LS_PROBE_ITERS = 50          # dock_tune times at most this many iterations per chain


def default_cache_path() -> str:
    base = os.environ.get("DOCK_TUNE_CACHE")
    if base:
        return base
    return os.path.join(os.path.expanduser("~"), ".cache", "gb300_dock", "tune.json")


class Tuner:
    """Times candidate launch shapes and remembers the fastest per shape."""

    def __init__(self, ctx: capi.Context, path: str | None = None, reps: int = 3):
        import torch
        self.ctx = ctx
        self.path = path or default_cache_path()
        self.reps = reps
        self.device_name = torch.cuda.get_device_name(ctx.device)
        self._lock = threading.Lock()
        self.entries: dict = {}
        if os.path.exists(self.path):
            with open(self.path) as f:
                self.entries = json.load(f)

    def _save(self):
        os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
        tmp = f"{self.path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(self.entries, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    def _pick(self, key: str, cand, measure) -> int:
        with self._lock:
            hit = self.entries.get(key)
            if hit is not None:
                return int(hit["choice"])
            ms = measure(cand)
            ok = [(m, c) for m, c in zip(ms, cand) if m > 0]
            if not ok:
                raise RuntimeError(f"autotune: no candidate of {list(cand)} fits ({key})")
            choice = min(ok)[1]
            self.entries[key] = {"choice": int(choice), "ms": {str(c): float(m) for c, m in zip(cand, ms)}}
            self._save()
            return int(choice)

    def ls_threads(self, grids: capi.Grids, lig: capi.Ligand, params: capi.DockParams) -> int:
        """Threads per local-search chain for dock() of this ligand at these
        parameters (chain count nruns * ls_count)."""
        n_ls = params.ls_count if params.ls_count >= 0 else (6 * params.pop_size + 99) // 100
        key = "|".join(str(v) for v in (self.device_name, "ls", params.ls_method, lig.n_atoms, lig.n_torsions,
                                         lig.n_pairs, params.nruns * n_ls, min(params.ls_iters, LS_PROBE_ITERS)))
        return self._pick(key, LS_CANDIDATES, lambda c: capi.dock_tune(self.ctx, grids, [lig], params,
                                                                       capi.TUNE_LS_THREADS, c, self.reps))

    def batch_warps(self, grids: capi.Grids, ligs, params: capi.DockParams, probe_generations: int = 2) -> int:
        """Warps per block of dock_batch for this set of ligands, timed on a
        budget of a few generations."""
        sizes = sorted(l.n_atoms for l in ligs)
        key = "|".join(str(v) for v in (self.device_name, "batch", params.ls_method, params.pop_size, len(ligs),
                                         params.nruns, sizes[0], sizes[len(sizes) // 2], sizes[-1]))
        probe = capi.DockParams.from_buffer_copy(params)
        n_ls = params.ls_count if params.ls_count >= 0 else (6 * params.pop_size + 99) // 100
        probe.max_evals = params.pop_size + probe_generations * ((params.pop_size - 1) + n_ls * params.ls_iters)
        return self._pick(key, BATCH_CANDIDATES, lambda c: capi.dock_tune(self.ctx, grids, ligs, probe,
                                                                          capi.TUNE_BATCH_WARPS, c, 1))

    def batch_blocks(self, grids: capi.Grids, ligs, params: capi.DockParams, probe_generations: int = 2,
                     apply: bool = True) -> int:
        """Register cap of the persistent docking kernel for this ligand set
        (timed like batch_warps); set on the context."""
        sizes = sorted(l.n_atoms for l in ligs)
        key = "|".join(str(v) for v in (self.device_name, "batchregs", params.ls_method, params.pop_size, len(ligs),
                                         params.nruns, params.batch_warps, sizes[0], sizes[len(sizes) // 2],
                                         sizes[-1]))
        probe = capi.DockParams.from_buffer_copy(params)
        n_ls = params.ls_count if params.ls_count >= 0 else (6 * params.pop_size + 99) // 100
        probe.max_evals = params.pop_size + probe_generations * ((params.pop_size - 1) + n_ls * params.ls_iters)
        choice = self._pick(key, BATCH_BLOCK_CANDIDATES, lambda c: capi.dock_tune(self.ctx, grids, ligs, probe,
                                                                                  capi.TUNE_BATCH_BLOCKS, c, 1))
        if apply:
            capi.set_option(self.ctx, capi.OPT_BATCH_BLOCKS, choice)
        return choice

    def score_blocks(self, grids: capi.Grids, lig: capi.Ligand, batch: int = 65536, apply: bool = True) -> int:
        """Register cap of score_batch / score_grad_batch for this ligand,
        timed on a batch of about `batch` genotypes; set on the context."""
        key = "|".join(str(v) for v in (self.device_name, "score", lig.n_atoms, lig.n_torsions, lig.n_pairs, batch))
        probe = capi.default_params(pop_size=1024, nruns=max(1, batch // 1024))
        choice = self._pick(key, SCORE_BLOCK_CANDIDATES,
                            lambda c: capi.dock_tune(self.ctx, grids, [lig], probe, capi.TUNE_SCORE_BLOCKS, c, self.reps))
        if apply:
            capi.set_option(self.ctx, capi.OPT_SCORE_BLOCKS, choice)
        return choice

    def tuned(self, grids: capi.Grids, ligs, params: capi.DockParams) -> capi.DockParams:
        """A copy of params with ls_threads (one ligand) or batch_warps (a list) chosen."""
        p = capi.DockParams.from_buffer_copy(params)
        if isinstance(ligs, (list, tuple)):
            p.batch_warps = self.batch_warps(grids, ligs, params)
        else:
            p.ls_threads = self.ls_threads(grids, ligs, params)
        return p

    def curve(self, key_part: str) -> dict:
        """Cached timings whose key contains key_part (for reports)."""
        return {k: v for k, v in self.entries.items() if key_part in k}


def ls_curve(ctx, grids, lig, params, reps: int = 3) -> dict:
    """Milliseconds per local-search launch and evaluations/s per candidate
    width (the tuning curve itself, not cached)."""
    ms = capi.dock_tune(ctx, grids, [lig], params, capi.TUNE_LS_THREADS, LS_CANDIDATES, reps)
    n_ls = params.ls_count if params.ls_count >= 0 else (6 * params.pop_size + 99) // 100
    evals = params.nruns * n_ls * min(params.ls_iters, LS_PROBE_ITERS)
    return {int(c): {"ms": float(m), "evals_per_s": (evals / (m / 1e3)) if m > 0 else None}
            for c, m in zip(LS_CANDIDATES, ms)}


__all__ = ["Tuner", "ls_curve", "default_cache_path", "LS_CANDIDATES", "BATCH_CANDIDATES", "SCORE_BLOCK_CANDIDATES",
           "BATCH_BLOCK_CANDIDATES"]
