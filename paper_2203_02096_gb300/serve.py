"""Request loop of the docking service: continuous batching over server_*.

Requests (a ligand, a receptor's grids, a seed) arrive over time; each is
admitted as soon as the device memory it needs -- its ligand data and its
result rows -- fits the budget and the server has free task slots, and is
then submitted to the running persistent kernel, where its runs share the
GPU with whatever else is in flight.  Completed requests release their
memory at once.  Reports per-request latency (arrival to all runs done)
and throughput.

With ``idle_plain``, requests that arrive while nothing is served in
flight and the queue is short are docked one at a time in the plain form
instead: a request's local searches spread over the whole GPU, so it ends
in a fraction of a second rather than after one warp's sequential run.
Under load everything goes to the persistent kernel, which has the higher
throughput; the two never share the GPU (server submissions wait for a
running plain docking, which is short).  ``plain_threads`` sets the plain
dockings' local-search team width: 0 (the library's choice, several warps
per chain) is the fastest and runs the same search with a different FP32
summation order, so its results differ from the served ones at rounding
level; 32 (one warp per chain, as in the persistent kernel) gives the
served results bit for bit, at several times the plain latency.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import capi

ROW_BYTES = 4 * capi.GENE_STRIDE + 4 + 8 + 8   # result row of one run on the device


@dataclass
class Request:
    ligand: object          # synth.Ligand
    grid_index: int
    seed: int
    arrival: float = 0.0    # seconds from the start of the run


@dataclass
class Done:
    request: Request
    latency: float
    best_geno: np.ndarray
    best_E: np.ndarray
    evals: np.ndarray
    route: str = "served"   # "served" (persistent kernel) or "plain" (idle GPU)


class PlainDocking:
    """One request docked in the plain form on its own stream (queued,
    device outputs), with its completion event."""

    def __init__(self, ctx, grids, lig, params, seed):
        import torch
        self.stream = torch.cuda.Stream(torch.device("cuda", ctx.device))
        self.stream.wait_stream(torch.cuda.current_stream(self.stream.device))
        self.out = capi.dock_async(ctx, grids, lig, params, seed, stream=self.stream)
        self.event = torch.cuda.Event()
        self.event.record(self.stream)

    def done(self) -> bool:
        return self.event.query()

    def result(self):
        self.event.synchronize()
        return (self.out["best_geno"].cpu().numpy(), self.out["best_E"].cpu().numpy(),
                self.out["evals"].cpu().numpy())


def plain_params(params: capi.DockParams, threads: int = 32) -> capi.DockParams:
    """The plain-form parameters with local-search teams of `threads`
    threads; 32 (one warp per chain, like the persistent kernel) makes the
    results equal the served ones bit for bit."""
    p = capi.DockParams.from_buffer_copy(params)
    p.ls_threads = threads
    return p


@dataclass
class ServiceReport:
    done: list = field(default_factory=list)
    wall: float = 0.0
    max_in_flight: int = 0

    def latencies(self) -> np.ndarray:
        return np.array([d.latency for d in self.done])

    def steady_throughput(self):
        """Completions per second while requests were still arriving (from
        the first completion to the last arrival), or None when that window
        is under a second: the served rate without the ramp-up and drain of
        a finite stream."""
        if not self.done:
            return None
        finish = np.sort([d.request.arrival + d.latency for d in self.done])
        last_arrival = max(d.request.arrival for d in self.done)
        t1 = finish[0]
        if last_arrival - t1 < 1.0:
            return None
        n = int(np.searchsorted(finish, last_arrival, side="right")) - 1
        return n / (last_arrival - t1)

    def summary(self) -> dict:
        lat = self.latencies()
        return {"requests": len(self.done), "plain_route": sum(d.route == "plain" for d in self.done),
                "wall_s": self.wall,
                "throughput_per_s": len(self.done) / self.wall if self.wall > 0 else 0.0,
                "steady_throughput_per_s": self.steady_throughput(),
                "ligands_per_hour": 3600.0 * len(self.done) / self.wall if self.wall > 0 else 0.0,
                "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
                "p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
                "max_in_flight": self.max_in_flight}


def poisson_arrivals(n: int, rate: float, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def run(ctx: capi.Context, server: capi.Server, grids: list, requests: list, params: capi.DockParams,
        mem_budget: int = 2 << 30, poll_sleep: float = 2e-3, timeout: float = 600.0,
        idle_plain: bool = False, plain_queue: int = 4, plain_threads: int = 0) -> ServiceReport:
    """Serve ``requests`` (their ``arrival`` times set) until all are done.
    idle_plain: while nothing is in flight on the persistent kernel and at
    most plain_queue requests wait, requests are docked one at a time in
    the plain form with plain_threads threads per local-search chain
    (module docstring); past that every waiting request goes to the
    persistent kernel once the running plain docking is done.  Requires the
    ADADELTA search (ls_method 0)."""
    if idle_plain and params.ls_method != 0:
        raise ValueError("idle_plain needs the ADADELTA local search (ls_method 0)")
    pending = deque(sorted(requests, key=lambda r: r.arrival))
    waiting = deque()          # arrived, not yet admitted
    in_flight = []             # (request, ligand handle, first task, bytes)
    plain = None               # (request, ligand handle, PlainDocking, bytes)
    p_plain = plain_params(params, plain_threads) if idle_plain else None
    used = 0
    rep = ServiceReport()
    t0 = time.perf_counter()
    while pending or waiting or in_flight or plain:
        now = time.perf_counter() - t0
        if now > timeout:
            raise TimeoutError(f"service did not finish within {timeout} s")
        while pending and pending[0].arrival <= now:
            waiting.append(pending.popleft())
        # light load: the queue's head docks in the plain form, the others
        # wait for it; otherwise admission to the persistent kernel
        plain_mode = idle_plain and not in_flight and len(waiting) <= plain_queue
        if plain_mode and waiting and plain is None:
            req = waiting.popleft()
            lig = capi.ligand_from(ctx, req.ligand)
            need = lig.device_bytes() + params.nruns * ROW_BYTES
            plain = (req, lig, PlainDocking(ctx, grids[req.grid_index], lig, p_plain, req.seed), need)
            used += need
        # admission: device memory budget and free task slots, in arrival
        # order; not beside a running plain docking, which the persistent
        # kernel would starve
        while waiting and not plain_mode and plain is None:
            req = waiting[0]
            lig = capi.ligand_from(ctx, req.ligand)
            need = lig.device_bytes() + params.nruns * ROW_BYTES
            if (in_flight or plain) and used + need > mem_budget:
                lig.free()
                break
            first = server.submit(grids[req.grid_index], lig, params, req.seed)
            if first is None:   # no free slots yet
                lig.free()
                break
            waiting.popleft()
            in_flight.append((req, lig, first, need))
            used += need
        rep.max_in_flight = max(rep.max_in_flight, len(in_flight))
        still = []
        for req, lig, first, need in in_flight:
            if server.done(first, params.nruns):
                g, e, v = server.result(first, params.nruns, lig.n_genes)
                rep.done.append(Done(req, time.perf_counter() - t0 - req.arrival, g, e, v))
                lig.free()
                used -= need
            else:
                still.append((req, lig, first, need))
        in_flight = still
        if plain is not None and plain[2].done():
            req, lig, pd, need = plain
            g, e, v = pd.result()
            rep.done.append(Done(req, time.perf_counter() - t0 - req.arrival, g, e, v, route="plain"))
            lig.free()
            used -= need
            plain = None
        if in_flight or waiting or plain:
            time.sleep(poll_sleep)
        elif pending:
            time.sleep(max(0.0, min(pending[0].arrival - (time.perf_counter() - t0), 0.01)))
    rep.wall = time.perf_counter() - t0
    return rep
