"""Serving with continuous batching: requests arriving while others run are
admitted into the running persistent kernel; each request's result is the
same alone, in a mix of requests of different sizes on two receptors, and
from dock_batch on the same inputs."""
import numpy as np
import pytest
import torch

from paper_2203_02096_gb300 import capi, serve, synth

pytestmark = pytest.mark.gpu


def _ligand(k):
    rng = np.random.default_rng(100 + k)
    n = int(np.exp(rng.uniform(np.log(10), np.log(128))))
    return synth.make_ligand(n, int(rng.integers(0, 33)), seed=200 + k)


def test_results_same_alone_in_the_mix_and_batched(gpu, drug_system):
    G0 = capi.grids_from_maps(gpu, drug_system["maps"], drug_system["box"])
    box1 = synth.make_box(48, center=(-20.0, 5.0, 11.0))
    G1 = capi.grids_from_receptor(gpu, synth.make_receptor(1500, center=(-20.0, 5.0, 11.0), seed=9), box1)
    grids = [G0, G1]
    P = capi.default_params(pop_size=40, nruns=4, max_evals=2500, ls_iters=10)
    server = capi.Server(gpu, capacity=1024, max_atoms=128, pop_max=150)
    reqs = [serve.Request(_ligand(k), k % 2, seed=31 * k + 1) for k in range(10)]
    # request 3 alone
    alone = serve.run(gpu, server, grids, [serve.Request(reqs[3].ligand, reqs[3].grid_index, reqs[3].seed)], P)
    assert len(alone.done) == 1
    # all ten, arriving at 200/s (most while others run)
    for r, t in zip(reqs, serve.poisson_arrivals(len(reqs), 200.0, seed=1)):
        r.arrival = float(t)
    mixed = serve.run(gpu, server, grids, reqs, P)
    assert len(mixed.done) == 10 and mixed.max_in_flight >= 2
    by_seed = {d.request.seed: d for d in mixed.done}
    a, m = alone.done[0], by_seed[reqs[3].seed]
    assert np.array_equal(a.best_geno, m.best_geno) and np.array_equal(a.best_E, m.best_E)
    assert np.array_equal(a.evals, m.evals)
    # the same runs through dock_batch
    for k in (0, 3, 7):
        L = capi.ligand_from(gpu, reqs[k].ligand)
        out = capi.dock_batch(gpu, grids[reqs[k].grid_index], [L], P, np.array([reqs[k].seed], np.uint64))
        torch.cuda.synchronize()
        d = by_seed[reqs[k].seed]
        assert np.array_equal(out["best_geno"][0, :, :L.n_genes].cpu().numpy(), d.best_geno)
        assert np.array_equal(out["best_E"][0].cpu().numpy(), d.best_E)
    lat = mixed.latencies()
    assert np.all(np.isfinite(lat)) and np.all(lat > 0)
    server.close()


def test_idle_plain_route_gives_the_served_results(gpu, drug_system):
    """With idle_plain and one-warp plain teams, requests that find the GPU
    idle dock in the plain form; their results equal dock_batch's (and so
    the served ones) bit for bit, so the route does not change a request's
    answer.  A burst that queues past the bound goes to the persistent
    kernel."""
    G0 = capi.grids_from_maps(gpu, drug_system["maps"], drug_system["box"])
    P = capi.default_params(pop_size=40, nruns=4, max_evals=2500, ls_iters=10)
    server = capi.Server(gpu, capacity=1024, max_atoms=128, pop_max=150)
    reqs = [serve.Request(_ligand(k), 0, seed=31 * k + 1, arrival=0.5 * k) for k in range(4)]
    burst = [serve.Request(_ligand(10 + k), 0, seed=7 * k + 5, arrival=2.5) for k in range(8)]
    rep = serve.run(gpu, server, [G0], reqs + burst, P, idle_plain=True, plain_queue=4, plain_threads=32)
    assert len(rep.done) == 12
    by_seed = {d.request.seed: d for d in rep.done}
    assert all(by_seed[r.seed].route == "plain" for r in reqs)
    assert sum(by_seed[r.seed].route == "served" for r in burst) >= 7
    for r in reqs[:2] + burst[:2]:
        L = capi.ligand_from(gpu, r.ligand)
        out = capi.dock_batch(gpu, G0, [L], P, np.array([r.seed], np.uint64))
        torch.cuda.synchronize()
        d = by_seed[r.seed]
        assert np.array_equal(out["best_geno"][0, :, :L.n_genes].cpu().numpy(), d.best_geno), d.route
        assert np.array_equal(out["best_E"][0].cpu().numpy(), d.best_E), d.route
        assert np.array_equal(out["evals"][0].cpu().numpy(), d.evals), d.route
    server.close()
