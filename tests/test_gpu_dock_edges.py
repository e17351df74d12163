"""Docking at the edges of its parameters and at the drug-size workload's
full size (Section II-A: runs of a population of 150, local search on a
random sample of each generation), against the FP64 oracle:

* degenerate searches -- no generation at all (budget <= population), no
  local search (ls_count 0 or ls_iters 0), a rigid ligand, one run,
  population 2 -- give the oracle's evaluation counts exactly and poses
  whose FP64 re-score is the oracle's energy of the pose;
* the drug-size docking in the launch shape bench.py times (50 runs x 2.5M
  evaluations, 128 threads per local-search chain), checked on every run's
  returned pose (FP64 re-score = oracle energy) and on its counts;
* the service's error paths: a full queue, an oversized ligand, invalid
  parameters."""
import numpy as np
import pytest
import torch

from paper_2203_02096_gb300 import capi, synth

pytestmark = pytest.mark.gpu


def _oparams(oracle_mod, p):
    return oracle_mod.make_params(pop_size=p.pop_size, nruns=p.nruns, max_evals=p.max_evals, ls_iters=p.ls_iters,
                                  rho=p.rho, eps=p.eps, p_tour=p.p_tour, p_cross=p.p_cross, p_mut=p.p_mut,
                                  trans_mut=p.trans_mut,
                                  ls_count=(6 * p.pop_size + 99) // 100 if p.ls_count < 0 else p.ls_count)


CASES = {
    "no generation": dict(pop_size=50, nruns=3, max_evals=40),
    "budget = population": dict(pop_size=50, nruns=3, max_evals=50),
    "no local search (count 0)": dict(pop_size=40, nruns=2, max_evals=500, ls_count=0),
    "no local search (iters 0)": dict(pop_size=40, nruns=2, max_evals=500, ls_iters=0),
    "one run, population 2": dict(pop_size=2, nruns=1, max_evals=60, ls_iters=5),
    "rigid ligand": dict(pop_size=30, nruns=2, max_evals=900, ls_iters=10),
}


@pytest.mark.parametrize("case", list(CASES))
def test_degenerate_dockings_match_the_oracle(gpu, oracle_mod, small_system, case):
    kw = dict(CASES[case])
    lig = small_system["lig"] if case != "rigid ligand" else synth.make_ligand(12, 0, ("C", "A", "N", "OA", "HD"), seed=3)
    olig = small_system["olig"] if case != "rigid ligand" else oracle_mod.OracleLigand(lig)
    L = capi.ligand_from(gpu, lig)
    G = capi.grids_from_maps(gpu, small_system["maps"], small_system["box"])
    P = capi.default_params(**kw)
    bg, bE, ev = capi.dock(gpu, G, L, P, 7)
    og, oE, oev = oracle_mod.dock(olig, small_system["grid"], _oparams(oracle_mod, P), 7)
    assert np.array_equal(ev, oev), (ev, oev)
    assert np.all(ev >= min(P.max_evals, P.pop_size)) and np.all(ev >= P.pop_size)
    assert np.allclose(bE, olig.score_batch(small_system["grid"], bg, with_grad=False), rtol=1e-9, atol=1e-9)
    assert np.allclose(np.linalg.norm(bg[:, 3:7], axis=1), 1.0, atol=1e-6)
    if P.max_evals <= P.pop_size:
        # no generation: the best of the initial population (bit-identical
        # genes on both sides), the same individual wherever the oracle's best
        # is clear of the runner-up by more than the FP32/FP64 gap
        for r in range(P.nruns):
            pop0 = oracle_mod.init_population(olig.n_torsions, small_system["grid"], 7, r, P.pop_size)
            e0 = np.sort(olig.score_batch(small_system["grid"], pop0, with_grad=False))
            if e0[1] - e0[0] > 1e-3 * max(1.0, abs(e0[0])):
                assert np.array_equal(bg[r], og[r]), r


def test_drug_docking_full_size(gpu, oracle_mod, drug_system):
    """50 runs x 2.5M evaluations, 128 threads per chain: counts by the stop
    rule, every returned pose's FP64 energy = the oracle's, and a median best
    energy below zero."""
    w = drug_system["w"]
    L = capi.ligand_from(gpu, w.ligand)
    G = capi.grids_from_maps(gpu, drug_system["maps"], drug_system["box"])
    P = capi.default_params(pop_size=w.pop_size, nruns=w.nruns, max_evals=w.max_evals, ls_iters=w.ls_iters,
                            ls_threads=128)
    out = capi.dock_async(gpu, G, L, P, w.seed)
    torch.cuda.synchronize()
    bg, bE, ev = (out[k].cpu().numpy() for k in ("best_geno", "best_E", "evals"))
    n_ls = (6 * w.pop_size + 99) // 100
    per_gen = (w.pop_size - 1) + n_ls * w.ls_iters
    ngen = -(-(w.max_evals - w.pop_size) // per_gen)
    assert np.all(ev == w.pop_size + ngen * per_gen)
    olig, ogrid = drug_system["olig"], drug_system["grid"]
    assert np.allclose(bE, olig.score_batch(ogrid, bg, with_grad=False), rtol=1e-9, atol=1e-9)
    # the FP32 energy the search kept agrees with the FP64 re-score within the tolerance
    e32 = out["best_E32"].cpu().numpy().astype(np.float64)
    assert np.all(np.abs(e32 - bE) <= np.maximum(1e-4 * np.abs(bE), 1e-3) + 0.05)
    assert np.median(bE) < 0.0


def test_server_error_paths(gpu, drug_system):
    G = capi.grids_from_maps(gpu, drug_system["maps"], drug_system["box"])
    small = capi.ligand_from(gpu, synth.make_ligand(12, 2, seed=1))
    big = capi.ligand_from(gpu, synth.make_ligand(40, 4, seed=2))
    P = capi.default_params(pop_size=20, nruns=3, max_evals=400, ls_iters=5)
    server = capi.Server(gpu, capacity=4, max_atoms=32, pop_max=32)
    with pytest.raises(capi.DockError):               # above max_atoms
        server.submit(G, big, P, 1)
    with pytest.raises(capi.DockError):               # population above pop_max
        server.submit(G, small, capi.default_params(pop_size=64, nruns=1), 1)
    with pytest.raises(capi.DockError):               # more runs than slots
        server.submit(G, small, capi.default_params(pop_size=20, nruns=5), 1)
    import time
    first = server.submit(G, small, P, 1)             # 3 of 4 slots
    assert first == 0
    t0 = time.time()
    while not server.done(first, 3) and time.time() - t0 < 60:   # polling keeps the kernel running
        time.sleep(1e-3)
    g1, e1, v1 = server.result(first, 3, small.n_genes)
    second = server.submit(G, small, P, 2)            # reuses slots 0 and 1: admitted now the first is done
    assert second == 3
    while not server.done(second, 3) and time.time() - t0 < 60:
        time.sleep(1e-3)
    g2, e2, v2 = server.result(second, 3, small.n_genes)
    assert np.all(v1 >= 400) and np.all(v2 >= 400)
    with pytest.raises(capi.DockError):               # its slots now hold the second request
        server.result(first, 3, small.n_genes)
    # tasks 6-8 take slots 2, 3, 0, whose tasks are done: admitted
    third = server.submit(G, small, P, 3)
    assert third == 6
    # tasks 9-11 need slots 1, 2, 3; slots 2 and 3 hold tasks 6 and 7, so
    # the request is admitted only if those have finished, else refused (None)
    fourth = server.submit(G, small, P, 4)
    assert fourth is None or fourth == 9
    server.close()


def test_server_cancel(gpu, drug_system):
    """Cancelling a large request right after submitting it: every run
    completes, each either withdrawn (no evaluation, energy +inf) or run in
    full; runs no warp had claimed are withdrawn; a request submitted
    afterwards is unaffected (same result as alone)."""
    import time
    G = capi.grids_from_maps(gpu, drug_system["maps"], drug_system["box"])
    lig = capi.ligand_from(gpu, synth.make_ligand(12, 2, seed=5))
    server = capi.Server(gpu, capacity=16384, max_atoms=32, pop_max=64)
    P = capi.default_params(pop_size=40, nruns=8192, max_evals=60_000, ls_iters=20)
    first = server.submit(G, lig, P, 11)
    server.cancel(first, 8192)
    t0 = time.time()
    while not server.done(first, 8192) and time.time() - t0 < 120:
        time.sleep(1e-3)
    g, e, v = server.result(first, 8192, lig.n_genes)
    withdrawn = v == 0
    assert np.all(np.isinf(e[withdrawn])) and np.all(np.isfinite(e[~withdrawn]))
    assert np.all(v[~withdrawn] >= 60_000)
    assert withdrawn.sum() > 0
    P2 = capi.default_params(pop_size=40, nruns=2, max_evals=3000, ls_iters=10)
    second = server.submit(G, lig, P2, 12)
    while not server.done(second, 2) and time.time() - t0 < 120:
        time.sleep(1e-3)
    g2, e2, v2 = server.result(second, 2, lig.n_genes)
    server.close()
    out = capi.dock_batch(gpu, G, [lig], P2, np.array([12], np.uint64))
    torch.cuda.synchronize()
    assert np.array_equal(out["best_geno"][0, :, :lig.n_genes].cpu().numpy(), g2)
    assert np.array_equal(out["best_E"][0].cpu().numpy(), e2)
    with pytest.raises(capi.DockError):
        capi.Server(gpu, capacity=8, max_atoms=32, pop_max=64).cancel(0, 1)   # nothing submitted
