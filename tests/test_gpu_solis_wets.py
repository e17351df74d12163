"""The Solis-Wets local search on the GPU against the oracle (Section II-A:
the miniapp's local search; Solis and Wets 1981).  Candidates are built with
single rounded FP32 operations from the same Philox stream on both sides, so
a chain whose accept decisions are clear-cut in the oracle (every energy
comparison decided by more than the FP32/FP64 gap) must end on the same
point bit for bit, after the same number of energies.  Dockings with it are
compared as distributions; the batched and served forms as bit-identical."""
import numpy as np
import pytest
import torch

from paper_2203_02096_gb300 import capi, synth
from tests.tolerances import energy_tol

pytestmark = pytest.mark.gpu


def _margin_ok(E0, trace, rel=2e-3, abs_=2e-3):
    """True when every accept decision of an oracle chain clears the gap."""
    e = E0
    for Ef, Eb, _, out in trace:
        if abs(Ef - e) <= abs_ + rel * max(abs(Ef), abs(e)):
            return False
        if out > 0:
            e = Ef
            continue
        if abs(Eb - e) <= abs_ + rel * max(abs(Eb), abs(e)):
            return False
        if out < 0:
            e = Eb
    return True


@pytest.mark.parametrize("threads,iters", [(32, 1), (128, 1), (32, 40), (64, 40), (128, 40), (256, 40)])
def test_solis_wets_chains_match_the_oracle(gpu, oracle_mod, drug_system, threads, iters):
    L = capi.ligand_from(gpu, drug_system["lig"])
    G = capi.grids_from_maps(gpu, drug_system["maps"], drug_system["box"])
    olig, ogrid = drug_system["olig"], drug_system["grid"]
    x0 = oracle_mod.init_population(olig.n_torsions, ogrid, 9, 0, 64)
    seed, run, gen = 77, 3, 5
    P = capi.default_params(ls_iters=iters, ls_threads=threads)
    xt = torch.from_numpy(x0).cuda()
    xb, Eb, ev = capi.dock_solis_wets(gpu, G, L, xt, P, seed=seed, run=run, generation=gen)
    xb2, Eb2, ev2 = capi.dock_solis_wets(gpu, G, L, xt, P, seed=seed, run=run, generation=gen)
    assert torch.equal(xb, xb2) and torch.equal(Eb, Eb2) and torch.equal(ev, ev2)   # deterministic
    xb, Eb, ev = xb.cpu().numpy(), Eb.cpu().numpy().astype(np.float64), ev.cpu().numpy()
    sw = oracle_mod.make_sw()
    clear = 0
    for c in range(len(x0)):
        Eo, xo, no, it, tr = oracle_mod.solis_wets(olig, ogrid, x0[c], iters, sw=sw, seed=seed, run=run, gen=gen,
                                                   entity=c)
        E0 = olig.score(ogrid, x0[c].astype(np.float64), with_grad=False)
        if _margin_ok(E0, tr):
            clear += 1
            assert np.array_equal(xb[c], xo), c
            assert ev[c] == no, c
            F = olig.atom_forces(ogrid, xo.astype(np.float64))[1]
            assert abs(Eb[c] - Eo) <= energy_tol(np.array([Eo]), F[None])[0], (c, Eb[c], Eo)
    assert clear >= (0.9 if iters == 1 else 0.25) * len(x0), clear
    # every chain: no worse than its start, reported energy = the oracle's energy of the returned pose
    E0s = olig.score_batch(ogrid, x0, with_grad=False)
    F0 = np.stack([olig.atom_forces(ogrid, x.astype(np.float64))[1] for x in x0])
    assert np.all(Eb <= E0s + energy_tol(E0s, F0))
    Er = olig.score_batch(ogrid, xb, with_grad=False)
    F = np.stack([olig.atom_forces(ogrid, x.astype(np.float64))[1] for x in xb])
    assert np.all(np.abs(Er - Eb) <= energy_tol(Er, F))
    assert np.allclose(np.linalg.norm(xb[:, 3:7], axis=1), 1.0, atol=1e-6)
    assert np.all((ev >= 1 + iters) & (ev <= 1 + 2 * iters)) if iters == 1 else np.all(ev <= 1 + 2 * iters)


def test_given_start_energies_are_used(gpu, oracle_mod, drug_system):
    """With E0 given the start is not re-evaluated: one energy fewer, the same
    points (the GPU's own start energies are passed back in)."""
    L = capi.ligand_from(gpu, drug_system["lig"])
    G = capi.grids_from_maps(gpu, drug_system["maps"], drug_system["box"])
    x0 = torch.from_numpy(oracle_mod.init_population(L.n_torsions, drug_system["grid"], 4, 0, 32)).cuda()
    P = capi.default_params(ls_iters=20, ls_threads=32)   # one-warp teams, as score_batch
    E0 = capi.score_batch(gpu, G, L, x0)
    xa, Ea, na = capi.dock_solis_wets(gpu, G, L, x0, P, seed=1)
    xb, Eb, nb = capi.dock_solis_wets(gpu, G, L, x0, P, E0=E0, seed=1)
    assert torch.equal(xa, xb) and torch.equal(Ea, Eb) and torch.equal(na, nb + 1)


def _ks(a, b):
    a, b = np.sort(a), np.sort(b)
    xs = np.concatenate([a, b])
    return np.max(np.abs(np.searchsorted(a, xs, side="right") / len(a) - np.searchsorted(b, xs, side="right") / len(b)))


def test_dock_with_solis_wets_small_ligand_workload(gpu, oracle_mod):
    """The small-ligand workload with Solis-Wets: every run stops at the first
    generation boundary at or past the budget, FP64 re-scores equal the
    oracle's energy of the returned poses, deterministic, and the best-energy
    distribution matches the oracle's docking of the same inputs."""
    w = synth.small_ligand_workload()
    maps = oracle_mod.build_maps(w.receptor, w.box).astype(np.float32)
    ogrid = oracle_mod.OracleGrid(maps, w.box)
    olig = oracle_mod.OracleLigand(w.ligand)
    L = capi.ligand_from(gpu, w.ligand)
    G = capi.grids_from_maps(gpu, maps, w.box)
    P = capi.default_params(pop_size=w.pop_size, nruns=w.nruns, max_evals=w.max_evals, ls_iters=w.ls_iters,
                            ls_method=1)
    bg, bE, ev = capi.dock(gpu, G, L, P, w.seed)
    bg2, bE2, ev2 = capi.dock(gpu, G, L, P, w.seed)
    assert np.array_equal(bg, bg2) and np.array_equal(bE, bE2) and np.array_equal(ev, ev2)
    n_ls = (6 * w.pop_size + 99) // 100
    per_gen_max = (w.pop_size - 1) + n_ls * 2 * w.ls_iters
    assert np.all(ev >= w.max_evals) and np.all(ev < w.max_evals + per_gen_max)
    rescored = olig.score_batch(ogrid, bg, with_grad=False)
    assert np.allclose(bE, rescored, rtol=1e-9, atol=1e-9)
    op = oracle_mod.make_params(pop_size=w.pop_size, nruns=w.nruns, max_evals=w.max_evals, ls_iters=w.ls_iters,
                                ls_method=1)
    og, oE, oev = oracle_mod.dock(olig, ogrid, op, w.seed)
    assert np.all(oev >= w.max_evals)
    assert abs(np.median(bE) - np.median(oE)) < 0.5, (np.sort(bE), np.sort(oE))
    assert _ks(bE, oE) <= 0.7


def test_batched_and_served_solis_wets_equal_plain(gpu, drug_system):
    """dock_batch and the service with Solis-Wets give, run for run, the bits
    of the plain docking with one-warp searches."""
    rng = np.random.default_rng(5)
    ligs = [synth.make_ligand(int(rng.integers(10, 70)), int(rng.integers(0, 20)), seed=300 + k) for k in range(5)]
    L = [capi.ligand_from(gpu, l) for l in ligs]
    G = capi.grids_from_maps(gpu, drug_system["maps"], drug_system["box"])
    P = capi.default_params(pop_size=40, nruns=3, max_evals=3000, ls_iters=30, ls_threads=32, ls_method=1)
    seeds = np.arange(5, dtype=np.uint64) * 104729 + 11
    out = capi.dock_batch(gpu, G, L, P, seeds)
    torch.cuda.synchronize()
    bg, bE, ev = (out[k].cpu().numpy() for k in ("best_geno", "best_E", "evals"))
    for k in range(5):
        g1, e1, v1 = capi.dock(gpu, G, L[k], P, int(seeds[k]))
        assert np.array_equal(bg[k, :, :L[k].n_genes], g1), k
        assert np.array_equal(bE[k], e1) and np.array_equal(ev[k], v1), k
    from paper_2203_02096_gb300 import serve
    server = capi.Server(gpu, capacity=256, max_atoms=128, pop_max=64)
    reqs = [serve.Request(ligs[k], 0, seed=int(seeds[k])) for k in range(5)]
    for r, t in zip(reqs, serve.poisson_arrivals(5, 100.0, seed=2)):
        r.arrival = float(t)
    rep = serve.run(gpu, server, [G], reqs, P)
    server.close()
    by_seed = {d.request.seed: d for d in rep.done}
    for k in range(5):
        d = by_seed[int(seeds[k])]
        assert np.array_equal(d.best_geno, bg[k, :, :L[k].n_genes]) and np.array_equal(d.best_E, bE[k])
