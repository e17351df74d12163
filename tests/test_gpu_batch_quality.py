"""Batched and served docking against the oracle (configs of the batching and
serving workloads, at a reduced budget): three ligands of different sizes,
20 runs each, docked in one persistent launch (dock_batch) and through the
continuous-batching server, and by the FP64 oracle (orc_dock) on the same
ligands, grids and seeds.  A docking's best energies are a stochastic search
result, so the runs are compared as distributions: medians within
0.5 kcal/mol and a two-sample Kolmogorov-Smirnov distance at most 0.5 (the
1% level for 20 against 20 runs).  Each returned FP64 energy is also the
oracle's energy of the returned pose."""
import numpy as np
import pytest
import torch

from paper_2203_02096_gb300 import capi, serve, synth

pytestmark = pytest.mark.gpu

NRUNS, EVALS = 20, 60_000
SIZES = [(16, 4), (40, 10), (64, 16)]


def _ks(a, b):
    a, b = np.sort(a), np.sort(b)
    xs = np.concatenate([a, b])
    return np.max(np.abs(np.searchsorted(a, xs, side="right") / len(a) - np.searchsorted(b, xs, side="right") / len(b)))


@pytest.fixture(scope="module")
def quality_case(oracle_mod, drug_system):
    ligs = [synth.make_ligand(n, t, seed=500 + n) for n, t in SIZES]
    seeds = np.array([11, 12, 13], dtype=np.uint64)
    P = oracle_mod.make_params(pop_size=150, nruns=NRUNS, max_evals=EVALS, ls_iters=300)
    ref = []
    for lig, sd in zip(ligs, seeds):
        olig = oracle_mod.OracleLigand(lig)
        _, oE, oev = oracle_mod.dock(olig, drug_system["grid"], P, int(sd))
        ref.append((olig, oE, oev))
    return ligs, seeds, ref


def _check(kind, ligs, ref, geno, E, ev, ogrid):
    for k, (olig, oE, oev) in enumerate(ref):
        g, e = geno[k][:, :olig.n_genes], E[k]
        assert np.array_equal(ev[k], oev), (kind, k)      # same stop rule, same evaluation counts
        assert np.allclose(e, olig.score_batch(ogrid, g, with_grad=False), rtol=1e-9, atol=1e-9)
        dm, ks = abs(np.median(e) - np.median(oE)), _ks(e, oE)
        print(f"\n{kind} ligand {ligs[k].n_atoms} atoms / {olig.n_torsions} torsions: median best E "
              f"{np.median(e):.3f} (oracle {np.median(oE):.3f}); KS {ks:.2f}")
        assert dm < 0.5 and ks <= 0.5, (kind, k, np.sort(e), np.sort(oE))


def test_dock_batch_matches_oracle_distribution(gpu, drug_system, quality_case):
    ligs, seeds, ref = quality_case
    L = [capi.ligand_from(gpu, l) for l in ligs]
    G = capi.grids_from_maps(gpu, drug_system["maps"], drug_system["box"])
    P = capi.default_params(pop_size=150, nruns=NRUNS, max_evals=EVALS, ls_iters=300)
    out = capi.dock_batch(gpu, G, L, P, seeds)
    torch.cuda.synchronize()
    geno, E, ev = (out[k].cpu().numpy() for k in ("best_geno", "best_E", "evals"))
    _check("dock_batch", ligs, ref, geno, E, ev, drug_system["grid"])


def test_server_matches_oracle_distribution(gpu, drug_system, quality_case):
    ligs, seeds, ref = quality_case
    G = capi.grids_from_maps(gpu, drug_system["maps"], drug_system["box"])
    P = capi.default_params(pop_size=150, nruns=NRUNS, max_evals=EVALS, ls_iters=300)
    server = capi.Server(gpu, capacity=1024, max_atoms=128, pop_max=150)
    reqs = [serve.Request(l, 0, seed=int(s)) for l, s in zip(ligs, seeds)]
    for r, t in zip(reqs, [0.0, 0.01, 0.02]):
        r.arrival = t
    rep = serve.run(gpu, server, [G], reqs, P)
    server.close()
    by_seed = {d.request.seed: d for d in rep.done}
    geno = [by_seed[int(s)].best_geno for s in seeds]
    E = [by_seed[int(s)].best_E for s in seeds]
    ev = [by_seed[int(s)].evals for s in seeds]
    _check("server", ligs, ref, geno, E, ev, drug_system["grid"])
