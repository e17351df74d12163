"""Many ligands in one persistent launch (dock_batch): each run's result is
bit-identical to the per-ligand docking with one-warp local searches (same
operators, same Philox stream, same evaluator), is the same alone and in a
mixed batch, and its FP64 re-score is the oracle's energy of its pose."""
import numpy as np
import pytest
import torch

from paper_2203_02096_gb300 import capi, synth

pytestmark = pytest.mark.gpu


def _ligands(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        na = int(rng.integers(10, 109))
        nt = int(rng.integers(0, 33))
        out.append(synth.make_ligand(na, nt, seed=1000 + k))
    return out


def test_batch_equals_per_ligand_docking_and_is_mix_independent(gpu, drug_system, oracle_mod):
    ligs = _ligands(12, 0)
    L = [capi.ligand_from(gpu, l) for l in ligs]
    G = capi.grids_from_maps(gpu, drug_system["maps"], drug_system["box"])
    P = capi.default_params(pop_size=40, nruns=3, max_evals=2500, ls_iters=15, ls_threads=32)
    seeds = np.arange(12, dtype=np.uint64) * 7919 + 3
    out = capi.dock_batch(gpu, G, L, P, seeds)
    torch.cuda.synchronize()
    bg, bE, ev = (out[k].cpu().numpy() for k in ("best_geno", "best_E", "evals"))
    per_gen = 39 + P.ls_count * 15 if P.ls_count >= 0 else 39 + 3 * 15
    n_ls = (6 * 40 + 99) // 100
    per_gen = 39 + n_ls * 15
    for k in (0, 5, 11):
        g1, e1, v1 = capi.dock(gpu, G, L[k], P, int(seeds[k]))
        G_k = L[k].n_genes
        assert np.array_equal(bg[k, :, :G_k], g1), k
        assert np.array_equal(bE[k], e1) and np.array_equal(ev[k], v1), k
    assert np.all(ev >= 2500) and np.all((ev - 40) % per_gen == 0)
    # the same ligands alone and in another mix
    sub = [3, 7]
    out2 = capi.dock_batch(gpu, G, [L[i] for i in sub], P, seeds[sub])
    torch.cuda.synchronize()
    assert torch.equal(out2["best_geno"], out["best_geno"][sub])
    assert torch.equal(out2["best_E"], out["best_E"][sub])
    # FP64 re-score = oracle energy of the returned pose
    ogrid = drug_system["grid"]
    for k in (1, 4, 9):
        olig = oracle_mod.OracleLigand(ligs[k])
        ref = olig.score_batch(ogrid, bg[k, :, :L[k].n_genes], with_grad=False)
        assert np.allclose(bE[k], ref, rtol=1e-9, atol=1e-9)


def test_packing_by_atom_count_changes_nothing(gpu, drug_system):
    """batch_pack = 1 (one launch per atom-count class, each sized for its own
    largest ligand) gives the same results, bit for bit, as one launch."""
    ligs = _ligands(14, 5) + [synth.make_ligand(20, 3, seed=77), synth.make_ligand(120, 20, seed=78)]
    L = [capi.ligand_from(gpu, l) for l in ligs]
    G = capi.grids_from_maps(gpu, drug_system["maps"], drug_system["box"])
    seeds = np.arange(len(L), dtype=np.uint64) * 31 + 5
    outs = []
    for pack in (0, 1):
        P = capi.default_params(pop_size=40, nruns=2, max_evals=1500, ls_iters=10, batch_pack=pack)
        outs.append(capi.dock_batch(gpu, G, L, P, seeds))
    torch.cuda.synchronize()
    for k in ("best_geno", "best_E32", "best_E", "evals"):
        assert torch.equal(outs[0][k], outs[1][k]), k
    with pytest.raises(capi.DockError, match="INVALID"):
        capi.dock_batch(gpu, G, L[:2], capi.default_params(batch_pack=2), seeds[:2])
