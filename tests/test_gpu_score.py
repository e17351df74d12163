"""GPU parity of the evaluator (pose, particle-grid + intramolecular energy,
analytic gradient) against the FP64 oracle, through the C-ABI.  Same seeded
inputs on both sides; maps come from the oracle and are loaded into the
library with load_grids, so both read identical FP32 node values."""
import numpy as np
import pytest
import torch

from paper_2203_02096_gb300 import capi, synth
from tests.tolerances import energy_tol, grad_tol

pytestmark = pytest.mark.gpu


def _load(gpu, system):
    return capi.ligand_from(gpu, system["lig"]), capi.grids_from_maps(gpu, system["maps"], system["box"])


def _genos(n, nt, box, seed, outside=0.1):
    g = synth.make_genotypes(n, nt, box, seed=seed)
    rng = np.random.default_rng(seed + 1000)
    k = int(n * outside)
    if k:  # some translations outside the box (out-of-box penalty and clamped reads)
        g[:k, 0:3] = rng.uniform(box.box_lo() - 6.0, box.box_hi() + 6.0, size=(k, 3)).astype(np.float32)
    return g


def _compare(gpu, system, genos, check_grad=True, require_plain=0.97):
    L, G = _load(gpu, system)
    olig, ogrid = system["olig"], system["grid"]
    x = torch.from_numpy(genos).cuda()
    if check_grad:
        E, grad = capi.score_grad_batch(gpu, G, L, x)
        E2 = capi.score_batch(gpu, G, L, x)
    else:
        E = capi.score_batch(gpu, G, L, x)
    torch.cuda.synchronize()
    E = E.cpu().numpy().astype(np.float64)
    Eo, Go = olig.score_batch(ogrid, genos, with_grad=True)
    F = np.stack([olig.atom_forces(ogrid, g.astype(np.float64))[1] for g in genos])
    err = np.abs(E - Eo)
    tol = energy_tol(Eo, F)
    bad = np.nonzero(err > tol)[0]
    assert len(bad) == 0, [(int(b), float(E[b]), float(Eo[b]), float(tol[b])) for b in bad[:5]]
    plain = np.mean(err <= energy_tol(Eo))
    assert plain >= require_plain, plain
    if check_grad:
        assert np.array_equal(E, E2.cpu().numpy().astype(np.float64))  # same energy with or without gradient
        g = grad.cpu().numpy().astype(np.float64)
        margins = np.stack([olig.margins(ogrid, gg.astype(np.float64)) for gg in genos])
        smooth = (margins[:, 0] > 1e-4) & (margins[:, 1] > 1e-4) & (margins[:, 2] > 1e-4)
        gerr = np.abs(g - Go).max(axis=1)
        gbad = np.nonzero(smooth & (gerr > grad_tol(Go)))[0]
        assert len(gbad) == 0, [(int(b), float(gerr[b]), float(grad_tol(Go)[b])) for b in gbad[:5]]
        # near-face / near-cutoff genotypes are excluded, more of them for big
        # ligands; enough smooth ones must remain for the check to mean something
        assert smooth.sum() >= max(8, len(genos) // 4), int(smooth.sum())
    return E, Eo


def test_pose_matches_oracle(gpu, small_system):
    L = capi.ligand_from(gpu, small_system["lig"])
    genos = _genos(300, L.n_torsions, small_system["box"], seed=1)
    xyz = capi.pose_batch(gpu, L, torch.from_numpy(genos).cuda()).cpu().numpy()
    ref = np.stack([small_system["olig"].pose(g.astype(np.float64)) for g in genos])
    assert np.abs(xyz - ref).max() < 1e-4


def test_score_small_ligand_tiles_and_ragged_tail(gpu, small_system):
    # 4 warps per block: 397 genotypes = many blocks plus a ragged tail
    genos = _genos(397, small_system["olig"].n_torsions, small_system["box"], seed=2)
    _compare(gpu, small_system, genos)


def test_score_drug_ligand(gpu, drug_system):
    genos = _genos(1029, drug_system["olig"].n_torsions, drug_system["box"], seed=3)
    _compare(gpu, drug_system, genos)


def test_score_grad_full_size_sampled(gpu, diff_system):
    """65536 genotypes of the 64-atom / 16-torsion ligand in one launch (the
    differentiation workload); the oracle checks a 256-genotype sample."""
    box = diff_system["box"]
    L, G = _load(gpu, diff_system)
    genos = synth.make_genotypes(65536, L.n_torsions, box, seed=0)
    x = torch.from_numpy(genos).cuda()
    E, grad = capi.score_grad_batch(gpu, G, L, x)
    E, grad = E.cpu().numpy().astype(np.float64), grad.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(E)) and np.all(np.isfinite(grad))
    idx = np.random.default_rng(0).choice(65536, 256, replace=False)
    olig, ogrid = diff_system["olig"], diff_system["grid"]
    Eo, Go = olig.score_batch(ogrid, genos[idx], with_grad=True)
    F = np.stack([olig.atom_forces(ogrid, genos[i].astype(np.float64))[1] for i in idx])
    assert np.all(np.abs(E[idx] - Eo) <= energy_tol(Eo, F))
    margins = np.stack([olig.margins(ogrid, genos[i].astype(np.float64)) for i in idx])
    smooth = (margins > 1e-4).all(axis=1)
    assert np.all((np.abs(grad[idx] - Go).max(axis=1) <= grad_tol(Go))[smooth])


def test_deterministic(gpu, drug_system):
    L, G = _load(gpu, drug_system)
    x = torch.from_numpy(_genos(500, L.n_torsions, drug_system["box"], seed=4)).cuda()
    a = capi.score_grad_batch(gpu, G, L, x)
    b = capi.score_grad_batch(gpu, G, L, x)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


@pytest.mark.parametrize("n,t", [(1, 0), (2, 0), (12, 0), (10, 32), (108, 31), (128, 32)])
def test_edge_ligands(gpu, oracle_mod, drug_system, n, t):
    """Single atom, no pairs, rigid ligands, 32 torsions, the paper's largest size."""
    lig = synth.make_ligand(n, t, seed=n)
    sysd = dict(lig=lig, box=drug_system["box"], maps=drug_system["maps"], grid=drug_system["grid"],
                olig=oracle_mod.OracleLigand(lig))
    genos = _genos(97, lig.n_torsions, drug_system["box"], seed=n)
    _compare(gpu, sysd, genos)


def test_max_atoms_ligand(gpu, oracle_mod, drug_system):
    lig = synth.make_ligand(255, 32, seed=5)
    sysd = dict(lig=lig, box=drug_system["box"], maps=drug_system["maps"], grid=drug_system["grid"],
                olig=oracle_mod.OracleLigand(lig))
    _compare(gpu, sysd, _genos(40, lig.n_torsions, drug_system["box"], seed=6), require_plain=0.9)


def test_empty_batch_and_errors(gpu, small_system):
    L, G = _load(gpu, small_system)
    e = torch.empty(0, device="cuda")
    capi.score_batch(gpu, G, L, torch.empty((0, L.n_genes), device="cuda"), E=e)
    lig = small_system["lig"]
    with pytest.raises(capi.DockError, match="DISCONNECTED"):
        capi.load_ligand(gpu, lig.xyz, lig.types, lig.charges, lig.bonds[:-1], lig.rotatable[:-1])
    with pytest.raises(capi.DockError, match="TYPE"):
        capi.load_ligand(gpu, lig.xyz, np.full_like(lig.types, 9), lig.charges, lig.bonds, lig.rotatable)
    with pytest.raises(capi.DockError, match="SIZE"):
        big = synth.make_ligand(256, 0, seed=0)
        capi.load_ligand(gpu, big.xyz, big.types, big.charges, big.bonds, big.rotatable)
    # a ring: close the tree with one extra bond and mark a ring bond rotatable
    bonds = np.vstack([lig.bonds, [[0, lig.n_atoms - 1]]])
    rot = np.concatenate([np.zeros(len(lig.bonds), np.int32), [1]])
    with pytest.raises(capi.DockError, match="RING"):
        capi.load_ligand(gpu, lig.xyz, lig.types, lig.charges, bonds, rot)
    # a ligand type without a map
    box = synth.make_box(24, type_names=("C",))
    with pytest.raises(capi.DockError, match="NOMAP"):
        G1 = capi.grids_from_maps(gpu, np.zeros((3, 24, 24, 24), np.float32), box)
        capi.score_batch(gpu, G1, L, torch.zeros((1, L.n_genes), device="cuda"))
    with pytest.raises(capi.DockError, match="INVALID"):
        capi.load_grids(gpu, np.zeros((3, 4, 4, 4), np.float32), (4, 4, 4), (0, 0, 0), 0.0, [0, -1, -2])


def test_map_builder_matches_oracle(gpu, oracle_mod):
    """Device direct-sum maps vs the oracle's, on a box reaching into the receptor."""
    rec = synth.make_receptor(600, inner=4.0, outer=12.0, seed=3)
    box = synth.make_box(20)
    G = capi.grids_from_receptor(gpu, rec, box)
    got = G.read_maps(box.dims).astype(np.float64)
    ref = oracle_mod.build_maps(rec, box)
    cap = ref >= 1e5
    assert cap.any() and np.all(got[cap] >= 0.99e5)
    ok = ~cap
    scale = np.abs(ref[ok]) + 1e-3 * np.abs(ref[ok]).max()
    assert np.max(np.abs(got[ok] - ref[ok]) / scale) < 1e-3
