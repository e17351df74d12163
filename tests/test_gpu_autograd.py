"""The differentiation workload: 65536 random genotypes of a 64-atom /
16-torsion ligand in the 64^3 grid set through torch.autograd; on a
256-genotype subset the autograd gradient matches the FP64 oracle's analytic
gradient and its central finite differences (h = 1e-4)."""
import numpy as np
import pytest
import torch

from paper_2203_02096_gb300 import autograd, capi, synth
from tests.tolerances import energy_tol, grad_tol

pytestmark = pytest.mark.gpu


def test_autograd_matches_oracle_and_finite_differences(gpu, diff_system):
    L = capi.ligand_from(gpu, diff_system["lig"])
    G = capi.grids_from_maps(gpu, diff_system["maps"], diff_system["box"])
    olig, ogrid, box = diff_system["olig"], diff_system["grid"], diff_system["box"]
    genos = synth.make_genotypes(65536, L.n_torsions, box, seed=4)
    x = torch.from_numpy(genos).cuda().requires_grad_(True)
    E = autograd.score(x, gpu, G, L)
    w = torch.linspace(0.5, 1.5, E.shape[0], device="cuda")   # a non-trivial grad_output
    (E * w).sum().backward()
    g = (x.grad / w[:, None]).cpu().numpy().astype(np.float64)
    # forward without grad gives the same energies
    with torch.no_grad():
        E2 = autograd.score(x.detach(), gpu, G, L)
    assert torch.equal(E.detach(), E2)
    idx = np.random.default_rng(1).choice(65536, 256, replace=False)
    Eo, Go = olig.score_batch(ogrid, genos[idx], with_grad=True)
    F = np.stack([olig.atom_forces(ogrid, genos[i].astype(np.float64))[1] for i in idx])
    assert np.all(np.abs(E.detach().cpu().numpy()[idx] - Eo) <= energy_tol(Eo, F))
    margins = np.stack([olig.margins(ogrid, genos[i].astype(np.float64)) for i in idx])
    smooth = (margins > 1e-3).all(axis=1)
    assert smooth.sum() >= 64
    gs = g[idx]
    assert np.all((np.abs(gs - Go).max(axis=1) <= grad_tol(Go))[smooth])
    # central differences of the FP64 oracle energy, h = 1e-4
    h = 1e-4
    checked = 0
    for b in np.nonzero(smooth)[0][:64]:
        g0 = genos[idx[b]].astype(np.float64)
        fd = np.zeros_like(g0)
        for j in range(len(g0)):
            a, c = g0.copy(), g0.copy()
            a[j] += h
            c[j] -= h
            fd[j] = (olig.score(ogrid, a, with_grad=False) - olig.score(ogrid, c, with_grad=False)) / (2 * h)
        if np.abs(fd - Go[b]).max() > 1e-2 * max(1.0, np.abs(Go[b]).max()):
            continue   # the +-h step crossed a cell face or the cutoff
        assert np.abs(gs[b] - fd).max() <= 2e-3 * max(1.0, np.abs(fd).max())
        checked += 1
    assert checked >= 32


def test_autograd_drives_an_optimiser(gpu, drug_system):
    """Plain torch.optim on genotypes through the differentiable energy lowers it."""
    L = capi.ligand_from(gpu, drug_system["lig"])
    G = capi.grids_from_maps(gpu, drug_system["maps"], drug_system["box"])
    x = torch.from_numpy(synth.make_genotypes(256, L.n_torsions, drug_system["box"], seed=7)).cuda()
    x.requires_grad_(True)
    opt = torch.optim.Adam([x], lr=0.05)
    E0 = autograd.score(x.detach(), gpu, G, L)
    for _ in range(50):
        opt.zero_grad()
        autograd.score(x, gpu, G, L).sum().backward()
        opt.step()
    E1 = autograd.score(x.detach(), gpu, G, L)
    assert torch.median(E1) < torch.median(E0)
    assert (E1 < E0).float().mean() > 0.8
