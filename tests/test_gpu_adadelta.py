"""ADADELTA parity, element by element (the memetic local search of the
paper's Section II-A, read as ADADELTA, Zeiler 2012).

* The step alone: dock_adadelta_step (the update the local-search kernel
  applies after each evaluation) against orc_adadelta_step on the same FP32
  inputs, gene by gene, over gradients and running averages spanning eight
  decades, torsions crossing +-pi included.
* The chain: dock_local_search_trace records, at every iteration k, the
  point x_k it evaluated, its gradient g_k and energy E_k.  At every k the
  oracle evaluated at the same x_k gives E and the gradient (stated
  tolerance in the relaxed regime), and the oracle's step from x_k with g_k
  -- its running averages replayed from g_0..g_k -- gives x_{k+1} to FP32
  rounding.  So each iteration of the device chain is checked against the
  oracle; a sign, rho/eps or wrap mistake anywhere fails it.
* Whole trajectories from the same start agree only for the first steps:
  FP32 and FP64 chains part ways geometrically even from docked poses
  (measured on the drug-size ligand: 7e-5 after 2 steps, 4e-3 after 5, 0.8
  after 7).  The first step, whose only error source is the gradient, is
  compared with a bound propagated from the gradient tolerance.
* The point returned is the best of the chain (strictly lowest energy,
  first on ties), quaternion normalised."""
import numpy as np
import pytest
import torch

from paper_2203_02096_gb300 import capi, synth
from tests.tolerances import G_ABS, G_REL, energy_tol, grad_block_errors, grad_tol, gene_blocks

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -23          # FP32 unit roundoff x 2 (one ulp of 1.0)
RELAXED_E_MAX = 50.0
MARGIN = 1e-4


def _circ(d):
    """Differences of torsion genes taken on the circle."""
    return (d + np.pi) % (2 * np.pi) - np.pi


def _diff(a, b):
    d = np.asarray(a, np.float64) - np.asarray(b, np.float64)
    d[..., 7:] = _circ(d[..., 7:])
    return d


def test_step_matches_oracle(gpu, oracle_mod):
    rng = np.random.default_rng(11)
    B, nt = 4096, 10
    Gn = 7 + nt
    x = rng.uniform(-3.6, 3.6, (B, Gn)).astype(np.float32)
    x[:, 0:3] = rng.uniform(-40.0, 40.0, (B, 3))
    x[: B // 4, 7:] = np.float32(np.pi) - rng.uniform(0, 0.3, (B // 4, nt)).astype(np.float32)   # near +pi
    x[B // 4: B // 2, 7:] = -np.float32(np.pi) + rng.uniform(0, 0.3, (B // 4, nt)).astype(np.float32)
    g = (rng.standard_normal((B, Gn)) * 10.0 ** rng.uniform(-4, 4, (B, Gn))).astype(np.float32)
    Eg2 = (rng.uniform(0, 1, (B, Gn)) * 10.0 ** rng.uniform(-5, 5, (B, Gn))).astype(np.float32)
    Edx2 = (rng.uniform(0, 1, (B, Gn)) * 10.0 ** rng.uniform(-5, 0, (B, Gn))).astype(np.float32)
    Eg2[:64] = 0.0
    Edx2[:64] = 0.0          # first iteration of a chain: state reset
    g[64:80] = 0.0
    for rho, eps in [(np.float32(0.8), np.float32(1e-2)), (np.float32(0.95), np.float32(1e-6))]:
        # the oracle takes the FP32 parameters the device holds
        tx, tg, te, td = (torch.from_numpy(a.copy()).cuda() for a in (x, g, Eg2, Edx2))
        capi.dock_adadelta_step(gpu, tx, tg, te, td, rho=rho, eps=eps)
        gx, ge, gd = (t.cpu().numpy().astype(np.float64) for t in (tx, te, td))
        ox, oe, od = (np.zeros((B, Gn)) for _ in range(3))
        for b in range(B):
            ox[b], oe[b], od[b] = oracle_mod.adadelta_step(x[b], g[b], Eg2[b], Edx2[b], nt, rho=rho, eps=eps)
        # Eg2: two products and an fma of positive terms (4 ulp); dx: sqrt,
        # rsqrt (2 ulp) and two products (4 ulp), so Edx2 (16 ulp) and x
        # (half an ulp of the result, 8 ulp of the step); a wrapped torsion
        # also carries the FP32 rounding of 2 pi (1.7e-7, under an ulp of pi)
        assert np.all(np.abs(ge - oe) <= 4 * U32 * np.abs(oe)), np.max(np.abs(ge - oe) / np.maximum(oe, 1e-300))
        assert np.all(np.abs(gd - od) <= 16 * U32 * np.abs(od)), np.max(np.abs(gd - od) / np.maximum(od, 1e-300))
        step = _diff(ox, x)
        allowed = 2 * np.spacing(np.abs(ox).astype(np.float32)).astype(np.float64) + 8 * U32 * np.abs(step)
        assert np.all(np.abs(_diff(gx, ox)) <= allowed), np.max(np.abs(_diff(gx, ox)) / allowed)
        assert np.all((gx[:, 7:] >= -np.pi - 1e-6) & (gx[:, 7:] < np.pi + 1e-6))
        # the near-pi starts do cross the boundary in both directions
        crossed = np.sign(gx[: B // 2, 7:]) != np.sign(x[: B // 2, 7:])
        assert crossed.sum() > 100
        # zero gradient: no move
        assert np.all(np.abs(_diff(gx[64:80], x[64:80])) <= 2 * np.spacing(np.float32(np.pi)))


@pytest.fixture(scope="module")
def docked_starts(oracle_mod, drug_system):
    """Relaxed start points: the best pose of each run of an oracle docking of
    the drug-size ligand, plus one start per direction whose first step
    carries a torsion across +pi / -pi."""
    olig, ogrid = drug_system["olig"], drug_system["grid"]
    P = oracle_mod.make_params(pop_size=150, nruns=10, max_evals=100_000, ls_iters=300)
    docked, _, _ = oracle_mod.dock(olig, ogrid, P, 21)
    starts = [d for d in docked]
    base = docked[0].astype(np.float64)
    found = set()
    for k in range(olig.n_torsions):
        for side in (+1, -1):
            if side in found:
                continue
            x = base.copy()
            x[7 + k] = side * (np.pi - 0.02)
            x = x.astype(np.float32)
            _, gx = olig.score(ogrid, x.astype(np.float64))
            first = -np.sqrt(1e-2) / np.sqrt(0.2 * gx[7 + k] ** 2 + 1e-2) * gx[7 + k]
            if side * first > 0.05:      # the first step moves it over the boundary
                starts.append(x)
                found.add(side)
    assert found == {+1, -1}
    return np.array(starts, dtype=np.float32)


def _oracle_at(olig, ogrid, xs):
    E, Gr = zip(*[olig.score(ogrid, x.astype(np.float64)) for x in xs])
    M = np.stack([olig.margins(ogrid, x.astype(np.float64)) for x in xs])
    return np.array(E), np.array(Gr), M


@pytest.mark.parametrize("rho,eps", [(0.8, 1e-2), (0.95, 1e-6)])
@pytest.mark.parametrize("threads", [32, 128, 256])
def test_chain_step_by_step(gpu, oracle_mod, drug_system, docked_starts, threads, rho, eps):
    L = capi.ligand_from(gpu, drug_system["lig"])
    G = capi.grids_from_maps(gpu, drug_system["maps"], drug_system["box"])
    olig, ogrid = drug_system["olig"], drug_system["grid"]
    nt, iters = olig.n_torsions, 20
    x0 = torch.from_numpy(docked_starts).cuda()
    _, _, xt, gt, Et = capi.dock_local_search_trace(gpu, G, L, x0, iters, rho=rho, eps=eps, threads=threads)
    xt, gt, Et = xt.cpu().numpy(), gt.cpu().numpy().astype(np.float64), Et.cpu().numpy().astype(np.float64)
    assert np.array_equal(xt[:, 0], docked_starts)
    n_relaxed = n_all = 0
    worst = dict(E=0.0, g=0.0, x=0.0)
    for b in range(len(docked_starts)):
        Eo, Go, M = _oracle_at(olig, ogrid, xt[b])
        # energies: every iterate at the stated tolerance
        e_ok = M[:, 1] > MARGIN
        eerr = np.abs(Et[b] - Eo) / energy_tol(Eo)
        assert np.all(eerr[e_ok] <= 1.0), (b, np.argmax(eerr), Et[b][eerr > 1], Eo[eerr > 1])
        worst["E"] = max(worst["E"], eerr[e_ok].max())
        # gradients: stated per-block tolerance in the relaxed regime, the
        # clash-pose tolerance elsewhere
        g_ok = (M > MARGIN).all(axis=1)
        relaxed = g_ok & (Eo <= RELAXED_E_MAX)
        gerr, gtol = grad_block_errors(gt[b], Go, nt)
        r = gerr / gtol
        assert np.all(r[relaxed] <= 1.0), (b, np.argwhere(r > 1)[:4])
        clash = g_ok & ~relaxed
        assert np.all(np.abs(gt[b] - Go).max(axis=1)[clash] <= grad_tol(Go)[clash])
        if relaxed.any():
            worst["g"] = max(worst["g"], r[relaxed].max())
        n_relaxed += int(relaxed.sum())
        n_all += iters
        # steps: x_{k+1} = the oracle's ADADELTA step from x_k with the
        # device's gradient g_k, running averages replayed from g_0..g_k.
        # The device keeps its running averages in FP32: a sum of positive
        # terms, so each step adds a few ulp to their relative error (Eg2 2,
        # Edx2 its own plus Eg2's plus 8 through dx^2), which reaches the
        # step as half their sum: (16 + 4k + k^2) ulp of dx after k steps,
        # plus 2 ulp of x (rounding of x + dx, and of 2 pi in a wrap).
        Eg2 = np.zeros(7 + nt)
        Edx2 = np.zeros(7 + nt)
        for k in range(iters - 1):
            xp, Eg2, Edx2 = oracle_mod.adadelta_step(xt[b, k], gt[b, k], Eg2, Edx2, nt, rho=np.float32(rho),
                                                     eps=np.float32(eps))
            step = _diff(xp, xt[b, k])
            allowed = (2 * np.spacing(np.abs(xp).astype(np.float32)).astype(np.float64)
                       + (16 + 4 * k + k * k) * U32 * np.abs(step))
            dx = np.abs(_diff(xt[b, k + 1], xp))
            assert np.all(dx <= allowed), (b, k, np.argmax(dx / allowed), np.max(dx / allowed))
            worst["x"] = max(worst["x"], np.max(dx / allowed))
    assert n_relaxed >= n_all // 4, (n_relaxed, n_all)
    if eps == 1e-2:  # the last two starts carry a torsion across +pi and -pi in their first step
        tau0 = docked_starts[-2:, 7:]
        tau1 = xt[-2:, 1, 7:]
        assert np.sum(np.sign(tau0) != np.sign(tau1)) >= 2 and np.all(np.abs(tau1) <= np.pi + 1e-6)
    print(f"\nthreads {threads} rho {rho} eps {eps}: {n_all} iterates ({n_relaxed} relaxed); worst error/tolerance: "
          f"E {worst['E']:.3f}, gradient {worst['g']:.3f}, step {worst['x']:.3f}")


@pytest.mark.parametrize("iters", [2, 5, 20])
def test_returns_best_of_chain(gpu, oracle_mod, drug_system, docked_starts, iters):
    L = capi.ligand_from(gpu, drug_system["lig"])
    G = capi.grids_from_maps(gpu, drug_system["maps"], drug_system["box"])
    olig, ogrid = drug_system["olig"], drug_system["grid"]
    xb, Eb, xt, _, Et = capi.dock_local_search_trace(gpu, G, L, torch.from_numpy(docked_starts).cuda(), iters)
    plain_x, plain_E = capi.dock_local_search(gpu, G, L, torch.from_numpy(docked_starts).cuda(), iters)
    assert torch.equal(xb, plain_x) and torch.equal(Eb, plain_E)   # tracing changes nothing
    xb, Eb, xt, Et = xb.cpu().numpy(), Eb.cpu().numpy(), xt.cpu().numpy(), Et.cpu().numpy()
    for b in range(len(docked_starts)):
        k = int(np.argmin(Et[b]))                       # first of the lowest
        assert Eb[b] == Et[b, k]
        want = xt[b, k].astype(np.float64)
        want[3:7] /= np.linalg.norm(want[3:7])
        assert np.all(np.abs(xb[b] - want) <= np.spacing(np.abs(want).astype(np.float32)) * 2), (b, k)
        # the choice is right by the oracle's energies too, up to the tolerance
        Eo = np.array([olig.score(ogrid, x.astype(np.float64), with_grad=False) for x in xt[b]])
        assert Eo[k] <= Eo.min() + 2 * energy_tol(np.array([Eo.min()]))[0]


def test_first_step_trajectory(gpu, oracle_mod, drug_system, docked_starts):
    """Two iterations from the same start: x_1 of the device against x_1 of
    the FP64 oracle chain.  Its error comes from the gradient at x_0 only;
    |d dx_j / d g_j| <= |dx_j / g_j|, so it is bounded by |dx_j / g_j| times
    the gradient tolerance of j's block (the stated one at a relaxed start,
    the clash-pose one at a start in clash), plus rounding."""
    L = capi.ligand_from(gpu, drug_system["lig"])
    G = capi.grids_from_maps(gpu, drug_system["maps"], drug_system["box"])
    olig, ogrid = drug_system["olig"], drug_system["grid"]
    nt = olig.n_torsions
    _, _, xt, _, _ = capi.dock_local_search_trace(gpu, G, L, torch.from_numpy(docked_starts).cuda(), 2)
    xt = xt.cpu().numpy()
    checked = 0
    for b, x0 in enumerate(docked_starts):
        if not (olig.margins(ogrid, x0.astype(np.float64)) > MARGIN).all():
            continue                     # gradient discontinuity within reach of FP32 rounding
        checked += 1
        e0, g0 = olig.score(ogrid, x0.astype(np.float64))
        x1, _, _ = oracle_mod.adadelta_step(x0, g0, np.zeros(7 + nt), np.zeros(7 + nt), nt)
        step = _diff(x1, x0)
        gtol = np.zeros(7 + nt)
        for sl in gene_blocks(nt):
            gtol[sl] = G_REL * np.linalg.norm(g0[sl]) + G_ABS
        if e0 > RELAXED_E_MAX:
            gtol[:] = grad_tol(g0[None])[0]
        ratio = np.divide(np.abs(step), np.abs(g0), out=np.zeros_like(step), where=g0 != 0)
        allowed = ratio * gtol + np.spacing(np.abs(x1).astype(np.float32)) + 64 * U32 * np.abs(step)
        assert np.all(np.abs(_diff(xt[b, 1], x1)) <= allowed), (b, np.max(np.abs(_diff(xt[b, 1], x1)) / allowed))
    assert checked >= len(docked_starts) - 2


def _near_reference_starts(olig, box, n, seed):
    """Starts around the ligand's own conformation (small torsion offsets,
    random orientation, near the box centre) and two random genotypes of the
    initial population (deep intramolecular clash)."""
    rng = np.random.default_rng(seed)
    centre = (np.asarray(box.box_lo()) + np.asarray(box.box_hi())) / 2
    X = np.zeros((n, olig.n_genes), np.float32)
    X[:, 0:3] = centre + rng.uniform(-1.5, 1.5, (n, 3))
    q = rng.standard_normal((n, 4))
    X[:, 3:7] = q / np.linalg.norm(q, axis=1, keepdims=True)
    X[:, 7:] = rng.uniform(-0.4, 0.4, (n, olig.n_torsions))
    return X


@pytest.mark.parametrize("threads", [32, 64, 128, 256])
@pytest.mark.parametrize("n,t", [(108, 31), (255, 32)])
def test_chain_large_ligands(gpu, oracle_mod, drug_system, n, t, threads):
    """The team evaluator at the largest sizes, every team width: a thread
    places and grid-scores several atoms, each warp runs several pair steps,
    the torsion tree is 32 lanes deep.  Each iterate of a traced chain is
    checked against the oracle: energy (stated tolerance at E <= 50, the
    clash-pose one above), gradient (per block at E <= 50, clash-pose
    above) where no discontinuity is within reach of FP32 rounding, and the
    step x_k -> x_{k+1} to FP32 rounding."""
    lig = synth.make_ligand(n, t, seed=n)
    olig, ogrid = oracle_mod.OracleLigand(lig), drug_system["grid"]
    nt, iters = olig.n_torsions, 6
    starts = np.concatenate([_near_reference_starts(olig, drug_system["box"], 12, seed=n),
                             oracle_mod.init_population(nt, ogrid, n, 0, 2)])
    L = capi.ligand_from(gpu, lig)
    G = capi.grids_from_maps(gpu, drug_system["maps"], drug_system["box"])
    _, _, xt, gt, Et = capi.dock_local_search_trace(gpu, G, L, torch.from_numpy(starts).cuda(), iters,
                                                    threads=threads)
    xt, gt, Et = xt.cpu().numpy(), gt.cpu().numpy().astype(np.float64), Et.cpu().numpy().astype(np.float64)
    assert np.array_equal(xt[:, 0], starts)
    n_grad = n_relaxed = 0
    for b in range(len(starts)):
        Eo, Go, M = _oracle_at(olig, ogrid, xt[b])
        F = np.stack([olig.atom_forces(ogrid, x.astype(np.float64))[1] for x in xt[b]])
        relaxed = Eo <= RELAXED_E_MAX
        e_ok = M[:, 1] > MARGIN
        etol = np.where(relaxed, energy_tol(Eo), energy_tol(Eo, F))
        assert np.all(np.abs(Et[b] - Eo)[e_ok] <= etol[e_ok]), (b, Et[b], Eo)
        g_ok = (M > MARGIN).all(axis=1)
        gerr, gtol = grad_block_errors(gt[b], Go, nt)
        assert np.all((gerr <= gtol)[g_ok & relaxed]), (b, np.argwhere(gerr > gtol)[:4])
        clash = g_ok & ~relaxed
        assert np.all(np.abs(gt[b] - Go).max(axis=1)[clash] <= grad_tol(Go)[clash]), b
        n_grad += int(g_ok.sum())
        n_relaxed += int((g_ok & relaxed).sum())
        Eg2, Edx2 = np.zeros(7 + nt), np.zeros(7 + nt)
        for k in range(iters - 1):
            xp, Eg2, Edx2 = oracle_mod.adadelta_step(xt[b, k], gt[b, k], Eg2, Edx2, nt, rho=np.float32(0.8),
                                                     eps=np.float32(1e-2))
            allowed = (2 * np.spacing(np.abs(xp).astype(np.float32)).astype(np.float64)
                       + (16 + 4 * k + k * k) * U32 * np.abs(_diff(xp, xt[b, k])))
            assert np.all(np.abs(_diff(xt[b, k + 1], xp)) <= allowed), (b, k)
    # a 255-atom pose has ~760 coordinates and ~32k pairs: two thirds of its
    # iterates have an atom within 1e-4 A of a cell face or a pair that close
    # to the cutoff (a fifth at 108 atoms); enough others remain
    assert n_grad >= len(starts) * iters // 5, n_grad
    print(f"\n{n} atoms / {t} torsions, {threads} threads: {n_grad} of {len(starts) * iters} iterates "
          f"gradient-checked ({n_relaxed} at E <= {RELAXED_E_MAX})")


def test_new_entry_points_reject_bad_arguments(gpu, drug_system):
    """dock_adadelta_step and dock_local_search_trace: argument errors come
    back as DOCK_ERR_INVALID, an empty batch is a no-op, and the largest
    genotype (32 torsions, 39 genes) steps like any other."""
    x = torch.zeros((4, 17), dtype=torch.float32, device="cuda")
    g, a, b = torch.ones_like(x), torch.zeros_like(x), torch.zeros_like(x)
    for kw in (dict(rho=1.0), dict(rho=-0.1), dict(eps=0.0)):
        with pytest.raises(capi.DockError, match="INVALID"):
            capi.dock_adadelta_step(gpu, x, g, a, b, **kw)
    bad = torch.zeros((4, 6), dtype=torch.float32, device="cuda")
    with pytest.raises(capi.DockError, match="INVALID"):
        capi.dock_adadelta_step(gpu, bad, torch.ones_like(bad), torch.zeros_like(bad), torch.zeros_like(bad))
    big = torch.zeros((4, 40), dtype=torch.float32, device="cuda")
    with pytest.raises(capi.DockError, match="INVALID"):
        capi.dock_adadelta_step(gpu, big, torch.ones_like(big), torch.zeros_like(big), torch.zeros_like(big))
    empty = torch.zeros((0, 17), dtype=torch.float32, device="cuda")
    capi.dock_adadelta_step(gpu, empty, empty.clone(), empty.clone(), empty.clone())
    x39 = torch.zeros((3, 39), dtype=torch.float32, device="cuda")
    capi.dock_adadelta_step(gpu, x39, torch.ones_like(x39), torch.zeros_like(x39), torch.zeros_like(x39))
    assert torch.all(x39 < 0)     # a positive gradient moves every gene down
    L = capi.ligand_from(gpu, drug_system["lig"])
    G = capi.grids_from_maps(gpu, drug_system["maps"], drug_system["box"])
    x0 = torch.from_numpy(synth.make_genotypes(2, L.n_torsions, drug_system["box"], seed=1)).cuda()
    xb, Eb = torch.empty_like(x0), torch.empty(2, device="cuda")
    xt = torch.empty((2, 3, L.n_genes), device="cuda")
    rc = gpu.lib.dock_local_search_trace(gpu.h, G.h, L.h, capi._ptr(x0), 2, 3, 0.8, 0.01, 0, capi._ptr(xb),
                                         capi._ptr(Eb), capi._ptr(xt), None, None, capi._stream(None))
    assert capi.ERRORS.get(rc) == "DOCK_ERR_INVALID", rc
