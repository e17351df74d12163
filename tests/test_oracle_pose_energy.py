"""Pins of the oracle's ligand model, pose builder, intramolecular energy and
analytic gradient (Section II-A: atoms, rotatable bonds and rigid motion as
degrees of freedom; Section IV-B: rotations applied in a fixed order)."""
import itertools

import numpy as np
import pytest

from paper_2203_02096_gb300 import synth

nx = pytest.importorskip("networkx")


def _graph(lig):
    g = nx.Graph()
    g.add_nodes_from(range(lig.n_atoms))
    g.add_edges_from(map(tuple, lig.bonds))
    return g


@pytest.mark.parametrize("n,t,seed", [(16, 4, 0), (40, 10, 1), (64, 16, 2), (10, 32, 3)])
def test_torsion_tree_and_pair_list_brute_force(oracle_mod, n, t, seed):
    """Moving set of torsion k = the side of bond k away from the root fragment
    (largest rigid fragment); pair list = pairs in different rigid fragments
    at >= 4 bonds apart.  Both recomputed here with networkx."""
    lig = synth.make_ligand(n, t, seed=seed)
    L = oracle_mod.OracleLigand(lig)
    g = _graph(lig)
    rigid = g.copy()
    rot_bonds = [tuple(b) for b, r in zip(lig.bonds, lig.rotatable) if r]
    rigid.remove_edges_from(rot_bonds)
    comps = sorted((sorted(c) for c in nx.connected_components(rigid)), key=lambda c: (-len(c), c[0]))
    frag = {a: fi for fi, c in enumerate(comps) for a in c}
    root_atoms = set(comps[0])
    assert L.n_frag == len(comps) and L.n_torsions == len(rot_bonds)
    for k, (u, v) in enumerate(rot_bonds):
        a, b, depth, moves = L.torsion(k)
        assert {a, b} == {u, v}
        cut = g.copy()
        cut.remove_edge(u, v)
        side_b = nx.node_connected_component(cut, b)
        assert not (side_b & root_atoms)
        assert set(np.nonzero(moves)[0]) == side_b
        # depth = rotatable bonds on the path root -> b
        path = nx.shortest_path(g, min(root_atoms), b)
        assert depth == sum(1 for e in zip(path, path[1:]) if tuple(e) in rot_bonds or tuple(e[::-1]) in rot_bonds)
    dist = dict(nx.all_pairs_shortest_path_length(g))
    expect = {(i, j) for i, j in itertools.combinations(range(n), 2) if frag[i] != frag[j] and dist[i][j] >= 4}
    assert {tuple(p) for p in L.pairs()} == expect


def test_identity_genotype_is_centred_reference(small_system):
    lig, L = small_system["lig"], small_system["olig"]
    geno = np.zeros(L.n_genes)
    geno[3] = 1.0
    x = L.pose(geno)
    assert np.allclose(x, lig.xyz - lig.xyz.mean(axis=0), atol=1e-13)


def test_quaternion_convention_matches_scipy(small_system):
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    lig, L = small_system["lig"], small_system["olig"]
    rng = np.random.default_rng(4)
    ref = lig.xyz - lig.xyz.mean(axis=0)
    for _ in range(5):
        q = rng.standard_normal(4) * 3.0          # unnormalised on purpose
        t = rng.uniform(-5, 5, 3)
        geno = np.concatenate([t, q, np.zeros(L.n_torsions)])
        qn = q / np.linalg.norm(q)
        R = Rot.from_quat([qn[1], qn[2], qn[3], qn[0]]).as_matrix()
        assert np.allclose(L.pose(geno), ref @ R.T + t, atol=1e-12)


def test_bond_lengths_preserved_and_2pi_identity(oracle_mod):
    lig = synth.make_ligand(40, 10, seed=7)
    L = oracle_mod.OracleLigand(lig)
    box = synth.make_box(64)
    genos = synth.make_genotypes(20, L.n_torsions, box, seed=1).astype(np.float64)
    d0 = np.linalg.norm(lig.xyz[lig.bonds[:, 0]] - lig.xyz[lig.bonds[:, 1]], axis=1)
    for gno in genos:
        x = L.pose(gno)
        d = np.linalg.norm(x[lig.bonds[:, 0]] - x[lig.bonds[:, 1]], axis=1)
        assert np.allclose(d, d0, atol=1e-12)
        g2 = gno.copy()
        g2[7:] += 2 * np.pi
        assert np.allclose(L.pose(g2), x, atol=1e-11)


def test_torsion_order_equivalence(oracle_mod):
    """Deepest-first with fixed axes == root-first with moving axes."""
    lig = synth.make_ligand(64, 16, seed=3)
    L = oracle_mod.OracleLigand(lig)
    rng = np.random.default_rng(0)
    for _ in range(10):
        tau = rng.uniform(-np.pi, np.pi, L.n_torsions)
        assert np.allclose(L.pose_local(tau, 0), L.pose_local(tau, 1), atol=1e-12)


def test_torsion_right_hand_rule(small_system):
    """A small positive tau_k moves atom i by tau * (u x (p_i - p_b)), u = unit(p_b - p_a)."""
    L = small_system["olig"]
    ref = L.pose_local(np.zeros(L.n_torsions))
    for k in range(L.n_torsions):
        a, b, _, moves = L.torsion(k)
        tau = np.zeros(L.n_torsions)
        tau[k] = 1e-7
        dx = (L.pose_local(tau) - ref) / 1e-7
        u = (ref[b] - ref[a]) / np.linalg.norm(ref[b] - ref[a])
        expect = np.cross(u, ref - ref[b]) * moves[:, None]
        assert np.allclose(dx, expect, atol=1e-6)


def test_intramolecular_energy_rigid_motion_invariance(oracle_mod):
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    lig = synth.make_ligand(40, 10, seed=11)
    L = oracle_mod.OracleLigand(lig)
    rng = np.random.default_rng(5)
    for _ in range(10):
        tau = rng.uniform(-np.pi, np.pi, L.n_torsions)
        x = L.pose_local(tau)
        e, f = L.intra_xyz(x, with_grad=True)
        R = Rot.random(random_state=int(rng.integers(1 << 30))).as_matrix()
        y = x @ R.T + rng.uniform(-20, 20, 3)
        assert L.intra_xyz(y) == pytest.approx(e, rel=1e-12, abs=1e-12)
        scale = np.abs(f).max() + 1e-30
        assert np.abs(f.sum(axis=0)).max() <= 1e-10 * scale * len(f)
        assert np.abs(np.cross(x, f).sum(axis=0)).max() <= 1e-10 * scale * len(f) * np.abs(x).max()


def _smooth_between(L, box, pairs, a, b):
    """True when no atom changes grid cell and no pair crosses the cutoff or
    the distance floor between genotypes a and b (E is smooth on the segment)."""
    xa, xb = L.pose(a), L.pose(b)
    lo = box.box_lo()
    ca = np.floor((xa - lo) / box.spacing)
    cb = np.floor((xb - lo) / box.spacing)
    if not np.array_equal(ca, cb):
        return False
    ra = np.linalg.norm(xa[pairs[:, 0]] - xa[pairs[:, 1]], axis=1)
    rb = np.linalg.norm(xb[pairs[:, 0]] - xb[pairs[:, 1]], axis=1)
    return np.array_equal(ra < 8.0, rb < 8.0) and np.array_equal(ra < 0.5, rb < 0.5)


@pytest.mark.parametrize("h,tol", [(1e-6, 1e-6), (1e-4, 1e-3)])
def test_gradient_matches_central_differences(small_system, h, tol):
    """Analytic genotype gradient vs central differences; a gene is skipped only
    when its +-h step carries an atom across a cell face or a pair across the
    cutoff or the distance floor (where E or its gradient is not smooth)."""
    L, grid, box = small_system["olig"], small_system["grid"], small_system["box"]
    pairs = L.pairs()
    genos = synth.make_genotypes(40, L.n_torsions, box, seed=9).astype(np.float64)
    genos[:, 0:3] = np.clip(genos[:, 0:3], box.box_lo() + 2.0, box.box_hi() - 2.0)
    checked = skipped = 0
    for g in genos:
        e, gr = L.score(grid, g)
        scale = max(1.0, np.max(np.abs(gr)))
        for j in range(len(g)):
            a, b = g.copy(), g.copy()
            a[j] += h
            b[j] -= h
            if not _smooth_between(L, box, pairs, a, b):
                skipped += 1
                continue
            fd = (L.score(grid, a, with_grad=False) - L.score(grid, b, with_grad=False)) / (2 * h)
            assert abs(fd - gr[j]) <= tol * scale, (j, fd, gr[j])
            checked += 1
    assert checked >= 0.8 * (checked + skipped)


def test_gradient_properties(small_system):
    """dE/dq is tangent to q (no radial part); E does not change with |q|."""
    L, grid, box = small_system["olig"], small_system["grid"], small_system["box"]
    for g in synth.make_genotypes(10, L.n_torsions, box, seed=2).astype(np.float64):
        e, gr = L.score(grid, g)
        assert abs(np.dot(gr[3:7], g[3:7])) <= 1e-9 * (np.abs(gr[3:7]).max() + 1e-30)
        g2 = g.copy()
        g2[3:7] *= 2.5
        e2, gr2 = L.score(grid, g2)
        assert e2 == pytest.approx(e, rel=1e-12)
        assert np.allclose(gr2[3:7] * 2.5, gr[3:7], rtol=1e-9, atol=1e-9 * np.abs(gr).max())


def test_score_batch_matches_single(small_system):
    L, grid, box = small_system["olig"], small_system["grid"], small_system["box"]
    genos = synth.make_genotypes(17, L.n_torsions, box, seed=8)
    E, G = L.score_batch(grid, genos, nthreads=3)
    for b in range(17):
        e, g = L.score(grid, genos[b].astype(np.float64))
        assert E[b] == e and np.array_equal(G[b], g)
