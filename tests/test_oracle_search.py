"""Pins of the oracle's random numbers, genetic operators, ADADELTA and the
whole Lamarckian GA (Section II-A: crossover, fitness-based selection, local
search on a random sample of each generation, Lamarckian write-back,
independent runs of population 150, best pose over all runs)."""
import os

import numpy as np
import pytest

from paper_2203_02096_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers(oracle_mod):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert list(oracle_mod.philox(v[0:4], v[4:6])) == v[6:10]


def test_init_population(small_system, oracle_mod):
    L, grid, box = small_system["olig"], small_system["grid"], small_system["box"]
    pop = oracle_mod.init_population(L.n_torsions, grid, seed=3, run=0, pop=4000)
    assert np.all(pop[:, 0:3] >= box.box_lo().astype(np.float32))
    assert np.all(pop[:, 0:3] <= box.box_hi().astype(np.float32))
    assert np.all(np.abs(np.linalg.norm(pop[:, 3:7], axis=1) - 1) < 1e-6)
    assert np.all(pop[:, 7:] >= -np.float32(np.pi)) and np.all(pop[:, 7:] < np.float32(np.pi))
    # uniform on S^3: zero mean, second moments 1/4 each, uncorrelated
    q = pop[:, 3:7].astype(np.float64)
    assert np.abs(q.mean(axis=0)).max() < 0.05
    cov = q.T @ q / len(q)
    assert np.abs(np.diag(cov) - 0.25).max() < 0.02 and np.abs(cov - np.diag(np.diag(cov))).max() < 0.02
    # deterministic; runs and seeds draw different streams
    assert np.array_equal(pop[:10], oracle_mod.init_population(L.n_torsions, grid, 3, 0, 10))
    assert not np.array_equal(pop[:10], oracle_mod.init_population(L.n_torsions, grid, 3, 1, 10))
    assert not np.array_equal(pop[:10], oracle_mod.init_population(L.n_torsions, grid, 4, 0, 10))


def _blocks(gene_idx_nt):
    nt = gene_idx_nt
    return [[0], [1], [2], [3, 4, 5, 6]] + [[7 + k] for k in range(nt)]


def test_ga_children_structure_and_rates(small_system, oracle_mod):
    L, grid = small_system["olig"], small_system["grid"]
    nt, popn = L.n_torsions, 150
    params = oracle_mod.make_params(pop_size=popn)
    rng = np.random.default_rng(0)
    blocks = _blocks(nt)
    wins = trials = cross = mut = nblk = 0
    for gen in range(1, 41):
        pop = oracle_mod.init_population(nt, grid, seed=gen, run=0, pop=popn)
        E = rng.standard_normal(popn).astype(np.float32).astype(np.float64)
        E[rng.integers(popn)] = E.min()          # a tie for the best
        kids, info, elite = oracle_mod.ga_children(nt, pop, E, seed=7, run=2, gen=gen, params=params)
        assert elite == int(np.argmin(E)) and np.array_equal(kids[0], pop[elite])
        for s in range(1, popn):
            p1, p2, lo, hi, mask = (int(v) for v in info[s])
            for b, genes in enumerate(blocks):
                src = pop[p2] if lo <= b < hi else pop[p1]
                if not (mask >> b) & 1:
                    assert np.array_equal(kids[s, genes], src[genes])
                elif b < 3:
                    assert abs(float(kids[s, b]) - float(src[b])) <= 2.0 + 1e-5
                elif b == 3:
                    assert abs(np.linalg.norm(kids[s, 3:7]) - 1) < 1e-6
                else:
                    assert -np.pi - 1e-6 <= kids[s, genes[0]] < np.pi + 1e-6
            cross += hi > lo
            mut += bin(mask).count("1")
            nblk += len(blocks)
        # selection pressure: re-derive which candidate was better from the drawn words
        for s in range(1, popn):
            for draw in (0, 1):
                w = oracle_mod.philox([(2 << 16) | draw, s, gen, 2], [7, 0])
                i1, i2 = (int(w[0] >> 8) * popn) >> 24, (int(w[1] >> 8) * popn) >> 24
                if i1 == i2 or E[i1] == E[i2]:
                    continue
                better = i1 if E[i1] < E[i2] else i2
                trials += 1
                wins += int(info[s][draw]) == better
    assert abs(wins / trials - 0.6) < 0.03
    # crossover happens with p=0.8 but draws lo==hi about 1/nblk of the time
    nb = len(blocks)
    assert abs(cross / (40 * 149) - 0.8 * (1 - 1 / nb)) < 0.03
    assert abs(mut / nblk - 0.02) < 0.005


def _ks_uniform(x, lo, hi):
    """Kolmogorov-Smirnov distance of a sample from U(lo, hi)."""
    x = np.sort(np.asarray(x, np.float64))
    n = len(x)
    F = np.clip((x - lo) / (hi - lo), 0.0, 1.0)
    i = np.arange(1, n + 1)
    return max(np.max(i / n - F), np.max(F - (i - 1) / n))


def _qmul(a, b):
    """Hamilton product of quaternions (w, x, y, z), rows of a and b."""
    aw, ax, ay, az = a.T
    bw, bx, by, bz = b.T
    return np.stack([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw], axis=1)


def test_ga_mutation_sizes(small_system, oracle_mod):
    """The sizes of the mutations (the reading of the GA's mutation operator):
    translation += U(-2, 2) A, torsion += U(-pi, pi) then wrapped,
    orientation <- normalise((1, v) (x) q) with v uniform in [-1, 1)^3.
    With crossover off and every block mutated, each child block is its first
    parent's block plus one mutation, so the deltas are recovered exactly
    (up to the FP32 rounding of the update) and compared, by Kolmogorov-
    Smirnov distance, with the distribution the reading states.  A range or
    scale slip (U(-1, 1), U(0, 2), a 10% stretch), a torsion delta drawn on
    [0, 2 pi) or the product taken as q (x) (1, v) moves a distance far beyond
    the 1e-3 significance level used (1.95 / sqrt(n))."""
    L, grid = small_system["olig"], small_system["grid"]
    nt, popn = L.n_torsions, 150
    params = oracle_mod.make_params(pop_size=popn, p_cross=0.0, p_mut=1.0)
    dt, dtau, v, ang = [], [], [], []
    for gen in range(1, 31):
        pop = oracle_mod.init_population(nt, grid, seed=100 + gen, run=0, pop=popn)
        E = np.arange(popn, dtype=np.float64)
        kids, info, _ = oracle_mod.ga_children(nt, pop, E, seed=5, run=1, gen=gen, params=params)
        p1 = info[1:, 0].astype(int)
        assert np.all(info[1:, 2] == info[1:, 3])                       # no crossover
        assert np.all(info[1:, 4] == (1 << (4 + nt)) - 1)              # every block mutated
        par, kid = pop[p1].astype(np.float64), kids[1:].astype(np.float64)
        dt.append((kid[:, 0:3] - par[:, 0:3]).ravel())
        dtau.append((((kid[:, 7:] - par[:, 7:]) + np.pi) % (2 * np.pi) - np.pi).ravel())
        conj = par[:, 3:7] * np.array([1.0, -1.0, -1.0, -1.0])
        r = _qmul(kid[:, 3:7], conj)                                    # = (1, v) / |(1, v)|
        assert np.all(r[:, 0] > 0)
        v.append(r[:, 1:4] / r[:, 0:1])
        ang.append(2.0 * np.arccos(np.clip(r[:, 0], -1.0, 1.0)))
    dt, dtau, v, ang = (np.concatenate(a) for a in (dt, dtau, v, ang))
    crit = lambda n: 1.95 / np.sqrt(n)                                  # noqa: E731
    assert _ks_uniform(dt, -2.0, 2.0) < crit(len(dt)), _ks_uniform(dt, -2.0, 2.0)
    assert dt.min() < -1.99 and dt.max() > 1.99 and np.abs(dt).max() <= 2.0 + 1e-5
    assert _ks_uniform(dtau, -np.pi, np.pi) < crit(len(dtau)), _ks_uniform(dtau, -np.pi, np.pi)
    assert np.abs(v).max() <= 1.0 + 1e-5 and np.abs(v).max() > 0.99
    for c in range(3):
        assert _ks_uniform(v[:, c], -1.0, 1.0) < crit(len(v)), (c, _ks_uniform(v[:, c], -1.0, 1.0))
    assert abs(np.corrcoef(v.T)[0, 1]) < 0.05 and abs(np.corrcoef(v.T)[1, 2]) < 0.05
    # the rotation angle 2 atan|v| against the angle of v drawn by numpy
    ref = np.random.default_rng(0).uniform(-1.0, 1.0, size=(400_000, 3))
    ref_ang = np.sort(2.0 * np.arctan(np.linalg.norm(ref, axis=1)))
    a = np.sort(ang)
    Fa = np.arange(1, len(a) + 1) / len(a)
    Fr = np.searchsorted(ref_ang, a, side="right") / len(ref_ang)
    assert np.max(np.abs(Fa - Fr)) < crit(len(a)), np.max(np.abs(Fa - Fr))


def test_ls_picks(oracle_mod):
    counts = np.zeros(150)
    for gen in range(2000):
        p = oracle_mod.ls_picks(150, 9, seed=1, run=0, gen=gen)
        assert len(set(p.tolist())) == 9 and p.min() >= 0 and p.max() < 150
        counts[p] += 1
    exp = 2000 * 9 / 150
    assert np.abs(counts - exp).max() < 5 * np.sqrt(exp)


def test_adadelta_closed_form_steps(oracle_mod):
    """First step -sqrt(eps)/sqrt((1-rho) g^2 + eps) g; second step from the
    recurrences written out for a scalar."""
    rho, eps = 0.8, 1e-2
    g1 = np.array([3.0, -0.5, 1e-3])
    x1, Eg2, Edx2 = oracle_mod.adadelta_step(np.zeros(3), g1, np.zeros(3), np.zeros(3), 0, rho, eps)
    d1 = -np.sqrt(eps) / np.sqrt((1 - rho) * g1 ** 2 + eps) * g1
    assert np.allclose(x1, d1, rtol=1e-14)
    g2 = np.array([1.0, 2.0, -4.0])
    x2, _, _ = oracle_mod.adadelta_step(x1, g2, Eg2, Edx2, 0, rho, eps)
    eg2 = rho * (1 - rho) * g1 ** 2 + (1 - rho) * g2 ** 2
    edx2 = (1 - rho) * d1 ** 2
    d2 = -np.sqrt(edx2 + eps) / np.sqrt(eg2 + eps) * g2
    assert np.allclose(x2, x1 + d2, rtol=1e-14)


def test_adadelta_descends_far_from_minimum(oracle_mod):
    """Far from the minimum of a bowl every step moves downhill along each
    coordinate (ADADELTA steps are bounded by sqrt(E[dx^2]+eps)/sqrt(E[g^2]+eps)|g|);
    on a torsion gene the update wraps into [-pi, pi)."""
    A = np.array([1.0, 4.0, 0.25, 9.0])
    x = np.array([30.0, -20.0, 50.0, 10.0])
    Eg2, Edx2 = np.zeros(4), np.zeros(4)
    for _ in range(20):
        xn, Eg2, Edx2 = oracle_mod.adadelta_step(x, A * x, Eg2, Edx2, 0, 0.8, 1e-2)
        assert np.all(np.abs(xn) < np.abs(x))
        x = xn
    g = np.zeros(8)
    g[7] = -1.0
    x = np.zeros(8)
    x[7] = np.pi - 0.05
    xw, _, _ = oracle_mod.adadelta_step(x, g, np.zeros(8), np.zeros(8), 1, 0.8, 1e-2)
    step = np.sqrt(1e-2) / np.sqrt(0.2 + 1e-2)
    assert xw[7] == pytest.approx(np.pi - 0.05 + step - 2 * np.pi, rel=1e-12)


def test_local_search_tracks_best(small_system, oracle_mod):
    L, grid, box = small_system["olig"], small_system["grid"], small_system["box"]
    x0 = oracle_mod.init_population(L.n_torsions, grid, seed=5, run=0, pop=3)
    for x in x0:
        E, xb, trace = oracle_mod.local_search(L, grid, x, iters=100)
        assert E == trace.min() and trace[0] == pytest.approx(L.score(grid, x.astype(np.float64), with_grad=False))
        assert trace.min() < trace[0]
        assert L.score(grid, xb.astype(np.float64), with_grad=False) == pytest.approx(E, rel=1e-4, abs=1e-3)


def test_dock_determinism_and_accounting(small_system, oracle_mod):
    L, grid = small_system["olig"], small_system["grid"]
    P = oracle_mod.make_params(pop_size=50, nruns=3, max_evals=3000, ls_iters=20)
    a = oracle_mod.dock(L, grid, P, seed=11, nthreads=1)
    b = oracle_mod.dock(L, grid, P, seed=11, nthreads=3)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
    per_gen = 49 + P.ls_count * 20
    assert np.all(a[2] >= 3000) and np.all(a[2] < 3000 + per_gen) and np.all((a[2] - 50) % per_gen == 0)
    for r in range(3):
        assert a[1][r] == pytest.approx(L.score(grid, a[0][r].astype(np.float64), with_grad=False), rel=1e-12)


def test_search_beats_brute_force_enumeration(oracle_mod):
    """3-torsion ligand: the LGA's best energy is no worse than the best of an
    exhaustive coarse enumeration of (translation, orientation, torsions) in
    at least 90% of runs."""
    types = ("C", "A", "N", "OA", "HD")
    lig = synth.make_ligand(8, 3, types, seed=0)
    L = oracle_mod.OracleLigand(lig)
    assert L.n_torsions == 3
    rec = synth.make_receptor(300, inner=4.5, outer=12.0, type_names=types, seed=2)
    box = synth.make_box(20, type_names=types)
    grid = oracle_mod.OracleGrid(oracle_mod.build_maps(rec, box).astype(np.float32), box)
    lo, hi = box.box_lo(), box.box_hi()
    ts = [np.linspace(lo[a] + 0.5, hi[a] - 0.5, 5) for a in range(3)]
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    qs = Rot.create_group("O").as_quat()[:, [3, 0, 1, 2]]        # 24 rotations, (w,x,y,z)
    taus = np.linspace(-np.pi, np.pi, 8, endpoint=False)
    T = np.stack(np.meshgrid(*ts, indexing="ij"), -1).reshape(-1, 3)
    TAU = np.stack(np.meshgrid(taus, taus, taus, indexing="ij"), -1).reshape(-1, 3)
    best = np.inf
    for t in T:
        g = np.zeros((len(qs) * len(TAU), 10), dtype=np.float32)
        g[:, 0:3] = t
        g[:, 3:7] = np.repeat(qs, len(TAU), axis=0)
        g[:, 7:10] = np.tile(TAU, (len(qs), 1))
        best = min(best, L.score_batch(grid, g, with_grad=False).min())
    P = oracle_mod.make_params(pop_size=150, nruns=10, max_evals=40_000, ls_iters=100)
    _, bestE, _ = oracle_mod.dock(L, grid, P, seed=0)
    assert np.mean(bestE <= best + 1e-3) >= 0.9, (bestE, best)
