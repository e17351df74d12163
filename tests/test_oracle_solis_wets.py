"""Pins of the oracle's Solis-Wets local search (the miniapp's local search,
Section II-A; Solis and Wets 1981, adaptive random search with a bias term):
its step-scale schedule in closed form on a flat field, its deviates on a
linear field, monotone descent with the returned point's energy, and a whole
docking with it against an exhaustive enumeration."""
import numpy as np
import pytest

from paper_2203_02096_gb300 import synth

TYPES = ("C", "A", "N", "OA", "HD")


def _one_atom():
    return synth.Ligand(xyz=np.array([[0.3, -0.2, 0.1]]), types=np.array([0], np.int32),
                        charges=np.array([0.0]), bonds=np.zeros((0, 2), np.int32), rotatable=np.zeros(0, np.int32))


def _field_grid(oracle_mod, n, slope):
    """n^3 box, every map zero except the C type map = slope * (x - x_origin)."""
    box = synth.make_box(n, type_names=TYPES)
    maps = np.zeros((box.n_maps, n, n, n), np.float32)
    xs = np.arange(n) * box.spacing
    maps[list(box.map_types).index(0)] = (slope * xs)[None, None, :]
    return box, oracle_mod.OracleGrid(maps, box)


def _centre_geno(box):
    c = 0.5 * (box.box_lo() + box.box_hi())
    return np.array([c[0], c[1], c[2], 1.0, 0.0, 0.0, 0.0], np.float32)


def test_flat_field_contracts_to_the_lower_bound(oracle_mod):
    """On a constant energy every try fails, so the scale halves after every
    n_fail iterations; the search stops at the first iteration with
    rho < rho_lo: from 1 to 0.01 that is 7 halvings = 28 iterations, 56
    energies, and the point never moves."""
    box, grid = _field_grid(oracle_mod, 24, 0.0)
    L = oracle_mod.OracleLigand(_one_atom())
    x0 = _centre_geno(box)
    E, x, n, it, tr = oracle_mod.solis_wets(L, grid, x0, 1000, E0=0.0, seed=5)
    assert it == 28 and n == 56 and E == 0.0
    assert np.array_equal(x, x0)
    assert np.all(tr[:, 3] == 0) and np.all(tr[:, 0] == 0.0) and np.all(tr[:, 1] == 0.0)
    assert np.array_equal(tr[:, 2], np.repeat(0.5 ** np.arange(7), 4))
    # without E0 the start is evaluated once more
    assert oracle_mod.solis_wets(L, grid, x0, 1000, seed=5)[2] == 57


def test_linear_field_always_succeeds_and_expands(oracle_mod):
    """E = a * x along the box: x + xi or x - xi is always lower (unless
    xi_x = 0), so every iteration is a success, the scale doubles after each
    n_succ of them, and the energy falls at every step."""
    box, grid = _field_grid(oracle_mod, 96, 1.0)
    L = oracle_mod.OracleLigand(_one_atom())
    x0 = _centre_geno(box)
    E0 = L.score(grid, x0.astype(np.float64), with_grad=False)
    E, x, n, it, tr = oracle_mod.solis_wets(L, grid, x0, 10, E0=E0, seed=3)
    assert it == 10 and np.all(tr[:, 3] != 0)
    assert np.array_equal(tr[:, 2], [1, 1, 1, 1, 2, 2, 2, 2, 4, 4])
    acc = np.where(tr[:, 3] > 0, tr[:, 0], tr[:, 1])
    assert np.all(np.diff(np.concatenate([[E0], acc])) < 0) and E == acc[-1]
    assert np.all(x[0:3] >= box.box_lo()) and np.all(x[0:3] <= box.box_hi())
    # energies computed: one per forward success, two per backward success
    assert n == int(np.sum(tr[:, 3] > 0) + 2 * np.sum(tr[:, 3] < 0))


def test_first_deviate_uniform_within_the_step(oracle_mod):
    """First try of a search, bias 0: on E = x the energy change is xi_x,
    which must be uniform on [-rho0 * step_t, rho0 * step_t)."""
    box, grid = _field_grid(oracle_mod, 48, 1.0)
    L = oracle_mod.OracleLigand(_one_atom())
    x0 = _centre_geno(box)
    E0 = L.score(grid, x0.astype(np.float64), with_grad=False)
    sw = oracle_mod.make_sw(rho0=0.5, step_t=1.5)
    d = np.array([oracle_mod.solis_wets(L, grid, x0, 1, E0=E0, sw=sw, seed=11, entity=k)[4][0, 0] - E0
                  for k in range(2000)])
    assert np.all(np.abs(d) <= 0.75 + 1e-9)
    stats = pytest.importorskip("scipy.stats")
    assert stats.kstest(d, stats.uniform(loc=-0.75, scale=1.5).cdf).pvalue > 1e-3


def test_descends_and_returns_its_energy(small_system, oracle_mod):
    L, grid, box = small_system["olig"], small_system["grid"], small_system["box"]
    x0 = synth.make_genotypes(6, L.n_torsions, box, seed=8)
    for k, x in enumerate(x0):
        E0 = L.score(grid, x.astype(np.float64), with_grad=False)
        E, xb, n, it, tr = oracle_mod.solis_wets(L, grid, x, 200, E0=E0, seed=1, entity=k)
        assert E <= E0
        assert abs(np.linalg.norm(xb[3:7]) - 1) < 1e-6
        assert np.all(xb[7:] >= -np.float32(np.pi)) and np.all(xb[7:] < np.float32(np.pi))
        # the reported energy is the returned point's (up to the normalisation's rounding)
        assert abs(L.score(grid, xb.astype(np.float64), with_grad=False) - E) <= 1e-4 * max(1.0, abs(E))
        acc = np.where(tr[:, 3] > 0, tr[:, 0], np.where(tr[:, 3] < 0, tr[:, 1], np.nan))
        done = acc[~np.isnan(acc)]
        assert np.all(np.diff(np.concatenate([[E0], done])) < 0)
        assert (E == done[-1]) if len(done) else (E == E0)
        assert n == it + int(np.sum(tr[:, 3] <= 0))


def test_dock_with_solis_wets_beats_brute_force(oracle_mod):
    """The same 3-torsion bound as the ADADELTA docking: the best energy of
    each run is no worse than an exhaustive coarse enumeration in >= 90%."""
    lig = synth.make_ligand(8, 3, TYPES, seed=0)
    L = oracle_mod.OracleLigand(lig)
    rec = synth.make_receptor(300, inner=4.5, outer=12.0, type_names=TYPES, seed=2)
    box = synth.make_box(20, type_names=TYPES)
    grid = oracle_mod.OracleGrid(oracle_mod.build_maps(rec, box).astype(np.float32), box)
    lo, hi = box.box_lo(), box.box_hi()
    ts = [np.linspace(lo[a] + 0.5, hi[a] - 0.5, 5) for a in range(3)]
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    qs = Rot.create_group("O").as_quat()[:, [3, 0, 1, 2]]
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
    P = oracle_mod.make_params(pop_size=150, nruns=10, max_evals=40_000, ls_iters=100, ls_method=1)
    _, bestE, evals = oracle_mod.dock(L, grid, P, seed=0)
    assert np.all(evals >= 40_000)
    assert np.mean(bestE <= best + 1e-3) >= 0.9, (bestE, best)
    # deterministic and independent of the thread count
    _, bestE1, evals1 = oracle_mod.dock(L, grid, P, seed=0, nthreads=1)
    assert np.array_equal(bestE, bestE1) and np.array_equal(evals, evals1)


def test_bias_and_stream_layout_on_a_linear_field(oracle_mod):
    """On E = x the energy change of each try is its deviation's x part, so
    the bias rule (0.2 b + 0.4 xi forward, b - 0.4 xi backward, b / 2 on a
    failure) and the draw layout (word 0 of the Philox block
    (6 << 16 | 10 it, entity, gen, run)) can be read off the trace."""
    box, grid = _field_grid(oracle_mod, 96, 1.0)
    L = oracle_mod.OracleLigand(_one_atom())
    x0 = _centre_geno(box)
    E0 = L.score(grid, x0.astype(np.float64), with_grad=False)
    seed, run, gen, ent = 0x1234_5678_9ABC, 3, 7, 2
    E, x, n, it, tr = oracle_mod.solis_wets(L, grid, x0, 8, E0=E0, seed=seed, run=run, gen=gen, entity=ent)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    b, e = 0.0, E0
    for k in range(it):
        w = oracle_mod.philox([(6 << 16) | (10 * k), ent, gen, run], key)[0]
        u = 2.0 * ((int(w) >> 8) * 2.0 ** -24) - 1.0
        xi = b + tr[k, 2] * 1.0 * u
        assert abs((tr[k, 0] - e) - xi) < 1e-5
        if tr[k, 3] > 0:
            b, e = 0.2 * b + 0.4 * xi, tr[k, 0]
        elif tr[k, 3] < 0:
            assert abs((tr[k, 1] - e) + xi) < 1e-5
            b, e = b - 0.4 * xi, tr[k, 1]
        else:
            b = 0.5 * b
    assert np.sum(tr[:, 3] < 0) >= 1 and np.sum(tr[:, 3] > 0) >= 1   # both branches seen
