"""Pins of the oracle's receptor maps and grid reads (the particle-grid
interaction of Section II-A): maps agree with a direct sum of pair energies,
trilinear interpolation is exact at nodes and on linear fields, and the
out-of-box treatment behaves as its reading states."""
import numpy as np
import pytest

from paper_2203_02096_gb300 import synth


def _tiny_receptor(center, n=6, seed=5):
    rng = np.random.default_rng(seed)
    xyz = np.asarray(center) + rng.uniform(-4.0, 4.0, size=(n, 3))
    types = rng.integers(0, 7, size=n).astype(np.int32)
    q = rng.uniform(-0.4, 0.4, size=n)
    return synth.Receptor(xyz=xyz, types=types, charges=q)


def test_map_read_equals_direct_pair_sum(oracle_mod):
    """M_t(p) + q E(p) + |q| D(p) at a point equals the sum over receptor atoms of
    the intramolecular pair energy (same force field), when every receptor atom
    is within the 8 A cutoff and no cap is active: the map split is exact."""
    p = np.array([1.0, 2.0, -1.5])
    rec = _tiny_receptor(p)
    assert np.all(np.linalg.norm(rec.xyz - p, axis=1) < 8.0)
    map_types = list(range(7))
    vals = oracle_mod.map_values_at(rec, map_types, p[None])[0]
    for t in range(7):
        for q in (-0.37, 0.0, 0.21):
            direct = sum(oracle_mod.pair_energy(t, q, int(rec.types[j]), float(rec.charges[j]),
                                                float(np.linalg.norm(rec.xyz[j] - p)))[0] for j in range(len(rec.types)))
            assert vals[t] + q * vals[7] + abs(q) * vals[8] == pytest.approx(direct, rel=1e-12, abs=1e-12)


def test_type_maps_are_capped(oracle_mod):
    p = np.array([0.0, 0.0, 0.0])
    rec = synth.Receptor(xyz=p[None] + 0.1, types=np.array([0], np.int32), charges=np.array([0.1]))
    vals = oracle_mod.map_values_at(rec, [0, 6], p[None])[0]
    assert vals[0] == 1e5 and vals[1] == 1e5


def test_build_maps_layout(oracle_mod):
    """[map][z][y][x] layout with node (i,j,k) at origin + (i,j,k)*h."""
    rec = _tiny_receptor((0.0, 0.0, 0.0), n=30, seed=2)
    box = synth.GridBox(dims=(5, 6, 7), origin=(-1.0, -1.5, -2.0), spacing=0.375, map_types=(0, 3, 6))
    maps = oracle_mod.build_maps(rec, box, nthreads=3)
    assert maps.shape == (5, 7, 6, 5)
    rng = np.random.default_rng(0)
    for _ in range(10):
        i, j, k = rng.integers(5), rng.integers(6), rng.integers(7)
        p = np.asarray(box.origin) + np.array([i, j, k]) * box.spacing
        v = oracle_mod.map_values_at(rec, box.map_types, p[None])[0]
        assert np.array_equal(maps[:, k, j, i], v)


def _linear_grid(oracle_mod, a, b, c, d, dims=(6, 7, 8), h=0.5, origin=(-1.0, 0.25, 2.0)):
    nx, ny, nz = dims
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    field = (a * i + b * j + c * k + d).astype(np.float32)   # dyadic -> exact in FP32
    maps = np.stack([field, 2 * field, -field])
    box = synth.GridBox(dims=dims, origin=origin, spacing=h, map_types=(0,))
    return oracle_mod.OracleGrid(maps, box), box


def test_interp_exact_on_nodes(small_system):
    g = small_system["grid"]
    box = small_system["box"]
    rng = np.random.default_rng(1)
    for _ in range(50):
        m = int(rng.integers(g.maps.shape[0]))
        i, j, k = (int(rng.integers(n)) for n in box.dims)
        p = np.asarray(box.origin) + np.array([i, j, k]) * box.spacing
        v, _ = g.interp(m, *p)
        assert v == pytest.approx(float(g.maps[m, k, j, i]), rel=1e-13, abs=1e-13)


def test_interp_exact_on_linear_field(oracle_mod):
    a, b, c, d = 0.5, -0.25, 1.75, 3.0
    g, box = _linear_grid(oracle_mod, a, b, c, d)
    rng = np.random.default_rng(2)
    lo, hi = box.box_lo(), box.box_hi()
    for _ in range(200):
        x = rng.uniform(lo, hi)
        u = (x - lo) / box.spacing
        v, gr = g.interp(0, *x)
        assert v == pytest.approx(a * u[0] + b * u[1] + c * u[2] + d, rel=1e-13, abs=1e-12)
        assert np.allclose(gr, np.array([a, b, c]) / box.spacing, rtol=1e-12, atol=1e-12)


def test_out_of_box_clamp_and_penalty(oracle_mod):
    """Outside the box: the read is that of the clamped point, its gradient along
    a clamped axis is zero, and 10 kcal/mol/A^2 * d^2 is added per axis."""
    a, b, c, d = 0.5, -0.25, 1.75, 3.0
    g, box = _linear_grid(oracle_mod, a, b, c, d)
    lo, hi = box.box_lo(), box.box_hi()
    x = np.array([lo[0] - 0.7, 0.5 * (lo[1] + hi[1]), hi[2] + 0.3])
    xc = np.clip(x, lo, hi)
    v, gr = g.interp(0, *x)
    vc, _ = g.interp(0, *xc)
    assert v == vc and gr[0] == 0.0 and gr[2] == 0.0 and gr[1] == pytest.approx(b / box.spacing)
    # full atom energy of type 0 with charge 0: map 0 value + penalty
    e, ge = g.atom_energy(0, 0.0, x)
    assert e == pytest.approx(vc + 10.0 * (0.7 ** 2 + 0.3 ** 2), rel=1e-12)
    h = 1e-6
    for ax in range(3):
        xp, xm = x.copy(), x.copy()
        xp[ax] += h
        xm[ax] -= h
        fd = (g.atom_energy(0, 0.0, xp)[0] - g.atom_energy(0, 0.0, xm)[0]) / (2 * h)
        assert ge[ax] == pytest.approx(fd, rel=1e-6, abs=1e-6)


def test_atom_energy_gradient_inside_cells(small_system):
    g = small_system["grid"]
    box = small_system["box"]
    rng = np.random.default_rng(3)
    lo, hi = box.box_lo(), box.box_hi()
    for _ in range(40):
        x = rng.uniform(lo + 0.1, hi - 0.1)
        u = (x - lo) / box.spacing
        if np.min(np.abs(u - np.round(u))) < 1e-3:
            continue
        t, q = int(rng.choice(box.map_types)), float(rng.uniform(-0.4, 0.4))
        e, ge = g.atom_energy(t, q, x)
        for ax in range(3):
            h = 1e-5     # inside one cell: the read is linear along each axis
            xp, xm = x.copy(), x.copy()
            xp[ax] += h
            xm[ax] -= h
            fd = (g.atom_energy(t, q, xp)[0] - g.atom_energy(t, q, xm)[0]) / (2 * h)
            # round-off of the differenced energies bounds the FD error
            assert ge[ax] == pytest.approx(fd, rel=1e-6, abs=1e-7 + 1e-14 * (abs(e) + 1.0) / h)
