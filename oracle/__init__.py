"""FP64 CPU oracle of the docking hot path -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library and its Python
binding never import it.  ``oracle.c`` is plain C compiled with gcc into
``liboracle.so`` beside it; this module is argument marshalling over ctypes.

Parity status of each entry point: see the header of ``oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAX_ATOMS = 255
MAX_TORSIONS = 32


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, no FMA contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-pthread",
                   "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


class Grid(C.Structure):
    _fields_ = [("maps", C.c_void_p), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("nmaps", C.c_int),
                ("ox", C.c_double), ("oy", C.c_double), ("oz", C.c_double), ("h", C.c_double),
                ("map_of_type", C.c_int * 8), ("emap", C.c_int), ("dmap", C.c_int)]


class SwParams(C.Structure):
    _fields_ = [("rho0", C.c_float), ("rho_lo", C.c_float), ("expand", C.c_float), ("contract", C.c_float),
                ("n_succ", C.c_int), ("n_fail", C.c_int),
                ("step_t", C.c_float), ("step_q", C.c_float), ("step_tau", C.c_float)]


# Solis-Wets constants (readings): rho from 1 down to 0.01, x2 after 4
# successes, x0.5 after 4 failures; half-widths 1 A, 0.2, 0.75 rad at rho = 1.
SW_DEFAULTS = dict(rho0=1.0, rho_lo=0.01, expand=2.0, contract=0.5, n_succ=4, n_fail=4,
                   step_t=1.0, step_q=0.2, step_tau=0.75)


def make_sw(**kw) -> SwParams:
    v = dict(SW_DEFAULTS, **kw)
    s = SwParams()
    for k, x in v.items():
        setattr(s, k, x)
    return s


class Params(C.Structure):
    _fields_ = [("pop_size", C.c_int), ("nruns", C.c_int), ("max_evals", C.c_longlong),
                ("ls_count", C.c_int), ("ls_iters", C.c_int), ("rho", C.c_double), ("eps", C.c_double),
                ("p_tour", C.c_float), ("p_cross", C.c_float), ("p_mut", C.c_float), ("trans_mut", C.c_float),
                ("ls_method", C.c_int), ("sw", SwParams)]


def _L():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        vp, i, d, u32, u64 = C.c_void_p, C.c_int, C.c_double, C.c_uint32, C.c_uint64
        P = C.POINTER
        sig = {
            "orc_vdw_hb": (d, [i, i, d, P(d)]),
            "orc_dielectric": (d, [d, P(d)]),
            "orc_elec": (d, [d, d, d, P(d)]),
            "orc_desolv": (d, [i, d, i, d, d, P(d)]),
            "orc_pair_energy": (d, [i, d, i, d, d, P(d)]),
            "orc_map_values_at": (None, [i, vp, vp, vp, i, vp, d, d, d, vp]),
            "orc_build_maps": (i, [i, vp, vp, vp, i, i, i, d, d, d, d, i, vp, i, vp]),
            "orc_interp": (d, [P(Grid), i, d, d, d, vp]),
            "orc_atom_grid_energy": (d, [P(Grid), i, d, vp, vp]),
            "orc_ligand_create": (i, [i, vp, vp, vp, i, vp, vp, P(vp)]),
            "orc_ligand_free": (None, [vp]),
            "orc_ligand_info": (i, [vp, P(i), P(i), P(i)]),
            "orc_ligand_pairs": (i, [vp, vp]),
            "orc_ligand_torsion": (i, [vp, i, P(i), P(i), P(i), vp]),
            "orc_pose_local": (i, [vp, vp, i, vp]),
            "orc_pose": (d, [vp, vp, vp]),
            "orc_intra_xyz": (d, [vp, vp, vp]),
            "orc_inter_xyz": (d, [vp, P(Grid), vp, vp]),
            "orc_score": (d, [vp, P(Grid), vp, vp, vp, vp]),
            "orc_score_batch": (i, [vp, P(Grid), vp, i, vp, vp, i]),
            "orc_pose_margins": (None, [vp, P(Grid), vp, vp]),
            "orc_atom_forces": (d, [vp, P(Grid), vp, vp]),
            "orc_philox": (None, [vp, vp, vp]),
            "orc_init_individual": (None, [i, P(Grid), u64, u32, u32, vp]),
            "orc_init_population": (None, [i, P(Grid), u64, u32, i, vp]),
            "orc_ga_children": (i, [i, i, vp, vp, u64, u32, u32, P(Params), vp, vp]),
            "orc_ls_picks": (None, [i, i, u64, u32, u32, vp]),
            "orc_adadelta_step": (None, [i, i, d, d, vp, vp, vp, vp]),
            "orc_local_search": (d, [vp, P(Grid), vp, i, d, d, vp, vp]),
            "orc_solis_wets": (d, [vp, P(Grid), vp, d, i, P(SwParams), u64, u32, u32, u32, vp, P(C.c_longlong),
                                   vp, P(i)]),
            "orc_dock": (i, [vp, P(Grid), P(Params), u64, i, vp, vp, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# --------------------------------------------------------------------------- pair terms

def vdw_hb(ta, tb, r):
    d = C.c_double()
    e = _L().orc_vdw_hb(int(ta), int(tb), float(r), C.byref(d))
    return e, d.value


def dielectric(r):
    d = C.c_double()
    e = _L().orc_dielectric(float(r), C.byref(d))
    return e, d.value


def elec(qa, qb, r):
    d = C.c_double()
    e = _L().orc_elec(float(qa), float(qb), float(r), C.byref(d))
    return e, d.value


def desolv(ta, qa, tb, qb, r):
    d = C.c_double()
    e = _L().orc_desolv(int(ta), float(qa), int(tb), float(qb), float(r), C.byref(d))
    return e, d.value


def pair_energy(ta, qa, tb, qb, r):
    d = C.c_double()
    e = _L().orc_pair_energy(int(ta), float(qa), int(tb), float(qb), float(r), C.byref(d))
    return e, d.value


# --------------------------------------------------------------------------- maps

def build_maps(receptor, box, nthreads: int | None = None) -> np.ndarray:
    """All maps of ``box`` from ``receptor``: [n_type_maps+2, nz, ny, nx] float64."""
    nx, ny, nz = box.dims
    nt = len(box.map_types)
    out = np.zeros((nt + 2, nz, ny, nx), dtype=np.float64)
    rx, rt, rq = _f64(receptor.xyz), _i32(receptor.types), _f64(receptor.charges)
    mt = _i32(box.map_types)
    rc = _L().orc_build_maps(len(rt), _p(rx), _p(rt), _p(rq), nx, ny, nz, *box.origin, box.spacing, nt, _p(mt),
                             int(nthreads or os.cpu_count() or 1), _p(out))
    if rc != 0:
        raise ValueError(f"orc_build_maps failed ({rc})")
    return out


def map_values_at(receptor, map_types, points) -> np.ndarray:
    pts = _f64(points).reshape(-1, 3)
    mt = _i32(map_types)
    rx, rt, rq = _f64(receptor.xyz), _i32(receptor.types), _f64(receptor.charges)
    out = np.zeros((len(pts), len(mt) + 2))
    row = np.zeros(len(mt) + 2)
    for k, p in enumerate(pts):
        _L().orc_map_values_at(len(rt), _p(rx), _p(rt), _p(rq), len(mt), _p(mt), float(p[0]), float(p[1]),
                               float(p[2]), _p(row))
        out[k] = row
    return out


class OracleGrid:
    """FP32 map values (as both sides receive them) plus the box geometry."""

    def __init__(self, maps_f32: np.ndarray, box):
        self.maps = _f32(maps_f32)
        nm, nz, ny, nx = self.maps.shape
        assert (nx, ny, nz) == tuple(box.dims)
        self.box = box
        g = Grid()
        g.maps = self.maps.ctypes.data
        g.nx, g.ny, g.nz, g.nmaps = nx, ny, nz, nm
        g.ox, g.oy, g.oz = box.origin
        g.h = box.spacing
        for t in range(8):
            g.map_of_type[t] = -1
        for m, t in enumerate(box.map_types):
            g.map_of_type[t] = m
        g.emap = len(box.map_types)
        g.dmap = len(box.map_types) + 1
        self.s = g

    @property
    def ref(self):
        return C.byref(self.s)

    def interp(self, m, x, y, z):
        gr = np.zeros(3)
        v = _L().orc_interp(self.ref, int(m), float(x), float(y), float(z), _p(gr))
        return v, gr

    def atom_energy(self, t, q, x):
        gr = np.zeros(3)
        xx = _f64(x)
        e = _L().orc_atom_grid_energy(self.ref, int(t), float(q), _p(xx), _p(gr))
        return e, gr


# --------------------------------------------------------------------------- ligand

class OracleLigand:
    def __init__(self, lig):
        self._keep = (_f64(lig.xyz), _i32(lig.types), _f64(lig.charges), _i32(lig.bonds), _i32(lig.rotatable))
        xyz, ty, q, bonds, rot = self._keep
        h = C.c_void_p()
        rc = _L().orc_ligand_create(len(ty), _p(xyz), _p(ty), _p(q), len(rot), _p(bonds), _p(rot), C.byref(h))
        if rc != 0:
            raise ValueError(f"orc_ligand_create failed ({rc})")
        self.h = h
        self.n_atoms = len(ty)
        nt, npairs, nf = C.c_int(), C.c_int(), C.c_int()
        _L().orc_ligand_info(h, C.byref(nt), C.byref(npairs), C.byref(nf))
        self.n_torsions, self.n_pairs, self.n_frag = nt.value, npairs.value, nf.value
        self.n_genes = 7 + self.n_torsions

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.orc_ligand_free(self.h)
            self.h = None

    def pairs(self) -> np.ndarray:
        ij = np.zeros((max(self.n_pairs, 1), 2), dtype=np.int32)
        _L().orc_ligand_pairs(self.h, _p(ij))
        return ij[: self.n_pairs]

    def torsion(self, k):
        a, b, d = C.c_int(), C.c_int(), C.c_int()
        moves = np.zeros(self.n_atoms, dtype=np.uint8)
        if _L().orc_ligand_torsion(self.h, int(k), C.byref(a), C.byref(b), C.byref(d), _p(moves)) != 0:
            raise IndexError(k)
        return a.value, b.value, d.value, moves.astype(bool)

    def pose_local(self, tau, order=0):
        t = _f64(tau)
        out = np.zeros((self.n_atoms, 3))
        _L().orc_pose_local(self.h, _p(t), int(order), _p(out))
        return out

    def pose(self, geno):
        g = _f64(geno)
        out = np.zeros((self.n_atoms, 3))
        _L().orc_pose(self.h, _p(g), _p(out))
        return out

    def intra_xyz(self, xyz, with_grad=False):
        x = _f64(xyz)
        f = np.zeros_like(x)
        e = _L().orc_intra_xyz(self.h, _p(x), _p(f) if with_grad else None)
        return (e, f) if with_grad else e

    def inter_xyz(self, grid, xyz, with_grad=False):
        x = _f64(xyz)
        f = np.zeros_like(x)
        e = _L().orc_inter_xyz(self.h, grid.ref, _p(x), _p(f) if with_grad else None)
        return (e, f) if with_grad else e

    def score(self, grid, geno, with_grad=True, terms=False):
        g = _f64(geno)
        gr = np.zeros(self.n_genes)
        tm = np.zeros(2)
        e = _L().orc_score(self.h, grid.ref, _p(g), _p(gr) if with_grad else None, None, _p(tm))
        out = (e, gr) if with_grad else (e,)
        if terms:
            out = out + (tm,)
        return out if len(out) > 1 else out[0]

    def score_batch(self, grid, genos, with_grad=True, nthreads=None):
        g = _f32(genos).reshape(-1, self.n_genes)
        B = g.shape[0]
        E = np.zeros(B)
        gr = np.zeros((B, self.n_genes)) if with_grad else None
        _L().orc_score_batch(self.h, grid.ref, _p(g), B, _p(E), _p(gr) if with_grad else None,
                             int(nthreads or os.cpu_count() or 1))
        return (E, gr) if with_grad else E

    def atom_forces(self, grid, geno):
        g = _f64(geno)
        f = np.zeros((self.n_atoms, 3))
        e = _L().orc_atom_forces(self.h, grid.ref, _p(g), _p(f))
        return e, f

    def margins(self, grid, geno):
        g = _f64(geno)
        out = np.zeros(3)
        _L().orc_pose_margins(self.h, grid.ref, _p(g), _p(out))
        return out


# --------------------------------------------------------------------------- random numbers and GA

def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _L().orc_philox(_p(c), _p(k), _p(out))
    return out


def make_params(pop_size=150, nruns=1, max_evals=10_000, ls_rate_pct=6, ls_iters=100, rho=0.8, eps=1e-2,
                p_tour=0.6, p_cross=0.8, p_mut=0.02, trans_mut=2.0, ls_count=None, ls_method=0,
                sw: SwParams | None = None) -> Params:
    p = Params()
    p.ls_method = ls_method
    p.sw = sw if sw is not None else make_sw()
    p.pop_size, p.nruns, p.max_evals = pop_size, nruns, max_evals
    p.ls_count = (ls_rate_pct * pop_size + 99) // 100 if ls_count is None else ls_count
    p.ls_iters, p.rho, p.eps = ls_iters, rho, eps
    p.p_tour, p.p_cross, p.p_mut, p.trans_mut = p_tour, p_cross, p_mut, trans_mut
    return p


def init_population(n_torsions, grid, seed, run, pop):
    out = np.zeros((pop, 7 + n_torsions), dtype=np.float32)
    _L().orc_init_population(int(n_torsions), grid.ref, int(seed), int(run), int(pop), _p(out))
    return out


def ga_children(n_torsions, pop_old, E_old, seed, run, gen, params):
    pop_old = _f32(pop_old)
    E = _f64(E_old)
    pop = pop_old.shape[0]
    out = np.zeros_like(pop_old)
    info = np.zeros((pop, 5), dtype=np.int64)
    elite = _L().orc_ga_children(int(n_torsions), pop, _p(pop_old), _p(E), int(seed), int(run), int(gen),
                                 C.byref(params), _p(out), _p(info))
    return out, info, elite


def ls_picks(pop, n_ls, seed, run, gen):
    out = np.zeros(max(n_ls, 1), dtype=np.int32)
    _L().orc_ls_picks(int(pop), int(n_ls), int(seed), int(run), int(gen), _p(out))
    return out[:n_ls]


def adadelta_step(x, g, Eg2, Edx2, n_torsions, rho=0.8, eps=1e-2):
    x, g, Eg2, Edx2 = (_f64(a).copy() for a in (x, g, Eg2, Edx2))
    _L().orc_adadelta_step(len(x), int(n_torsions), float(rho), float(eps), _p(x), _p(g), _p(Eg2), _p(Edx2))
    return x, Eg2, Edx2


def local_search(lig: OracleLigand, grid, x0, iters, rho=0.8, eps=1e-2):
    x0 = _f32(x0)
    out = np.zeros_like(x0)
    trace = np.zeros(max(iters, 1))
    e = _L().orc_local_search(lig.h, grid.ref, _p(x0), int(iters), float(rho), float(eps), _p(out), _p(trace))
    return e, out, trace[:iters]


def solis_wets(lig: OracleLigand, grid, x0, iters, E0=None, sw: SwParams | None = None, seed=0, run=0, gen=0,
               entity=0):
    """One Solis-Wets search from x0 (its energy E0, or None to evaluate it).
    Returns (E, x, evals, iterations done, trace [iters_done, 4])."""
    x0 = _f32(x0)
    out = np.zeros_like(x0)
    trace = np.full((max(iters, 1), 4), np.nan)
    n = C.c_longlong(0)
    it = C.c_int(0)
    e = _L().orc_solis_wets(lig.h, grid.ref, _p(x0), float("nan") if E0 is None else float(E0), int(iters),
                            C.byref(sw if sw is not None else make_sw()), int(seed), int(run), int(gen),
                            int(entity), _p(out), C.byref(n), _p(trace), C.byref(it))
    return e, out, int(n.value), int(it.value), trace[:it.value]


def dock(lig: OracleLigand, grid, params: Params, seed: int, nthreads=None):
    G = lig.n_genes
    best_geno = np.zeros((params.nruns, G), dtype=np.float32)
    best_E = np.zeros(params.nruns)
    evals = np.zeros(params.nruns, dtype=np.int64)
    rc = _L().orc_dock(lig.h, grid.ref, C.byref(params), int(seed), int(nthreads or os.cpu_count() or 1),
                       _p(best_geno), _p(best_E), _p(evals))
    if rc != 0:
        raise ValueError(f"orc_dock failed ({rc})")
    return best_geno, best_E, evals
