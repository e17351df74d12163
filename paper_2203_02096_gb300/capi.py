"""Python binding of libdock.so (include/dock.h): argument marshalling only.

Every entry point keeps the C name.  Device buffers are torch CUDA tensors
(passed by data pointer, no copies); device memory the library allocates
comes from torch's caching allocator through the ``dock_allocator``
callbacks; streams are torch streams.  Loading raises if libdock.so is
missing or CUDA is unavailable -- there is no CPU path.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np
import torch

from . import build as _build

_lock = threading.Lock()
_lib = None

DOCK_OK = 0
ERRORS = {-1: "DOCK_ERR_INVALID", -2: "DOCK_ERR_CUDA", -3: "DOCK_ERR_OOM", -4: "DOCK_ERR_DISCONNECTED",
          -5: "DOCK_ERR_RING", -6: "DOCK_ERR_SIZE", -7: "DOCK_ERR_TYPE", -8: "DOCK_ERR_NOMAP", -9: "DOCK_ERR_DEVICE",
          -10: "DOCK_ERR_BUSY"}
DOCK_ERR_BUSY = -10
MAP_ELEC, MAP_DESOLV = -1, -2

# Every symbol include/dock.h declares, with (restype, argtypes).
_vp, _i, _d, _f = C.c_void_p, C.c_int, C.c_double, C.c_float
_u32, _u64, _i64, _sz = C.c_uint32, C.c_uint64, C.c_int64, C.c_size_t
_P = C.POINTER


class DockParams(C.Structure):
    _fields_ = [("pop_size", _i), ("nruns", _i), ("max_evals", _i64), ("ls_count", _i), ("ls_iters", _i),
                ("rho", _f), ("eps", _f), ("p_tour", _f), ("p_cross", _f), ("p_mut", _f), ("trans_mut", _f),
                ("ls_threads", _i), ("ls_method", _i), ("sw_rho0", _f), ("sw_rho_lo", _f), ("sw_expand", _f),
                ("sw_contract", _f), ("sw_succ", _i), ("sw_fail", _i), ("sw_step", _f * 3), ("batch_warps", _i),
                ("batch_pack", _i)]


ALLOC_FN = C.CFUNCTYPE(_vp, _sz, _vp, _vp)
FREE_FN = C.CFUNCTYPE(None, _vp, _vp, _vp)


class DockAllocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", _vp)]


SIGNATURES = {
    "dock_version": (_i, []),
    "dock_default_params": (None, [_P(DockParams)]),
    "dock_create": (_i, [_P(_vp), _i, _P(DockAllocator)]),
    "dock_destroy": (_i, [_vp]),
    "dock_last_error": (C.c_char_p, [_vp]),
    "load_grids": (_i, [_vp, _vp, _i, _vp, _vp, _d, _vp, _P(_vp)]),
    "build_grids": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _vp, _d, _i, _vp, _P(_vp)]),
    "grids_read_maps": (_i, [_vp, _vp, _vp]),
    "free_grids": (_i, [_vp, _vp]),
    "load_ligand": (_i, [_vp, _i, _vp, _vp, _vp, _i, _vp, _vp, _P(_vp)]),
    "ligand_info": (_i, [_vp, _P(_i), _P(_i), _P(_i), _P(_i), _P(_i)]),
    "free_ligand": (_i, [_vp, _vp]),
    "ligand_device_bytes": (_i, [_vp, _P(_sz)]),
    "score_batch": (_i, [_vp, _vp, _vp, _vp, _i, _vp, _vp]),
    "score_grad_batch": (_i, [_vp, _vp, _vp, _vp, _i, _vp, _vp, _vp]),
    "pose_batch": (_i, [_vp, _vp, _vp, _i, _vp, _vp]),
    "dock": (_i, [_vp, _vp, _vp, _P(DockParams), _u64, _vp, _vp, _vp]),
    "dock_async": (_i, [_vp, _vp, _vp, _P(DockParams), _u64, _vp, _vp, _vp, _vp, _vp]),
    "dock_async_noalloc": (_i, [_vp, _vp, _vp, _P(DockParams), _u64, _vp, _vp, _vp, _vp, _vp]),
    "dock_batch": (_i, [_vp, _vp, _vp, _i, _P(DockParams), _vp, _vp, _vp, _vp, _vp, _vp]),
    "server_create": (_i, [_vp, _i, _i, _i, _P(_vp)]),
    "server_submit": (_i, [_vp, _vp, _vp, _P(DockParams), _u64, _P(_i64)]),
    "server_poll": (_i, [_vp, _i64, _i, _P(_i)]),
    "server_result": (_i, [_vp, _i64, _i, _i, _vp, _vp, _vp]),
    "server_destroy": (_i, [_vp]),
    "server_cancel": (_i, [_vp, _i64, _i]),
    "dock_init_population": (_i, [_vp, _vp, _i, _i, _i, _u64, _vp, _vp]),
    "dock_ga_children": (_i, [_vp, _i, _i, _i, _vp, _vp, _u64, _u32, _P(DockParams), _vp, _vp, _vp]),
    "dock_ls_picks": (_i, [_vp, _i, _i, _i, _u64, _u32, _vp, _vp]),
    "dock_local_search": (_i, [_vp, _vp, _vp, _vp, _i, _i, _f, _f, _i, _vp, _vp, _vp]),
    "dock_local_search_trace": (_i, [_vp, _vp, _vp, _vp, _i, _i, _f, _f, _i, _vp, _vp, _vp, _vp, _vp, _vp]),
    "dock_adadelta_step": (_i, [_vp, _i, _i, _f, _f, _vp, _vp, _vp, _vp, _vp]),
    "dock_philox": (_i, [_vp, _vp, _i, _u32, _u32, _vp, _vp]),
    "dock_tune": (_i, [_vp, _vp, _vp, _i, _P(DockParams), _i, _vp, _i, _i, _vp]),
    "dock_set_option": (_i, [_vp, _i, _i]),
    "dock_microbench": (_i, [_vp, _i, _P(_d)]),
    "dock_get_option": (_i, [_vp, _i, _P(_i)]),
    "dock_solis_wets": (_i, [_vp, _vp, _vp, _vp, _vp, _i, _P(DockParams), _u64, _u32, _u32, _vp, _vp, _vp, _vp]),
    "dock_set_timing": (_i, [_vp, _i]),
    "dock_kernel_time": (_i, [_vp, C.c_char_p, _P(_d), _P(_i64)]),
    "dock_reset_timing": (_i, [_vp]),
    "dock_launch_count": (_i64, [_vp]),
}


def lib_path() -> str:
    return _build.OUT


def load(build_if_missing: bool = True):
    """Load libdock.so (compiling it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.OUT
            if not os.path.exists(path):
                raise RuntimeError(f"libdock.so not found at {path}: the CUDA library must be built")
            lib = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class DockError(RuntimeError):
    pass


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_cuda:
            raise ValueError("expected a CUDA tensor")
        if not t.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return C.c_void_p(t.data_ptr())
    return t.ctypes.data_as(C.c_void_p)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def default_params(**kw) -> DockParams:
    p = DockParams()
    load().dock_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "sw_step":
            v = (_f * 3)(*v)
        setattr(p, k, v)
    return p


class Context:
    """dock_ctx bound to a CUDA device, device memory from torch's allocator."""

    def __init__(self, device: int = 0, use_torch_allocator: bool = True):
        if not torch.cuda.is_available():
            raise RuntimeError("CUDA is not available: libdock has no CPU path")
        self.lib = load()
        self.device = device
        torch.cuda.set_device(device)
        self._cb = None
        self.alloc_calls = 0   # device allocations the library asked for
        alloc = None
        if use_torch_allocator:
            def _alloc(nbytes, stream, user):
                self.alloc_calls += 1
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), device, stream=int(stream or 0))
                except Exception:  # reported to the caller as DOCK_ERR_OOM
                    return None

            def _free(ptr, stream, user):
                torch.cuda.caching_allocator_delete(int(ptr))

            self._cb = (ALLOC_FN(_alloc), FREE_FN(_free))
            alloc = DockAllocator(self._cb[0], self._cb[1], None)
        h = C.c_void_p()
        rc = self.lib.dock_create(C.byref(h), device, C.byref(alloc) if alloc is not None else None)
        if rc != DOCK_OK:
            raise DockError(f"dock_create failed: {ERRORS.get(rc, rc)}")
        self.h = h

    def check(self, rc, what):
        if rc != DOCK_OK:
            msg = self.lib.dock_last_error(self.h).decode()
            raise DockError(f"{what}: {ERRORS.get(rc, rc)}: {msg}")

    def close(self):
        if getattr(self, "h", None) is not None:
            torch.cuda.synchronize(self.device)
            self.lib.dock_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- tracing
    def set_timing(self, on: bool):
        self.check(self.lib.dock_set_timing(self.h, int(on)), "dock_set_timing")

    def reset_timing(self):
        self.check(self.lib.dock_reset_timing(self.h), "dock_reset_timing")

    def kernel_time(self, name: str):
        ms, n = C.c_double(), C.c_int64()
        self.check(self.lib.dock_kernel_time(self.h, name.encode(), C.byref(ms), C.byref(n)), "dock_kernel_time")
        return ms.value, n.value

    def launch_count(self) -> int:
        return int(self.lib.dock_launch_count(self.h))


class Grids:
    def __init__(self, ctx: Context, h, n_maps: int):
        self.ctx, self.h, self.n_maps = ctx, h, n_maps

    def read_maps(self, dims):
        nx, ny, nz = dims
        out = np.zeros((self.n_maps, nz, ny, nx), dtype=np.float32)
        self.ctx.check(self.ctx.lib.grids_read_maps(self.ctx.h, self.h, _ptr(out)), "grids_read_maps")
        return out

    def free(self):
        if self.h is not None and self.ctx.h is not None:
            self.ctx.lib.free_grids(self.ctx.h, self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def load_grids(ctx: Context, maps: np.ndarray, dims, origin, spacing: float, map_type) -> Grids:
    maps = np.ascontiguousarray(maps, dtype=np.float32)
    d = np.ascontiguousarray(dims, dtype=np.int32)
    o = np.ascontiguousarray(origin, dtype=np.float64)
    mt = np.ascontiguousarray(map_type, dtype=np.int32)
    h = C.c_void_p()
    ctx.check(ctx.lib.load_grids(ctx.h, _ptr(maps), len(mt), _ptr(d), _ptr(o), float(spacing), _ptr(mt), C.byref(h)),
              "load_grids")
    return Grids(ctx, h, len(mt))


def build_grids(ctx: Context, rxyz, rtype, rq, dims, origin, spacing: float, map_types) -> Grids:
    rx = np.ascontiguousarray(rxyz, dtype=np.float64)
    rt = np.ascontiguousarray(rtype, dtype=np.int32)
    q = np.ascontiguousarray(rq, dtype=np.float64)
    d = np.ascontiguousarray(dims, dtype=np.int32)
    o = np.ascontiguousarray(origin, dtype=np.float64)
    mt = np.ascontiguousarray(map_types, dtype=np.int32)
    h = C.c_void_p()
    ctx.check(ctx.lib.build_grids(ctx.h, len(rt), _ptr(rx), _ptr(rt), _ptr(q), _ptr(d), _ptr(o), float(spacing),
                                  len(mt), _ptr(mt), C.byref(h)), "build_grids")
    return Grids(ctx, h, len(mt) + 2)


class Ligand:
    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h
        v = [C.c_int() for _ in range(5)]
        ctx.check(ctx.lib.ligand_info(h, *[C.byref(x) for x in v]), "ligand_info")
        self.n_atoms, self.n_torsions, self.n_genes, self.n_pairs, self.n_fragments = (x.value for x in v)

    def device_bytes(self) -> int:
        b = C.c_size_t()
        self.ctx.check(self.ctx.lib.ligand_device_bytes(self.h, C.byref(b)), "ligand_device_bytes")
        return int(b.value)

    def free(self):
        if self.h is not None and self.ctx.h is not None:
            self.ctx.lib.free_ligand(self.ctx.h, self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def load_ligand(ctx: Context, xyz, types, charges, bonds, rotatable) -> Ligand:
    x = np.ascontiguousarray(xyz, dtype=np.float64)
    t = np.ascontiguousarray(types, dtype=np.int32)
    q = np.ascontiguousarray(charges, dtype=np.float64)
    b = np.ascontiguousarray(bonds, dtype=np.int32).reshape(-1, 2)
    r = np.ascontiguousarray(rotatable, dtype=np.int32)
    h = C.c_void_p()
    ctx.check(ctx.lib.load_ligand(ctx.h, len(t), _ptr(x), _ptr(t), _ptr(q), len(r), _ptr(b), _ptr(r), C.byref(h)),
              "load_ligand")
    return Ligand(ctx, h)


def score_batch(ctx: Context, grids: Grids, lig: Ligand, geno: torch.Tensor, E: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
    B = geno.shape[0]
    if E is None:
        E = torch.empty(B, dtype=torch.float32, device=geno.device)
    ctx.check(ctx.lib.score_batch(ctx.h, grids.h, lig.h, _ptr(geno), B, _ptr(E), _stream(stream)), "score_batch")
    return E


def score_grad_batch(ctx: Context, grids: Grids, lig: Ligand, geno: torch.Tensor, E: torch.Tensor | None = None,
                     grad: torch.Tensor | None = None, stream=None):
    B = geno.shape[0]
    if E is None:
        E = torch.empty(B, dtype=torch.float32, device=geno.device)
    if grad is None:
        grad = torch.empty_like(geno)
    ctx.check(ctx.lib.score_grad_batch(ctx.h, grids.h, lig.h, _ptr(geno), B, _ptr(E), _ptr(grad), _stream(stream)),
              "score_grad_batch")
    return E, grad


def pose_batch(ctx: Context, lig: Ligand, geno: torch.Tensor, stream=None) -> torch.Tensor:
    B = geno.shape[0]
    xyz = torch.empty((B, lig.n_atoms, 3), dtype=torch.float32, device=geno.device)
    ctx.check(ctx.lib.pose_batch(ctx.h, lig.h, _ptr(geno), B, _ptr(xyz), _stream(stream)), "pose_batch")
    return xyz


def dock(ctx: Context, grids: Grids, lig: Ligand, params: DockParams, seed: int):
    """Blocking form with host outputs: (best_geno [R,G] f32, best_E [R] f64, evals [R] i64)."""
    R, G = params.nruns, lig.n_genes
    bg = np.zeros((R, G), dtype=np.float32)
    be = np.zeros(R, dtype=np.float64)
    ev = np.zeros(R, dtype=np.int64)
    ctx.check(ctx.lib.dock(ctx.h, grids.h, lig.h, C.byref(params), int(seed), _ptr(bg), _ptr(be), _ptr(ev)), "dock")
    return bg, be, ev


def dock_async(ctx: Context, grids: Grids, lig: Ligand, params: DockParams, seed: int, out=None, stream=None):
    """Queued form with device outputs: dict of tensors best_geno, best_E32, best_E, evals."""
    R, G = params.nruns, lig.n_genes
    dev = torch.device("cuda", ctx.device)
    if out is None:
        out = dict(best_geno=torch.empty((R, G), dtype=torch.float32, device=dev),
                   best_E32=torch.empty(R, dtype=torch.float32, device=dev),
                   best_E=torch.empty(R, dtype=torch.float64, device=dev),
                   evals=torch.empty(R, dtype=torch.int64, device=dev))
    ctx.check(ctx.lib.dock_async(ctx.h, grids.h, lig.h, C.byref(params), int(seed), _ptr(out["best_geno"]),
                                 _ptr(out["best_E32"]), _ptr(out["best_E"]), _ptr(out["evals"]), _stream(stream)),
              "dock_async")
    return out


def dock_async_noalloc(ctx: Context, grids: Grids, lig: Ligand, params: DockParams, seed: int, out, stream=None):
    """dock_async with its working buffers in the library's fixed device array
    (no device allocation in the call); ``out`` holds caller-owned tensors
    best_geno, best_E32, best_E, evals as returned by dock_async."""
    ctx.check(ctx.lib.dock_async_noalloc(ctx.h, grids.h, lig.h, C.byref(params), int(seed), _ptr(out["best_geno"]),
                                         _ptr(out["best_E32"]), _ptr(out["best_E"]), _ptr(out["evals"]),
                                         _stream(stream)), "dock_async_noalloc")
    return out


GENE_STRIDE = 39   # 7 + maximum torsions: row stride of dock_batch's best_geno


def dock_batch(ctx: Context, grids: Grids, ligs, params: DockParams, seeds=None, stream=None):
    """Dock many ligands in one persistent launch.  Returns device tensors
    best_geno [n, nruns, 39], best_E32 [n, nruns], best_E [n, nruns] (FP64),
    evals [n, nruns]; ligand k uses genes [:, :, :ligs[k].n_genes]."""
    n, R = len(ligs), params.nruns
    dev = torch.device("cuda", ctx.device)
    out = dict(best_geno=torch.zeros((n, R, GENE_STRIDE), dtype=torch.float32, device=dev),
               best_E32=torch.empty((n, R), dtype=torch.float32, device=dev),
               best_E=torch.empty((n, R), dtype=torch.float64, device=dev),
               evals=torch.empty((n, R), dtype=torch.int64, device=dev))
    arr = (C.c_void_p * max(n, 1))(*[l.h for l in ligs])
    sd = None if seeds is None else np.ascontiguousarray(seeds, dtype=np.uint64)
    ctx.check(ctx.lib.dock_batch(ctx.h, grids.h, arr, n, C.byref(params), _ptr(sd) if sd is not None else None,
                                 _ptr(out["best_geno"]), _ptr(out["best_E32"]), _ptr(out["best_E"]),
                                 _ptr(out["evals"]), _stream(stream)), "dock_batch")
    return out


class Server:
    """Continuous-batching docking server (server_* in dock.h)."""

    def __init__(self, ctx: Context, capacity: int = 65536, max_atoms: int = 128, pop_max: int = 150):
        self.ctx = ctx
        h = C.c_void_p()
        ctx.check(ctx.lib.server_create(ctx.h, capacity, max_atoms, pop_max, C.byref(h)), "server_create")
        self.h = h

    def submit(self, grids: Grids, lig: Ligand, params: DockParams, seed: int):
        """Returns the first task number, or None when the queue is full."""
        t = C.c_int64()
        rc = self.ctx.lib.server_submit(self.h, grids.h, lig.h, C.byref(params), int(seed), C.byref(t))
        if rc == DOCK_ERR_BUSY:
            return None
        self.ctx.check(rc, "server_submit")
        return t.value

    def done(self, first_task: int, nruns: int) -> bool:
        d = C.c_int()
        self.ctx.check(self.ctx.lib.server_poll(self.h, int(first_task), int(nruns), C.byref(d)), "server_poll")
        return bool(d.value)

    def result(self, first_task: int, nruns: int, n_genes: int):
        g = np.zeros((nruns, n_genes), dtype=np.float32)
        e = np.zeros(nruns, dtype=np.float64)
        v = np.zeros(nruns, dtype=np.int64)
        self.ctx.check(self.ctx.lib.server_result(self.h, int(first_task), int(nruns), int(n_genes), _ptr(g), _ptr(e),
                                                  _ptr(v)), "server_result")
        return g, e, v

    def cancel(self, first_task: int, nruns: int):
        """Withdraw the request's runs no warp has started (they finish at once, evals 0, energy +inf)."""
        self.ctx.check(self.ctx.lib.server_cancel(self.h, int(first_task), int(nruns)), "server_cancel")

    def close(self):
        if getattr(self, "h", None) is not None and self.ctx.h is not None:
            self.ctx.lib.server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dock_init_population(ctx, grids, n_torsions, pop, nruns, seed, stream=None):
    out = torch.empty((nruns, pop, 7 + n_torsions), dtype=torch.float32, device=f"cuda:{ctx.device}")
    ctx.check(ctx.lib.dock_init_population(ctx.h, grids.h, n_torsions, pop, nruns, int(seed), _ptr(out),
                                           _stream(stream)), "dock_init_population")
    return out


def dock_ga_children(ctx, n_torsions, pop_old: torch.Tensor, E_old: torch.Tensor, seed, generation,
                     params: DockParams | None = None, with_info=True, stream=None):
    nruns, pop, _ = pop_old.shape
    new = torch.empty_like(pop_old)
    info = torch.empty((nruns, pop, 5), dtype=torch.int64, device=pop_old.device) if with_info else None
    ctx.check(ctx.lib.dock_ga_children(ctx.h, n_torsions, pop, nruns, _ptr(pop_old), _ptr(E_old), int(seed),
                                       int(generation), C.byref(params) if params is not None else None, _ptr(new),
                                       _ptr(info), _stream(stream)), "dock_ga_children")
    return new, info


def dock_ls_picks(ctx, pop, n_ls, nruns, seed, generation, stream=None):
    out = torch.empty((nruns, max(n_ls, 1)), dtype=torch.int32, device=f"cuda:{ctx.device}")
    ctx.check(ctx.lib.dock_ls_picks(ctx.h, pop, n_ls, nruns, int(seed), int(generation), _ptr(out), _stream(stream)),
              "dock_ls_picks")
    return out[:, :n_ls]


def dock_local_search(ctx, grids, lig, x0: torch.Tensor, iters: int, rho=0.8, eps=1e-2, threads=0, stream=None):
    B = x0.shape[0]
    xb = torch.empty_like(x0)
    Eb = torch.empty(B, dtype=torch.float32, device=x0.device)
    ctx.check(ctx.lib.dock_local_search(ctx.h, grids.h, lig.h, _ptr(x0), B, int(iters), float(rho), float(eps),
                                        int(threads), _ptr(xb), _ptr(Eb), _stream(stream)), "dock_local_search")
    return xb, Eb


def dock_local_search_trace(ctx, grids, lig, x0: torch.Tensor, iters: int, rho=0.8, eps=1e-2, threads=0,
                            stream=None):
    """ADADELTA as dock_local_search, plus every iteration's point, gradient
    and energy: returns (x_best, E_best, x_trace [B, iters, G], g_trace
    [B, iters, G], E_trace [B, iters]), device tensors."""
    B, G = x0.shape
    xb = torch.empty_like(x0)
    Eb = torch.empty(B, dtype=torch.float32, device=x0.device)
    xt = torch.empty((B, iters, G), dtype=torch.float32, device=x0.device)
    gt = torch.empty((B, iters, G), dtype=torch.float32, device=x0.device)
    Et = torch.empty((B, iters), dtype=torch.float32, device=x0.device)
    ctx.check(ctx.lib.dock_local_search_trace(ctx.h, grids.h, lig.h, _ptr(x0), B, int(iters), float(rho), float(eps),
                                              int(threads), _ptr(xb), _ptr(Eb), _ptr(xt), _ptr(gt), _ptr(Et),
                                              _stream(stream)), "dock_local_search_trace")
    return xb, Eb, xt, gt, Et


def dock_adadelta_step(ctx, x: torch.Tensor, g: torch.Tensor, Eg2: torch.Tensor, Edx2: torch.Tensor, rho=0.8,
                       eps=1e-2, stream=None):
    """One ADADELTA update of the rows of x in place (Eg2, Edx2 updated in
    place too); all four [B, G] FP32 device tensors."""
    B, G = x.shape
    for t in (g, Eg2, Edx2):
        if t.shape != x.shape or t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError("g, Eg2, Edx2 must be contiguous FP32 tensors shaped like x")
    ctx.check(ctx.lib.dock_adadelta_step(ctx.h, B, G, float(rho), float(eps), _ptr(x), _ptr(g), _ptr(Eg2), _ptr(Edx2),
                                         _stream(stream)), "dock_adadelta_step")


def dock_solis_wets(ctx, grids, lig, x0: torch.Tensor, params: DockParams, E0: torch.Tensor | None = None,
                    seed: int = 0, run: int = 0, generation: int = 0, stream=None):
    """Solis-Wets searches from the rows of x0 (device); returns (x_best,
    E_best, evals) as device tensors."""
    B = x0.shape[0]
    xb = torch.empty_like(x0)
    Eb = torch.empty(B, dtype=torch.float32, device=x0.device)
    ev = torch.empty(B, dtype=torch.int64, device=x0.device)
    ctx.check(ctx.lib.dock_solis_wets(ctx.h, grids.h, lig.h, _ptr(x0), _ptr(E0) if E0 is not None else None, B,
                                      C.byref(params), int(seed), int(run), int(generation), _ptr(xb), _ptr(Eb),
                                      _ptr(ev), _stream(stream)), "dock_solis_wets")
    return xb, Eb, ev


TUNE_LS_THREADS = 1
TUNE_BATCH_WARPS = 2
TUNE_SCORE_BLOCKS = 3
TUNE_BATCH_BLOCKS = 4
OPT_SCORE_BLOCKS = 1
OPT_BATCH_BLOCKS = 2


PEAK_FFMA, PEAK_EX2, PEAK_L2_READ = 1, 2, 3


def microbench(ctx, what: int) -> float:
    """A measured device rate: TFLOP/s (FFMA), Gop/s (ex2) or GB/s (L2 read)."""
    v = C.c_double()
    ctx.check(ctx.lib.dock_microbench(ctx.h, int(what), C.byref(v)), "dock_microbench")
    return v.value


def set_option(ctx, option: int, value: int):
    ctx.check(ctx.lib.dock_set_option(ctx.h, int(option), int(value)), "dock_set_option")


def get_option(ctx, option: int) -> int:
    v = C.c_int()
    ctx.check(ctx.lib.dock_get_option(ctx.h, int(option), C.byref(v)), "dock_get_option")
    return v.value


def dock_tune(ctx, grids, ligs, params: DockParams, what: int, cand, reps: int = 3) -> np.ndarray:
    """Mean device milliseconds per launch of each candidate shape (-1: does not fit)."""
    cand = np.ascontiguousarray(cand, dtype=np.int32)
    ms = np.zeros(len(cand), dtype=np.float64)
    arr = (C.c_void_p * len(ligs))(*[l.h for l in ligs])
    ctx.check(ctx.lib.dock_tune(ctx.h, grids.h, arr, len(ligs), C.byref(params), int(what), _ptr(cand), len(cand),
                                int(reps), _ptr(ms)), "dock_tune")
    return ms


def dock_philox(ctx, ctr: torch.Tensor, key_lo: int, key_hi: int, stream=None) -> torch.Tensor:
    n = ctr.shape[0]
    out = torch.empty((n, 4), dtype=torch.int32, device=ctr.device)
    ctx.check(ctx.lib.dock_philox(ctx.h, _ptr(ctr), n, key_lo, key_hi, _ptr(out), _stream(stream)), "dock_philox")
    return out


# ---------------------------------------------------------------------------
# convenience: objects from the seeded synthetic inputs

def ligand_from(ctx: Context, lig) -> Ligand:
    return load_ligand(ctx, lig.xyz, lig.types, lig.charges, lig.bonds, lig.rotatable)


def grids_from_maps(ctx: Context, maps: np.ndarray, box) -> Grids:
    mt = list(box.map_types) + [MAP_ELEC, MAP_DESOLV]
    return load_grids(ctx, maps, box.dims, box.origin, box.spacing, mt)


def grids_from_receptor(ctx: Context, rec, box) -> Grids:
    return build_grids(ctx, rec.xyz, rec.types, rec.charges, box.dims, box.origin, box.spacing, box.map_types)
