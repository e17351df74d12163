"""dock_async_noalloc: docking for callers that must not allocate device
memory during the call (an application whose device memory is all owned by
its own pool, a plugin handed only pointers, a loop that cannot afford
cudaMalloc's device synchronisation).  Checked through the C-ABI against
dock_async on the same inputs, on two calls in a row (the fixed scratch
array is reused and keeps the previous call's contents), with no request to
the context's allocator during those calls.  This file is collected last."""
import numpy as np
import pytest
import torch

from paper_2203_02096_gb300 import capi, synth

pytestmark = pytest.mark.gpu


def _outputs(R, G):
    return dict(best_geno=torch.empty((R, G), dtype=torch.float32, device="cuda"),
                best_E32=torch.empty(R, dtype=torch.float32, device="cuda"),
                best_E=torch.empty(R, dtype=torch.float64, device="cuda"),
                evals=torch.empty(R, dtype=torch.int64, device="cuda"))


def test_noalloc_matches_dock_async_twice():
    types = ("C", "A", "N", "OA", "HD")
    lig = synth.make_ligand(16, 4, types, seed=0)
    box = synth.make_box(24, type_names=types)
    rec = synth.make_receptor(300, inner=4.0, outer=12.0, type_names=types, seed=1)
    ctx = capi.Context(0)
    G = capi.grids_from_receptor(ctx, rec, box)
    L = capi.ligand_from(ctx, lig)
    P = capi.default_params(pop_size=60, nruns=6, max_evals=6000, ls_iters=30)
    for call, seed in enumerate((3, 4)):
        ref = capi.dock_async(ctx, G, L, P, seed, out=_outputs(P.nruns, L.n_genes))
        torch.cuda.synchronize()
        got = _outputs(P.nruns, L.n_genes)
        before = ctx.alloc_calls
        capi.dock_async_noalloc(ctx, G, L, P, seed, got)
        torch.cuda.synchronize()
        assert ctx.alloc_calls == before, "the no-allocation entry point asked the allocator for memory"
        # same kernels on the same inputs: identical results (tolerance 0)
        for k in ("best_geno", "best_E32", "best_E", "evals"):
            assert torch.equal(got[k], ref[k]), (call, k)
        assert np.all(got["evals"].cpu().numpy() >= 6000)


def test_noalloc_rejects_oversized_requests():
    types = ("C", "A", "N", "OA", "HD")
    lig = synth.make_ligand(16, 4, types, seed=0)
    box = synth.make_box(24, type_names=types)
    ctx = capi.Context(0)
    G = capi.grids_from_maps(ctx, np.zeros((7, 24, 24, 24), np.float32), box)
    L = capi.ligand_from(ctx, lig)
    P = capi.default_params(pop_size=2000, nruns=100, max_evals=10, ls_iters=1)
    with pytest.raises(capi.DockError, match="SIZE.*bytes of scratch"):
        capi.dock_async_noalloc(ctx, G, L, P, 0, _outputs(P.nruns, L.n_genes))
