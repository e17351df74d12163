"""The plain ADADELTA docking as a CUDA graph.  Its launch sequence is fixed
by the parameters (the number of generations follows from max_evals, the
population and the local-search counts), and dock_async_noalloc neither
allocates nor synchronises, so one call can be captured into a graph and
replayed.  Every replay must give the bits a direct call gives, rewriting
the caller's outputs, with no request to the allocator."""
import pytest
import torch

from paper_2203_02096_gb300 import capi, synth

pytestmark = pytest.mark.gpu


def _outputs(R, G):
    return dict(best_geno=torch.empty((R, G), dtype=torch.float32, device="cuda"),
                best_E32=torch.empty(R, dtype=torch.float32, device="cuda"),
                best_E=torch.empty(R, dtype=torch.float64, device="cuda"),
                evals=torch.empty(R, dtype=torch.int64, device="cuda"))


@pytest.mark.parametrize("threads", [0, 32])
def test_noalloc_docking_replays_as_a_cuda_graph(threads):
    types = ("C", "A", "N", "OA", "HD")
    lig = synth.make_ligand(16, 4, types, seed=0)
    box = synth.make_box(24, type_names=types)
    rec = synth.make_receptor(300, inner=4.0, outer=12.0, type_names=types, seed=1)
    ctx = capi.Context(0)
    G = capi.grids_from_receptor(ctx, rec, box)
    L = capi.ligand_from(ctx, lig)
    P = capi.default_params(pop_size=60, nruns=6, max_evals=6000, ls_iters=30, ls_threads=threads)
    # a direct call first: the reference, and every kernel of the path loaded
    ref = capi.dock_async(ctx, G, L, P, 5, out=_outputs(P.nruns, L.n_genes))
    torch.cuda.synchronize()
    out = _outputs(P.nruns, L.n_genes)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        capi.dock_async_noalloc(ctx, G, L, P, 5, out)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    before = ctx.alloc_calls
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        capi.dock_async_noalloc(ctx, G, L, P, 5, out)
    for _ in range(2):
        for t in out.values():
            t.zero_()
        graph.replay()
        torch.cuda.synchronize()
        for k in ("best_geno", "best_E32", "best_E", "evals"):
            assert torch.equal(out[k], ref[k]), k
    assert ctx.alloc_calls == before
    del graph
    ctx.close()
