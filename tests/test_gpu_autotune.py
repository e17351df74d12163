"""Autotuning on the GPU: dock_tune times every candidate width of the
local search and of the batch kernel; a tuned docking is the docking at the
chosen width; the batch kernel's warps per block never change a result."""
import numpy as np
import pytest
import torch

from paper_2203_02096_gb300 import autotune, capi, synth

pytestmark = pytest.mark.gpu


def test_ls_widths_timed_and_tuned_docking_reproducible(gpu, drug_system, tmp_path):
    L = capi.ligand_from(gpu, drug_system["lig"])
    G = capi.grids_from_maps(gpu, drug_system["maps"], drug_system["box"])
    P = capi.default_params(nruns=20, max_evals=20_000, ls_iters=60)
    curve = autotune.ls_curve(gpu, G, L, P)
    assert all(v["ms"] > 0 for v in curve.values()), curve
    t = autotune.Tuner(gpu, path=str(tmp_path / "tune.json"))
    Pt = t.tuned(G, L, P)
    assert Pt.ls_threads in autotune.LS_CANDIDATES
    assert t.tuned(G, L, P).ls_threads == Pt.ls_threads          # cached
    a = capi.dock(gpu, G, L, Pt, 3)
    P2 = capi.default_params(nruns=20, max_evals=20_000, ls_iters=60, ls_threads=Pt.ls_threads)
    b = capi.dock(gpu, G, L, P2, 3)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    # the Solis-Wets search is timed too
    Ps = capi.default_params(nruns=20, max_evals=20_000, ls_iters=60, ls_method=1)
    assert all(v["ms"] > 0 for v in autotune.ls_curve(gpu, G, L, Ps).values())


def test_batch_warps_do_not_change_results(gpu, drug_system, tmp_path):
    rng = np.random.default_rng(2)
    ligs = [synth.make_ligand(int(rng.integers(10, 109)), int(rng.integers(0, 33)), seed=500 + k) for k in range(9)]
    L = [capi.ligand_from(gpu, l) for l in ligs]
    G = capi.grids_from_maps(gpu, drug_system["maps"], drug_system["box"])
    outs = []
    for w in (1, 2, 4):
        P = capi.default_params(pop_size=30, nruns=2, max_evals=1500, ls_iters=10, batch_warps=w)
        outs.append(capi.dock_batch(gpu, G, L, P, np.arange(9, dtype=np.uint64)))
    torch.cuda.synchronize()
    for o in outs[1:]:
        for k in ("best_geno", "best_E", "evals"):
            assert torch.equal(o[k], outs[0][k]), k
    t = autotune.Tuner(gpu, path=str(tmp_path / "tune.json"))
    P = capi.default_params(pop_size=30, nruns=2, max_evals=1500, ls_iters=10)
    assert t.tuned(G, L, P).batch_warps in autotune.BATCH_CANDIDATES
    ms = capi.dock_tune(gpu, G, L, P, capi.TUNE_BATCH_WARPS, [1, 2, 4], 1)
    assert np.all(ms > 0)


def test_tune_rejects_bad_requests(gpu, drug_system):
    L = capi.ligand_from(gpu, drug_system["lig"])
    G = capi.grids_from_maps(gpu, drug_system["maps"], drug_system["box"])
    P = capi.default_params(nruns=2)
    with pytest.raises(capi.DockError):
        capi.dock_tune(gpu, G, [L], P, 99, [32])
    with pytest.raises(capi.DockError):
        capi.dock_tune(gpu, G, [L], P, capi.TUNE_LS_THREADS, [48])
    with pytest.raises(capi.DockError):
        capi.dock_batch(gpu, G, [L], capi.default_params(nruns=2, batch_warps=3))


def test_score_register_caps_do_not_change_results(gpu, drug_system, tmp_path):
    """score_grad_batch at every register cap gives the same bits; the tuner
    times them and sets its choice on the context."""
    L = capi.ligand_from(gpu, synth.make_ligand(64, 16, seed=0))
    G = capi.grids_from_maps(gpu, drug_system["maps"], drug_system["box"])
    x = torch.from_numpy(synth.make_genotypes(4099, L.n_torsions, drug_system["box"], seed=2)).cuda()
    res = []
    for b in (1, 6, 8):
        capi.set_option(gpu, capi.OPT_SCORE_BLOCKS, b)
        assert capi.get_option(gpu, capi.OPT_SCORE_BLOCKS) == b
        res.append(capi.score_grad_batch(gpu, G, L, x))
    capi.set_option(gpu, capi.OPT_SCORE_BLOCKS, 1)
    for E, g in res[1:]:
        assert torch.equal(E, res[0][0]) and torch.equal(g, res[0][1])
    t = autotune.Tuner(gpu, path=str(tmp_path / "tune.json"))
    b = t.score_blocks(G, L, batch=8192)
    assert b in autotune.SCORE_BLOCK_CANDIDATES and capi.get_option(gpu, capi.OPT_SCORE_BLOCKS) == b
    capi.set_option(gpu, capi.OPT_SCORE_BLOCKS, 1)
    with pytest.raises(capi.DockError):
        capi.set_option(gpu, capi.OPT_SCORE_BLOCKS, 3)


def test_batch_register_caps_do_not_change_results(gpu, drug_system):
    rng = np.random.default_rng(4)
    ligs = [synth.make_ligand(int(rng.integers(10, 109)), int(rng.integers(0, 33)), seed=700 + k) for k in range(6)]
    L = [capi.ligand_from(gpu, l) for l in ligs]
    G = capi.grids_from_maps(gpu, drug_system["maps"], drug_system["box"])
    P = capi.default_params(pop_size=30, nruns=2, max_evals=1500, ls_iters=10)
    outs = []
    for b in (4, 3):
        capi.set_option(gpu, capi.OPT_BATCH_BLOCKS, b)
        outs.append(capi.dock_batch(gpu, G, L, P, np.arange(6, dtype=np.uint64)))
    capi.set_option(gpu, capi.OPT_BATCH_BLOCKS, 4)
    torch.cuda.synchronize()
    for k in ("best_geno", "best_E", "evals"):
        assert torch.equal(outs[0][k], outs[1][k]), k
    ms = capi.dock_tune(gpu, G, L, P, capi.TUNE_BATCH_BLOCKS, [4, 3], 1)
    assert np.all(ms > 0)


def test_microbenchmarks_report_plausible_rates(gpu):
    """The roofline denominators measured on the device: FP32 FMA within
    (10, 120) TFLOP/s, ex2 within (100, 20000) Gop/s, L2 reads within
    (500, 50000) GB/s -- wide bands around GB300's unit counts."""
    assert 10 < capi.microbench(gpu, capi.PEAK_FFMA) < 120
    assert 100 < capi.microbench(gpu, capi.PEAK_EX2) < 20000
    assert 500 < capi.microbench(gpu, capi.PEAK_L2_READ) < 50000
    with pytest.raises(capi.DockError):
        capi.microbench(gpu, 99)
