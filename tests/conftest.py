"""Shared fixtures.  Tests marked ``gpu`` need a CUDA device and the built
CUDA library; everything else runs on the CPU only."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled CUDA library")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def small_system(oracle_mod):
    """16-atom / 4-torsion ligand in a 24^3 grid around a close receptor
    shell (inner radius 4 A) so that the field has structure."""
    from paper_2203_02096_gb300 import synth
    types = ("C", "A", "N", "OA", "HD")
    lig = synth.make_ligand(16, 4, types, seed=0)
    rec = synth.make_receptor(400, inner=4.0, outer=14.0, type_names=types, seed=1)
    box = synth.make_box(24, type_names=types)
    maps = oracle_mod.build_maps(rec, box)
    grid = oracle_mod.OracleGrid(maps.astype(np.float32), box)
    return dict(lig=lig, rec=rec, box=box, maps=maps, grid=grid, olig=oracle_mod.OracleLigand(lig))


@pytest.fixture(scope="session")
def gpu():
    """CUDA library context (fails loudly when CUDA or libdock is missing)."""
    from paper_2203_02096_gb300 import capi
    ctx = capi.Context(0)
    yield ctx
    ctx.close()


@pytest.fixture(scope="session")
def drug_system(oracle_mod):
    """40-atom / 10-torsion ligand in 64^3 x 9 maps from a 3000-atom receptor
    (the drug-size workload's inputs), maps built by the oracle."""
    from paper_2203_02096_gb300 import synth
    w = synth.drug_ligand_workload()
    maps = oracle_mod.build_maps(w.receptor, w.box)
    grid = oracle_mod.OracleGrid(maps.astype(np.float32), w.box)
    return dict(w=w, lig=w.ligand, box=w.box, rec=w.receptor, maps=grid.maps, grid=grid,
                olig=oracle_mod.OracleLigand(w.ligand))


@pytest.fixture(scope="session")
def diff_system(oracle_mod, drug_system):
    """64-atom / 16-torsion ligand in the same 64^3 grid set (differentiation workload)."""
    from paper_2203_02096_gb300 import synth
    lig = synth.make_ligand(64, 16, seed=0)
    return dict(lig=lig, box=drug_system["box"], maps=drug_system["maps"], grid=drug_system["grid"],
                olig=oracle_mod.OracleLigand(lig))
