"""The serving kernel winds down as a whole.  While one long run is still in
progress and every other warp is idle, the idle warps must not leave one by
one: a launch with most warps gone but one busy warp left is still
"running", so the host would not relaunch it, and new requests would be
served by the warps that remain.  Requests submitted in that spell must be
served at the same rate as requests submitted to a busy kernel."""
import time

import numpy as np
import pytest

from paper_2203_02096_gb300 import capi, synth

pytestmark = pytest.mark.gpu


def _wait(server, firsts, nruns, limit):
    t0 = time.perf_counter()
    while not all(server.done(f, nruns) for f in firsts):
        if time.perf_counter() - t0 > limit:
            return None
        time.sleep(0.002)
    return time.perf_counter() - t0


def test_requests_during_an_idle_spell_are_served_at_full_rate(gpu, drug_system):
    G = capi.grids_from_maps(gpu, drug_system["maps"], drug_system["box"])
    Ls = [capi.ligand_from(gpu, synth.make_ligand(24 + (k % 5) * 8, 4, seed=300 + k)) for k in range(96)]
    P = capi.default_params(pop_size=60, nruns=20, max_evals=20000, ls_iters=30)
    server = capi.Server(gpu, capacity=1 << 14, max_atoms=128, pop_max=150)
    # reference: the batch submitted while the kernel is busy
    ref = _wait(server, [server.submit(G, L, P, k) for k, L in enumerate(Ls)], P.nruns, 120.0)
    assert ref is not None
    # one long run (one warp busy for seconds), every other warp idle past
    # the second of idleness after which a launch winds down
    P1 = capi.default_params(pop_size=60, nruns=1, max_evals=150000, ls_iters=30)
    long_first = server.submit(G, Ls[0], P1, 7)
    time.sleep(1.5)
    t = _wait(server, [server.submit(G, L, P, 500 + k) for k, L in enumerate(Ls)], P.nruns, 20.0 * ref + 10.0)
    assert _wait(server, [long_first], 1, 120.0) is not None
    server.close()
    assert t is not None and t < 2.0 * ref + 0.5, (ref, t)
