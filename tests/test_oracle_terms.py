"""Pins of the oracle's pair terms against the properties that define them
(the intramolecular self-interactions of Section II-A: van der Waals,
hydrogen bonding, electrostatics, desolvation), not against the oracle's own
formulas.  The constants named here are this project's force-field readings."""
import math

import numpy as np
import pytest

C, A, N, NA, OA, SA, HD = range(7)
RADIUS = {C: 4.0, A: 4.0, N: 3.5, NA: 3.5, OA: 3.2, SA: 4.0, HD: 2.0}
WELL = {C: 0.15, A: 0.15, N: 0.16, NA: 0.16, OA: 0.20, SA: 0.20, HD: 0.02}
HBOND = {OA: (1.9, 5.0), NA: (1.9, 5.0), SA: (2.5, 1.0)}   # acceptor: (R_hb, eps_hb)
W_VDW, W_HB = 0.16, 0.12
SIGMA, CUTOFF, R_FLOOR = 3.6, 8.0, 0.5


def _argmin_r(f, lo, hi):
    rs = np.linspace(lo, hi, 200001)
    es = np.array([f(r) for r in rs[::50]])
    k = int(np.argmin(es)) * 50
    fine = rs[max(0, k - 60): k + 60]
    es = np.array([f(r) for r in fine])
    return fine[int(np.argmin(es))], es.min()


@pytest.mark.parametrize("ta,tb", [(C, C), (C, OA), (N, A), (HD, HD), (SA, C), (OA, OA)])
def test_vdw_minimum_location_and_depth(oracle_mod, ta, tb):
    """12-6 potential: minimum at R_ij = (R_i+R_j)/2, depth -w_vdw*sqrt(eps_i eps_j),
    zero crossing at R_ij / 2^(1/6)."""
    Rij = 0.5 * (RADIUS[ta] + RADIUS[tb])
    eps = math.sqrt(WELL[ta] * WELL[tb])
    e, d = oracle_mod.vdw_hb(ta, tb, Rij)
    assert e == pytest.approx(-W_VDW * eps, rel=1e-12)
    assert abs(d) < 1e-9 * W_VDW * eps / Rij
    r0 = Rij / 2 ** (1 / 6)
    assert abs(oracle_mod.vdw_hb(ta, tb, r0)[0]) < 1e-12
    rmin, emin = _argmin_r(lambda r: oracle_mod.vdw_hb(ta, tb, r)[0], 0.9 * r0, 3 * Rij)
    assert rmin == pytest.approx(Rij, abs=1e-3)


@pytest.mark.parametrize("acc", [OA, NA, SA])
@pytest.mark.parametrize("donor_first", [True, False])
def test_hbond_minimum(oracle_mod, acc, donor_first):
    """12-10 H-bond between donor HD and an acceptor: minimum -w_hb*eps_hb at R_hb,
    the same whichever atom comes first."""
    Rhb, ehb = HBOND[acc]
    ta, tb = (HD, acc) if donor_first else (acc, HD)
    e, d = oracle_mod.vdw_hb(ta, tb, Rhb)
    assert e == pytest.approx(-W_HB * ehb, rel=1e-12)
    assert abs(d) < 1e-9
    rmin, _ = _argmin_r(lambda r: oracle_mod.vdw_hb(ta, tb, r)[0], 0.8 * Rhb, 3 * Rhb)
    assert rmin == pytest.approx(Rhb, abs=1e-3)


def test_hbond_only_between_donor_and_acceptor(oracle_mod):
    # acceptor-acceptor and donor-donor pairs take the 12-6 form
    for ta, tb in [(OA, OA), (OA, NA), (HD, HD), (HD, C)]:
        Rij = 0.5 * (RADIUS[ta] + RADIUS[tb])
        assert oracle_mod.vdw_hb(ta, tb, Rij)[0] == pytest.approx(-W_VDW * math.sqrt(WELL[ta] * WELL[tb]))


def test_dielectric_limits_and_monotone(oracle_mod):
    """Sigmoidal dielectric eps(r) = A + B/(1 + k exp(-lambda B r)), B = eps0 - A:
    eps(0) = A + B/(1+k), eps(inf) = eps0 = 78.4, increasing in r."""
    Ad, eps0, k = -8.5525, 78.4, 7.7839
    B = eps0 - Ad
    assert oracle_mod.dielectric(0.0)[0] == pytest.approx(Ad + B / (1 + k), rel=1e-12)
    assert oracle_mod.dielectric(1e4)[0] == pytest.approx(eps0, rel=1e-12)
    rs = np.linspace(0, 40, 401)
    es = [oracle_mod.dielectric(r)[0] for r in rs]
    assert np.all(np.diff(es) > 0)


def test_electrostatics_is_screened_coulomb(oracle_mod):
    """E_el * eps(r) * r is the same constant at every r (and bilinear in the
    charges); far away it tends to w_el*332.06*qa*qb/78.4/r."""
    qa, qb = 0.3, -0.2
    vals = [oracle_mod.elec(qa, qb, r)[0] * oracle_mod.dielectric(r)[0] * r for r in (0.7, 1.5, 3.0, 6.0, 7.9)]
    assert np.allclose(vals, vals[0], rtol=1e-12)
    assert oracle_mod.elec(2 * qa, qb, 3.0)[0] == pytest.approx(2 * oracle_mod.elec(qa, qb, 3.0)[0], rel=1e-13)
    assert vals[0] < 0  # opposite charges attract
    r = 5000.0
    assert oracle_mod.elec(qa, qb, r)[0] == pytest.approx(0.14 * 332.06 * qa * qb / 78.4 / r, rel=1e-9)


def test_desolvation_is_gaussian(oracle_mod):
    """Desolvation term: Gaussian of width 3.6 A in r, linear in |q| of each atom."""
    e1 = oracle_mod.desolv(C, 0.2, OA, -0.1, 1.0)[0]
    e2 = oracle_mod.desolv(C, 0.2, OA, -0.1, 3.0)[0]
    assert e2 / e1 == pytest.approx(math.exp(-(9.0 - 1.0) / (2 * SIGMA ** 2)), rel=1e-12)
    # charge enters through |q|: the sign of a charge does not matter
    assert oracle_mod.desolv(C, -0.2, OA, 0.1, 2.0)[0] == pytest.approx(oracle_mod.desolv(C, 0.2, OA, -0.1, 2.0)[0])
    # HD has no volume, so an HD-HD pair has no desolvation
    assert oracle_mod.desolv(HD, 0.3, HD, 0.3, 1.0)[0] == 0.0
    # linear in |q_a|
    d0 = oracle_mod.desolv(C, 0.0, OA, 0.0, 2.0)[0]
    d1 = oracle_mod.desolv(C, 0.1, OA, 0.0, 2.0)[0]
    d2 = oracle_mod.desolv(C, 0.2, OA, 0.0, 2.0)[0]
    assert d2 - d1 == pytest.approx(d1 - d0, rel=1e-10)


@pytest.mark.parametrize("fn", ["vdw", "hb", "elec", "desolv", "pair"])
def test_term_derivatives_match_central_differences(oracle_mod, fn):
    f = {
        "vdw": lambda r: oracle_mod.vdw_hb(C, OA, r),
        "hb": lambda r: oracle_mod.vdw_hb(HD, OA, r),
        "elec": lambda r: oracle_mod.elec(0.25, -0.35, r),
        "desolv": lambda r: oracle_mod.desolv(N, 0.1, SA, -0.3, r),
        "pair": lambda r: oracle_mod.pair_energy(NA, 0.1, HD, 0.2, r),
    }[fn]
    for r in np.linspace(0.6, 7.8, 37):
        h = 1e-6 * r
        fd = (f(r + h)[0] - f(r - h)[0]) / (2 * h)
        assert f(r)[1] == pytest.approx(fd, rel=2e-6, abs=1e-9)


def test_pair_energy_sum_cutoff_and_floor(oracle_mod):
    for r in (0.7, 2.0, 5.5, 7.999):
        tot = oracle_mod.pair_energy(OA, -0.3, HD, 0.25, r)[0]
        parts = (oracle_mod.vdw_hb(OA, HD, r)[0] + oracle_mod.elec(-0.3, 0.25, r)[0]
                 + oracle_mod.desolv(OA, -0.3, HD, 0.25, r)[0])
        assert tot == pytest.approx(parts, rel=1e-14)
    assert oracle_mod.pair_energy(OA, -0.3, HD, 0.25, CUTOFF) == (0.0, 0.0)
    assert oracle_mod.pair_energy(OA, -0.3, HD, 0.25, 9.0) == (0.0, 0.0)
    # below the floor the energy is frozen at its floor value and the force is zero
    e_f = oracle_mod.pair_energy(C, 0.1, C, 0.1, R_FLOOR)[0]
    e_in, d_in = oracle_mod.pair_energy(C, 0.1, C, 0.1, 0.2)
    assert e_in == e_f and d_in == 0.0
