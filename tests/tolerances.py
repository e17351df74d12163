"""Parity tolerances between the FP32 CUDA path and the FP64 oracle.

Energies: 1e-4 relative or 1e-3 kcal/mol absolute, whichever is larger.
Gradients: 1e-3 relative to the largest component of the oracle gradient
(a floor of 1 kcal/mol per unit gene keeps near-zero gradients meaningful).

On top of that, an FP32 pose cannot place an atom closer than about one
rounding of its coordinates to the FP64 pose, and the energy moves by
sum_i |dE/dx_i|_1 * dx for a position error dx.  POS_DX bounds dx: the
coordinates are O(10 A) after up to ~10 nested rotations (each a few FP32
ulps, 2^-20 * 10 A ~ 1e-5 A) -- so the energy tolerance of a genotype is
the stated one plus POS_DX * sum_i |f_i|_1.  Tests report how many
genotypes meet the stated tolerance alone.
"""
import numpy as np

E_REL, E_ABS = 1e-4, 1e-3
G_REL, G_FLOOR = 1e-3, 1.0
POS_DX = 2e-5


def energy_tol(e_ref, forces=None):
    tol = np.maximum(E_REL * np.abs(e_ref), E_ABS)
    if forces is not None:
        tol = tol + POS_DX * np.abs(forces).reshape(len(tol), -1).sum(axis=1)
    return tol


def grad_tol(g_ref):
    return G_REL * np.maximum(np.abs(g_ref).max(axis=-1), G_FLOOR)
