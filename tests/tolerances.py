"""Parity tolerances between the FP32 CUDA path and the FP64 oracle.

The stated tolerance (checked on every genotype of the relaxed-pose tests):
  energies   |E - E_o| <= max(1e-4 |E_o|, 1e-3 kcal/mol);
  gradients  per gene block b (translation, quaternion, each torsion)
             ||g_b - g_o,b||_2 <= 1e-3 ||g_o,b||_2 + 1e-3,
the absolute 1e-3 (kcal/mol per A, per unit quaternion component or per
radian) being the gradient's counterpart of the energy's absolute 1e-3: a
relative bound alone is undefined where a block's gradient vanishes, as it
does for a torsion at a local minimum.

Clash poses (random genotypes, energies up to the 1e5 map cap) are checked
more loosely, because their error is set by the conditioning of the sum
rather than by its value:
  * an FP32 pose places an atom up to about one rounding of its coordinates
    away from the FP64 pose; the energy then moves by sum_i |dE/dx_i|_1 dx.
    POS_DX bounds dx (coordinates O(10 A) after up to ~10 nested rotations,
    each a few FP32 ulps: 2^-20 * 10 A ~ 1e-5 A), so the clash-pose energy
    tolerance is the stated one plus POS_DX * sum_i |f_i|_1;
  * a gradient block of a clash pose is a small difference of atom forces of
    up to ~1e4 kcal/mol/A, so its clash-pose tolerance is 1e-3 relative to
    the largest component of the whole gradient (floor 1).
"""
import numpy as np

E_REL, E_ABS = 1e-4, 1e-3
G_REL, G_ABS = 1e-3, 1e-3
G_FLOOR = 1.0
POS_DX = 2e-5


def energy_tol(e_ref, forces=None):
    """Stated energy tolerance; with forces, the clash-pose one."""
    tol = np.maximum(E_REL * np.abs(e_ref), E_ABS)
    if forces is not None:
        tol = tol + POS_DX * np.abs(forces).reshape(len(tol), -1).sum(axis=1)
    return tol


def grad_tol(g_ref):
    """Clash-pose gradient tolerance (per genotype, on the max-abs error)."""
    return G_REL * np.maximum(np.abs(g_ref).max(axis=-1), G_FLOOR)


def gene_blocks(n_torsions):
    """The gene blocks of a genotype: translation, quaternion, each torsion."""
    return [slice(0, 3), slice(3, 7)] + [slice(7 + k, 8 + k) for k in range(n_torsions)]


def grad_block_errors(g, g_ref, n_torsions):
    """Per genotype and block: (error norm, allowed error) under the stated
    per-block gradient tolerance.  Both arrays [B, 2 + n_torsions]."""
    g, g_ref = np.atleast_2d(g), np.atleast_2d(g_ref)
    err, tol = [], []
    for sl in gene_blocks(n_torsions):
        err.append(np.linalg.norm(g[:, sl] - g_ref[:, sl], axis=1))
        tol.append(G_REL * np.linalg.norm(g_ref[:, sl], axis=1) + G_ABS)
    return np.stack(err, axis=1), np.stack(tol, axis=1)
