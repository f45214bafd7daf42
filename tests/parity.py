"""Tolerances of the GPU-vs-oracle comparisons (shared by the GPU tests and smoke()).

Energy (FP64 path): |J - J*| <= 1e-12 * (sum_T |T| |W_T| + sum_n |b_n v_n|), the condition
number of the sum times the 1e-12 relative bar (a plain relative error is meaningless when
J_grad and b.v nearly cancel).  Gradient: ||g - g*||_inf <= 1e-10 ||g*||_inf.
Central differences amplify the rounding of the patch energies by 1/(2 eps).  The oracle
evaluates eq. neoHook as written, C1 (I1 - dim - 2 log det F) + D1 (det F - 1)^2, whose
rounding is relative to the size of its terms S_T = C1 (I1 + dim + 2 |log det F|) +
D1 (det F - 1)^2 rather than to W_T (near F = I the terms cancel to a W_T orders of magnitude
smaller); for the p-Laplacian S_T = |W_T|.  The FD comparison therefore adds
64 u max_n (sum_{T in patch(n)} |T| S_T) / eps to the gradient bar.
"""
import numpy as np

from paper_2109_01158_gb300 import meshgen as mg

U = np.finfo(np.float64).eps / 2

ENERGY_RTOL = 1e-12
GRAD_RTOL = 1e-10


def energy_scale(om, v):
    _, _, dens = om.energy(v, densities=True)
    return float(np.abs(om.vol * dens).sum() + np.abs(om.b * v).sum())


def density_term_scale(om, v):
    """S_T per element: the magnitude of the terms the oracle's density is evaluated from."""
    _, _, dens = om.energy(v, densities=True)
    if om.model != mg.MODEL_NEOHOOKE:
        return np.abs(dens)
    k = om.dim + 1
    dphi = om.dphi.reshape(om.ne, k, om.dim)
    vv = np.asarray(v, dtype=np.float64).reshape(om.nn, om.d)
    F = np.einsum("elj,elm->ejm", vv[om.elems], dphi)
    I1 = (F * F).sum(axis=(1, 2))
    det = np.linalg.det(F)
    with np.errstate(divide="ignore"):
        logdet = np.abs(np.log(np.abs(det)))
    return om.C1 * (I1 + om.dim + 2.0 * logdet) + om.D1 * (det - 1.0) ** 2


def patch_energy_max(om, v):
    ew = np.abs(om.vol * density_term_scale(om, v))
    k = om.dim + 1
    per_entry = ew[om.ent[: om.ne * k] // k]
    sums = np.add.reduceat(per_entry, om.row_ptr[:-1]) if om.ne else np.zeros(om.nn)
    sums[np.diff(om.row_ptr) == 0] = 0.0
    return float(sums.max()) if sums.size else 0.0


def check_energy(J, Jref, scale, rtol=ENERGY_RTOL):
    err = abs(J - Jref)
    assert err <= rtol * scale, f"|J-J*| = {err:.3e} > {rtol:g} * {scale:.3e} (J={J!r}, J*={Jref!r})"
    return err / max(scale, 1e-300)


def check_grad(g, gref, rtol=GRAD_RTOL, extra_abs=0.0):
    err = float(np.abs(np.asarray(g) - np.asarray(gref)).max()) if len(gref) else 0.0
    ref = float(np.abs(gref).max()) if len(gref) else 0.0
    assert err <= rtol * ref + extra_abs, f"||g-g*|| = {err:.3e} > {rtol:g} * {ref:.3e} + {extra_abs:.3e}"
    return err / max(ref, 1e-300)


def fd_extra(om, v, eps):
    return 64 * U * patch_energy_max(om, v) / eps
