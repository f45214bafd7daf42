"""Tolerances of the GPU-vs-oracle comparisons (shared by the GPU tests and smoke()).

Energy (FP64 path): |J - J*| <= 1e-12 * (sum_T |T| |W_T| + sum_n |b_n v_n|), the condition
number of the sum times the 1e-12 relative bar (a plain relative error is meaningless when
J_grad and b.v nearly cancel).  Gradient: ||g - g*||_inf <= 1e-10 ||g*||_inf.
Central differences amplify the rounding of W by 1/(2 eps), so the FD comparison adds
64 u max_n (sum_{T in patch(n)} |T| |W_T|) / eps to the gradient bar.
"""
import numpy as np

U = np.finfo(np.float64).eps / 2

ENERGY_RTOL = 1e-12
GRAD_RTOL = 1e-10


def energy_scale(om, v):
    _, _, dens = om.energy(v, densities=True)
    return float(np.abs(om.vol * dens).sum() + np.abs(om.b * v).sum())


def patch_energy_max(om, v):
    _, _, dens = om.energy(v, densities=True)
    ew = np.abs(om.vol * dens)
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
