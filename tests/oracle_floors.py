"""Rounding floors of the FP64 oracle's own output, used as the parity bar
for fields whose 1e-12 relative bar lies below what FP64 arithmetic can fix.

u = (j + F/2) / rho is formed from j = sum_i f_i c_i, a cancellation of
O(w_i) values. When |u| is small its relative error is set by the rounding of
those values, not by the method: a perturbation of the oracle's own initial
distributions by at most one unit in the last place moves u by that floor.
"""

import numpy as np

import oracle


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def oracle_u_floor(phi, steps, prm=None, rho=None, u=None, reference_u=None):
    """Relative L2 change of the oracle's u after `steps` steps when each of
    its initial distributions moves by -1, 0 or +1 ulp (seeded): the rounding
    floor of u for that start. `reference_u` (the unperturbed oracle's u at
    `steps`, if already computed) saves one oracle run."""
    prm = oracle.param_vector() if prm is None else prm
    f, g = oracle.init(phi, prm, rho=rho, u=u)
    rng = np.random.default_rng(1234)
    fp = f + np.spacing(f) * rng.choice([-1.0, 0.0, 1.0], size=f.shape)
    gp = g + np.spacing(g) * rng.choice([-1.0, 0.0, 1.0], size=g.shape)
    if reference_u is None:
        reference_u = oracle.macros(*oracle.step(f, g, prm, steps), prm)["u"]
    moved = oracle.macros(*oracle.step(fp, gp, prm, steps), prm)["u"]
    return rel_l2(moved, reference_u)
