"""FP64 CPU oracle for the binary-fluid D3Q19 lattice-Boltzmann step.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
(``paper_1609_01479_gb300``) never does, and the two share no code.

The arithmetic lives in ``ld_oracle.cpp`` (plain double, ``-ffp-contract=off``)
and follows the components of one Ludwig timestep named in Sec. 2.1.1 of the
paper (Collision, Propagation, Chemical stress, Order Parameter Gradients) in
their binary-fluid form: D3Q19 BGK with Guo forcing, the g collision, the
7-point Laplacian and central-difference force (or their 19-point isotropic
forms, ``stencil=19``), and periodic propagation.
This module only marshals numpy arrays through ctypes and builds the shared
object with g++.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ld_oracle.cpp")
_LC_SRC = os.path.join(_HERE, "lc_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

Q = 19
# Parameter vector order used by every call; then selectors of the stencils
# (0: 7-point Laplacian and central difference, 1: 19-point isotropic), the
# force form (0: -phi grad mu, 1: -div P) and the f collision (0: BGK, 1:
# two-relaxation-time), and the TRT magic parameter. Derivative directions
# cover the first seven.
PARAM_NAMES = ("A", "B", "kappa", "Gamma", "tau_f", "tau_g", "rho0", "stencil", "force", "collision", "magic")
DEFAULT_PARAMS = dict(A=-0.0625, B=0.0625, kappa=0.04, Gamma=0.5, tau_f=1.0, tau_g=1.0, rho0=1.0, stencil=0.0,
                      force=0.0, collision=0.0, magic=0.1875)
COLLISIONS = {"bgk": 0.0, "trt": 1.0}
STENCILS = {7: 0.0, 19: 1.0}
FORCES = {"potential": 0.0, "stress": 1.0}


def build(force: bool = False) -> str:
    """Compile ld_oracle.cpp and lc_oracle.cpp into _build/liboracle.so (g++, -O2, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_LC_SRC))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           _SRC, _LC_SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.POINTER(ctypes.c_double)
        IP = ctypes.POINTER(ctypes.c_int)
        i = ctypes.c_int
        lib.orc_version.restype = i
        lib.orc_set_threads.argtypes = [i]
        lib.orc_get_threads.restype = i
        lib.orc_lattice.argtypes = [IP, P]
        lib.orc_feq.argtypes = [ctypes.c_double, P, P]
        lib.orc_geq.argtypes = [ctypes.c_double, P, ctypes.c_double, ctypes.c_double, P]
        lib.orc_guo.argtypes = [P, P, ctypes.c_double, P]
        lib.orc_laplacian.argtypes = [i, i, i, i, P, P]
        lib.orc_gradient.argtypes = [i, i, i, i, P, P]
        lib.orc_propagate.argtypes = [i, i, i, i, P, P]
        lib.orc_init.argtypes = [i, i, i, P, P, P, P, P, P]
        lib.orc_step.argtypes = [i, i, i, P, P, P, i]
        lib.orc_macros.argtypes = [i, i, i, P, P, P, P, P, P, P, P, P, P]
        lib.orc_step_tl.argtypes = [i, i, i, P, P, P, P, P, P, i]
        lib.orc_loss_jvp.argtypes = [i, i, i, P, P, P, P, P, i, P, P]
        lib.orc_stress.argtypes = [i, i, i, P, P, P]
        lib.orc_lc_field.argtypes = [i, i, i, P, P, P, P]
        lib.orc_lc_corotation.argtypes = [P, P, P, P]
        lib.orc_lc_update.argtypes = [i, i, i, P, P, P, P, P]
        lib.orc_lc_macros.argtypes = [i, i, i, P, P, P, P, P, P]
        lib.orc_lc_init.argtypes = [i, i, i, P, P, P, P]
        lib.orc_lc_step.argtypes = [i, i, i, P, P, P, i]
        for name in ("orc_laplacian", "orc_gradient", "orc_propagate", "orc_init", "orc_step",
                     "orc_macros", "orc_step_tl", "orc_loss_jvp", "orc_stress", "orc_lc_field", "orc_lc_update",
                     "orc_lc_macros", "orc_lc_init", "orc_lc_step"):
            getattr(lib, name).restype = i
        _lib = lib
        return lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous float64"
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _prm(p):
    """The 11-entry parameter vector the C side reads (shorter ones get the
    defaults of the missing entries)."""
    p = _f64(p)
    if p.shape[0] < len(PARAM_NAMES):
        p = np.concatenate([p, [DEFAULT_PARAMS[k] for k in PARAM_NAMES[p.shape[0]:]]])
    assert p.shape == (len(PARAM_NAMES),), "parameter vector: " + ", ".join(PARAM_NAMES)
    return p


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} rejected its arguments (rc={rc})")


def param_vector(**overrides) -> np.ndarray:
    """Parameter vector; ``stencil`` is given as 7 or 19, ``force`` as
    "potential" or "stress", ``collision`` as "bgk" or "trt"."""
    p = dict(DEFAULT_PARAMS)
    names = {"stencil": lambda v: STENCILS[int(v)], "force": lambda v: FORCES[v], "collision": lambda v: COLLISIONS[v]}
    for k, v in overrides.items():
        if k not in p:
            raise KeyError(k)
        p[k] = names[k](v) if k in names else float(v)
    return np.array([p[k] for k in PARAM_NAMES], dtype=np.float64)


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def lattice():
    """Velocity set c (19x3 int) and weights w (19)."""
    lib = _load()
    c = np.zeros((Q, 3), dtype=np.int32)
    w = np.zeros(Q)
    lib.orc_lattice(c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _ptr(w))
    return c.astype(np.int64), w


def feq(rho, u):
    out = np.zeros(Q)
    _load().orc_feq(float(rho), _ptr(_f64(u)), _ptr(out))
    return out


def geq(phi, u, mu, Gamma):
    out = np.zeros(Q)
    _load().orc_geq(float(phi), _ptr(_f64(u)), float(mu), float(Gamma), _ptr(out))
    return out


def guo(u, F, tau):
    out = np.zeros(Q)
    _load().orc_guo(_ptr(_f64(u)), _ptr(_f64(F)), float(tau), _ptr(out))
    return out


def laplacian(phi, stencil=7):
    """Periodic Laplacian of a (nz, ny, nx) field: 7-point or 19-point isotropic."""
    phi = _f64(phi)
    nz, ny, nx = phi.shape
    out = np.zeros_like(phi)
    _check(_load().orc_laplacian(nx, ny, nz, int(STENCILS[stencil]), _ptr(phi), _ptr(out)), "laplacian")
    return out


def gradient(h, stencil=7):
    """Periodic gradient of a (nz, ny, nx) field -> (3, nz, ny, nx): central
    difference (7) or the 19-point isotropic form (19)."""
    h = _f64(h)
    nz, ny, nx = h.shape
    out = np.zeros((3,) + h.shape)
    _check(_load().orc_gradient(nx, ny, nz, int(STENCILS[stencil]), _ptr(h), _ptr(out)), "gradient")
    return out


def stress(phi, prm):
    """Chemical stress P of a (nz, ny, nx) phi field -> (6, nz, ny, nx), components
    xx, yy, zz, xy, xz, yz, with the stencils selected in prm."""
    phi = _f64(phi)
    nz, ny, nx = phi.shape
    out = np.zeros((6,) + phi.shape)
    _check(_load().orc_stress(nx, ny, nz, _ptr(_prm(prm)), _ptr(phi), _ptr(out)), "stress")
    return out


def propagate(dist, reverse=False):
    """Propagate a (19, nz, ny, nx) distribution (push), or its transpose."""
    dist = _f64(dist)
    _, nz, ny, nx = dist.shape
    out = np.zeros_like(dist)
    _check(_load().orc_propagate(nx, ny, nz, int(bool(reverse)), _ptr(dist), _ptr(out)), "propagate")
    return out


def init(phi, prm, rho=None, u=None):
    """Equilibrium initial state from phi (nz,ny,nx) [, rho, u (3,nz,ny,nx)] -> f, g."""
    phi = _f64(phi)
    nz, ny, nx = phi.shape
    f = np.zeros((Q,) + phi.shape)
    g = np.zeros((Q,) + phi.shape)
    _check(_load().orc_init(nx, ny, nz, _ptr(_prm(prm)), _ptr(phi), _ptr(_f64(rho)), _ptr(_f64(u)),
                            _ptr(f), _ptr(g)), "init")
    return f, g


def step(f, g, prm, nsteps=1):
    """Advance copies of (f, g) by nsteps full timesteps; returns the new pair."""
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    g = np.array(g, dtype=np.float64, order="C", copy=True)
    _, nz, ny, nx = f.shape
    _check(_load().orc_step(nx, ny, nz, _ptr(_prm(prm)), _ptr(f), _ptr(g), int(nsteps)), "step")
    return f, g


def macros(f, g, prm):
    """Macroscopic fields of a pre-collision state.

    Returns a dict with rho, u (3,...), phi, grad_phi (3,...), mu, force (3,...)
    and totals = [sum rho, sum phi, sum jx, sum jy, sum jz].
    """
    f = _f64(f)
    g = _f64(g)
    shp = f.shape[1:]
    nz, ny, nx = shp
    out = dict(rho=np.zeros(shp), u=np.zeros((3,) + shp), phi=np.zeros(shp),
               grad_phi=np.zeros((3,) + shp), mu=np.zeros(shp), force=np.zeros((3,) + shp),
               totals=np.zeros(5))
    _check(_load().orc_macros(nx, ny, nz, _ptr(_prm(prm)), _ptr(f), _ptr(g), _ptr(out["rho"]),
                              _ptr(out["u"]), _ptr(out["phi"]), _ptr(out["grad_phi"]),
                              _ptr(out["mu"]), _ptr(out["force"]), _ptr(out["totals"])), "macros")
    return out


def step_tl(f, g, df, dg, prm, dprm, nsteps=1):
    """Tangent-linear step: returns (f, g, df, dg) after nsteps."""
    arrs = [np.array(a, dtype=np.float64, order="C", copy=True) for a in (f, g, df, dg)]
    _, nz, ny, nx = arrs[0].shape
    _check(_load().orc_step_tl(nx, ny, nz, _ptr(_prm(prm)), _ptr(_f64(dprm)[:7].copy()), *[_ptr(a) for a in arrs],
                               int(nsteps)), "step_tl")
    return tuple(arrs)


def loss_jvp(phi0, phi_target, prm, nsteps, dphi0=None, dprm=None):
    """L = sum (phi_T - phi_target)^2 from an equilibrium start at phi0, and
    its directional derivative along (dphi0, dprm)."""
    phi0 = _f64(phi0)
    nz, ny, nx = phi0.shape
    dprm = np.zeros(7) if dprm is None else _f64(dprm)[:7].copy()
    loss = np.zeros(1)
    dloss = np.zeros(1)
    _check(_load().orc_loss_jvp(nx, ny, nz, _ptr(_prm(prm)), _ptr(dprm), _ptr(phi0), _ptr(_f64(dphi0)),
                                _ptr(_f64(phi_target)), int(nsteps), _ptr(loss), _ptr(dloss)), "loss_jvp")
    return float(loss[0]), float(dloss[0])


def loss(phi0, phi_target, prm, nsteps):
    """Forward-only loss (plain double path)."""
    f, g = init(phi0, prm)
    f, g = step(f, g, prm, nsteps)
    phi_T = g.sum(axis=0)
    return float(((phi_T - phi_target) ** 2).sum())


# ---------------------------------------------------------------------------
# Liquid crystal (lc_oracle.cpp): Landau-de Gennes Q-tensor, Beris-Edwards
# update, chemical stress coupled to the D3Q19 fluid. Q is held as its five
# independent components (xx, xy, xz, yy, yz), shaped (5, nz, ny, nx).
LC_PARAM_NAMES = ("A0", "gamma", "kappa", "Gamma", "xi", "tau_f", "rho0")
LC_DEFAULT_PARAMS = dict(A0=0.01, gamma=3.0, kappa=0.01, Gamma=0.3, xi=0.7, tau_f=1.0, rho0=1.0)


def lc_param_vector(**overrides) -> np.ndarray:
    p = dict(LC_DEFAULT_PARAMS)
    for k, v in overrides.items():
        if k not in p:
            raise KeyError(k)
        p[k] = float(v)
    return np.array([p[k] for k in LC_PARAM_NAMES], dtype=np.float64)


def lc_field(q, prm):
    """Molecular field H (5, ...) and chemical stress sigma (9, ..., row-major ab) of Q."""
    q = _f64(q)
    _, nz, ny, nx = q.shape
    h = np.zeros((5,) + q.shape[1:])
    sigma = np.zeros((9,) + q.shape[1:])
    _check(_load().orc_lc_field(nx, ny, nz, _ptr(_f64(prm)), _ptr(q), _ptr(h), _ptr(sigma)), "lc_field")
    return h, sigma


def lc_corotation(W, Q, prm):
    """S(W, Q) for full 3x3 W (W_ab = d_b u_a) and Q."""
    out = np.zeros(9)
    _load().orc_lc_corotation(_ptr(_f64(prm)), _ptr(_f64(np.asarray(W).reshape(9))),
                              _ptr(_f64(np.asarray(Q).reshape(9))), _ptr(out))
    return out.reshape(3, 3)


def lc_update(q, u, h, prm):
    """Q(t+1) from Q, a velocity field u (3, ...) and H (5, ...)."""
    q = _f64(q)
    _, nz, ny, nx = q.shape
    out = np.zeros_like(q)
    _check(_load().orc_lc_update(nx, ny, nz, _ptr(_f64(prm)), _ptr(q), _ptr(_f64(u)), _ptr(_f64(h)), _ptr(out)),
           "lc_update")
    return out


def lc_macros(f, q, prm):
    """rho, u = (j + F/2)/rho and F = div sigma of the state (f, Q)."""
    f = _f64(f)
    shp = f.shape[1:]
    nz, ny, nx = shp
    rho, u, F = np.zeros(shp), np.zeros((3,) + shp), np.zeros((3,) + shp)
    _check(_load().orc_lc_macros(nx, ny, nz, _ptr(_f64(prm)), _ptr(f), _ptr(_f64(q)), _ptr(rho), _ptr(u), _ptr(F)),
           "lc_macros")
    return dict(rho=rho, u=u, force=F)


def lc_init(shape, prm, rho=None, u=None):
    """f = feq(rho, u) (rho0 and rest where not given) on a (nz, ny, nx) lattice."""
    nz, ny, nx = shape
    f = np.zeros((Q, nz, ny, nx))
    _check(_load().orc_lc_init(nx, ny, nz, _ptr(_f64(prm)), _ptr(_f64(rho)), _ptr(_f64(u)), _ptr(f)), "lc_init")
    return f


def lc_step(f, q, prm, nsteps=1):
    """Advance copies of (f, Q) by nsteps coupled steps."""
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    q = np.array(q, dtype=np.float64, order="C", copy=True)
    _, nz, ny, nx = f.shape
    _check(_load().orc_lc_step(nx, ny, nz, _ptr(_f64(prm)), _ptr(f), _ptr(q), int(nsteps)), "lc_step")
    return f, q
