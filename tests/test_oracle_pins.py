"""Pins of the FP64 oracle to facts that do not come from the oracle itself:
textbook identities of the D3Q19 lattice and the equilibria, permutation
structure of propagation, exact discrete Fourier modes of the stencils,
conservation laws, fixed points, and closed-form hydrodynamic and
thermodynamic limits (viscosity, mobility, advection, interface profile).

Each test names the plausible mistakes it would catch.
"""

import math
import os

import numpy as np
import pytest

from paper_1609_01479_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_lattice():
    c, w = [], []
    with open(os.path.join(GOLDEN, "d3q19_lattice.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if not line:
                continue
            parts = line.split()
            c.append([int(v) for v in parts[1:4]])
            num, den = parts[4].split("/")
            w.append(float(num) / float(den))
    return np.array(c), np.array(w)


def golden_constants():
    out = {}
    with open(os.path.join(GOLDEN, "derived_constants.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()
                out[k] = float(v)
    return out


# --------------------------------------------------------------------------
# Velocity set (catches a wrong vector, weight or ordering).


def test_velocity_set_matches_textbook(orc):
    c, w = orc.lattice()
    cg, wg = _golden_lattice()
    assert np.array_equal(c, cg)
    assert np.array_equal(w, wg)
    # opposite pairs: odd i and i+1
    for i in range(1, 19, 2):
        assert np.array_equal(c[i], -c[i + 1])


def test_velocity_set_isotropy(orc):
    c, w = orc.lattice()
    d = np.eye(3)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.abs(np.einsum("i,ia->a", w, c)).max() < 1e-15
    assert np.abs(np.einsum("i,ia,ib->ab", w, c, c) - d / 3.0).max() < 1e-15
    assert np.abs(np.einsum("i,ia,ib,ic->abc", w, c, c, c)).max() < 1e-15
    iso4 = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
            + np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.abs(np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c) - iso4).max() < 1e-15


# --------------------------------------------------------------------------
# Equilibria and forcing: moments fixed by the model's definition
# (catches a wrong coefficient 3, 9/2, 3/2, a dropped u.u or (|c|^2-1) term,
# a sign error in the Guo term or its (1 - 1/(2 tau)) prefactor).


def _moments(c, dist):
    return dist.sum(), c.T @ dist, np.einsum("ia,ib,i->ab", c, c, dist)


@pytest.mark.parametrize("seed", range(5))
def test_feq_moments(orc, seed):
    rng = np.random.default_rng(seed)
    c, _ = orc.lattice()
    rho = 0.8 + 0.4 * rng.random()
    u = 0.1 * (rng.random(3) - 0.5)
    m0, m1, m2 = _moments(c, orc.feq(rho, u))
    assert abs(m0 - rho) < 1e-14
    assert np.abs(m1 - rho * u).max() < 1e-15
    assert np.abs(m2 - (rho / 3.0 * np.eye(3) + rho * np.outer(u, u))).max() < 1e-15


@pytest.mark.parametrize("seed", range(5))
def test_geq_moments(orc, seed):
    rng = np.random.default_rng(100 + seed)
    c, _ = orc.lattice()
    phi = 2.0 * rng.random() - 1.0
    mu = 0.2 * (rng.random() - 0.5)
    Gamma = 0.3 + rng.random()
    u = 0.1 * (rng.random(3) - 0.5)
    m0, m1, m2 = _moments(c, orc.geq(phi, u, mu, Gamma))
    assert abs(m0 - phi) < 1e-14
    assert np.abs(m1 - phi * u).max() < 1e-15
    assert np.abs(m2 - (Gamma * mu * np.eye(3) + phi * np.outer(u, u))).max() < 1e-14


@pytest.mark.parametrize("seed", range(5))
def test_guo_moments(orc, seed):
    rng = np.random.default_rng(200 + seed)
    c, _ = orc.lattice()
    u = 0.1 * (rng.random(3) - 0.5)
    F = 1e-3 * (rng.random(3) - 0.5)
    tau = 0.55 + 1.5 * rng.random()
    pre = 1.0 - 1.0 / (2.0 * tau)
    m0, m1, m2 = _moments(c, orc.guo(u, F, tau))
    assert abs(m0) < 1e-17
    assert np.abs(m1 - pre * F).max() < 1e-17
    assert np.abs(m2 - pre * (np.outer(u, F) + np.outer(F, u))).max() < 1e-17


# --------------------------------------------------------------------------
# Propagation is a permutation: component i moves by c_i (catches a sign or
# axis swap, a wrong periodic wrap, a transposed reverse).


@pytest.mark.parametrize("shape", [(4, 4, 4), (7, 6, 5), (3, 8, 2)])
def test_propagate_is_roll(orc, shape):
    rng = np.random.default_rng(7)
    c, _ = orc.lattice()
    d = rng.standard_normal((19,) + shape)
    out = orc.propagate(d)
    for i in range(19):
        ref = np.roll(d[i], shift=(c[i, 2], c[i, 1], c[i, 0]), axis=(0, 1, 2))
        assert np.array_equal(out[i], ref)
    back = orc.propagate(out, reverse=True)
    assert np.array_equal(back, d)
    y = rng.standard_normal(d.shape)
    lhs = float((out * y).sum())
    rhs = float((d * orc.propagate(y, reverse=True)).sum())
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


# --------------------------------------------------------------------------
# Stencils on exact discrete Fourier modes (catches a wrong sign, a missing
# neighbour, a wrong factor of 2 in the central difference, an axis mix-up).


def test_laplacian_on_fourier_mode(orc):
    nz, ny, nx = 6, 10, 8
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    k = (2 * math.pi * 1 / nx, 2 * math.pi * 3 / ny, 2 * math.pi * 2 / nz)
    phi = np.cos(k[0] * x + k[1] * y + k[2] * z + 0.3)
    lam = sum(2.0 * (1.0 - math.cos(ka)) for ka in k)
    lap = orc.laplacian(phi)
    assert np.abs(lap + lam * phi).max() < 1e-13


def test_gradient_on_fourier_mode(orc):
    nz, ny, nx = 6, 10, 8
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    k = (2 * math.pi * 1 / nx, 2 * math.pi * 3 / ny, 2 * math.pi * 2 / nz)
    arg = k[0] * x + k[1] * y + k[2] * z
    h = np.sin(arg)
    gr = orc.gradient(h)
    for a in range(3):
        assert np.abs(gr[a] - math.sin(k[a]) * np.cos(arg)).max() < 1e-14


def test_mu_and_force_of_uniform_phi(orc):
    prm = orc.param_vector()
    A, B = prm[0], prm[1]
    phi = np.full((4, 5, 6), 0.37)
    f, g = orc.init(phi, prm)
    m = orc.macros(f, g, prm)
    assert np.abs(m["mu"] - (A * 0.37 + B * 0.37 ** 3)).max() < 1e-16
    assert np.abs(m["force"]).max() == 0.0


def test_mu_of_fourier_mode(orc):
    """mu = A phi + B phi^3 - kappa lap(phi) with lap known exactly."""
    prm = orc.param_vector(kappa=0.07)
    A, B, kappa = prm[0], prm[1], prm[2]
    nx = 16
    phi = inputs.sine_phi(nx, 4, 4, 0.3, mode=2)
    lam = 2.0 * (1.0 - math.cos(2 * math.pi * 2 / nx))
    f, g = orc.init(phi, prm)
    m = orc.macros(f, g, prm)
    ref = A * phi + B * phi ** 3 + kappa * lam * phi
    assert np.abs(m["mu"] - ref).max() < 1e-15
    assert np.abs(m["phi"] - phi).max() < 1e-15


# --------------------------------------------------------------------------
# Initial state (catches init from the wrong equilibrium or wrong mu).


def test_init_moments(orc):
    prm = orc.param_vector()
    nz, ny, nx = 5, 6, 7
    phi = inputs.spinodal_phi(nx, ny, nz, seed=3)
    rng = np.random.default_rng(3)
    rho = 1.0 + 0.01 * rng.standard_normal((nz, ny, nx))
    u = 0.01 * rng.standard_normal((3, nz, ny, nx))
    f, g = orc.init(phi, prm, rho=rho, u=u)
    c, _ = orc.lattice()
    assert np.abs(f.sum(0) - rho).max() < 1e-15
    assert np.abs(g.sum(0) - phi).max() < 1e-15
    j = np.einsum("ia,i...->a...", c, f)
    assert np.abs(j - rho * u).max() < 1e-16
    # second moment of g = Gamma mu I + phi u u with mu from the 7-point stencil
    A, B, kappa, Gamma = prm[:4]
    mu = A * phi + B * phi ** 3 - kappa * orc.laplacian(phi)
    pxx = np.einsum("i,i...->...", c[:, 0] * c[:, 0], g)
    assert np.abs(pxx - (Gamma * mu + phi * u[0] * u[0])).max() < 1e-15


# --------------------------------------------------------------------------
# Conservation (catches any collision that leaks mass or phi, a Guo term
# with the wrong first moment, a propagation that drops values).


@pytest.mark.parametrize("shape", [(8, 8, 8), (7, 6, 5)])
def test_conservation(orc, shape):
    prm = orc.param_vector(tau_f=0.8, tau_g=1.3)
    nz, ny, nx = shape
    phi = inputs.spinodal_phi(nx, ny, nz, seed=11)
    f, g = orc.init(phi, prm)
    m = orc.macros(f, g, prm)
    tot0 = m["totals"].copy()
    n = nx * ny * nz
    for _ in range(20):
        force = m["force"].reshape(3, -1).sum(1)
        j_before = m["totals"][2:].copy()
        f, g = orc.step(f, g, prm, 5)  # advance 5, check the last step below
        m = orc.macros(f, g, prm)
        assert abs(m["totals"][0] - tot0[0]) < 1e-13 * n
        assert abs(m["totals"][1] - tot0[1]) < 1e-13 * n
    # Guo: one step changes total momentum by exactly the total force
    f1, g1 = orc.step(f, g, prm, 1)
    m1 = orc.macros(f1, g1, prm)
    force = m["force"].reshape(3, -1).sum(1)
    assert np.abs((m1["totals"][2:] - m["totals"][2:]) - force).max() < 1e-15 * n


# --------------------------------------------------------------------------
# Fixed point: a uniform equilibrium (any uniform u) is unchanged by a step
# (catches a collision that does not relax towards its own equilibrium).


@pytest.mark.parametrize("u0", [(0.0, 0.0, 0.0), (0.03, -0.02, 0.01)])
def test_uniform_equilibrium_is_fixed_point(orc, u0):
    prm = orc.param_vector(tau_f=0.7, tau_g=1.4)
    shape = (4, 5, 6)
    phi = np.full(shape, -0.4)
    rho = np.full(shape, 1.02)
    u = np.zeros((3,) + shape)
    for a in range(3):
        u[a] = u0[a]
    f, g = orc.init(phi, prm, rho=rho, u=u)
    f1, g1 = orc.step(f, g, prm, 1)
    eps = np.finfo(np.float64).eps
    assert np.abs(f1 - f).max() <= 4 * eps * np.abs(f).max()
    assert np.abs(g1 - g).max() <= 4 * eps * np.abs(g).max()


# --------------------------------------------------------------------------
# Hydrodynamic limits.


def _project(field, k_index, axis_len):
    x = np.arange(axis_len)
    return 2.0 / axis_len * float((field * np.sin(2 * math.pi * k_index * x / axis_len)).sum())


def _shear_rate(orc, ny, tau_f, t0=100, t1=1000, prm=None):
    prm = orc.param_vector(tau_f=tau_f) if prm is None else prm
    nx = nz = 1
    u = inputs.shear_wave_u(nx, ny, nz, 1e-3)
    phi = np.zeros((nz, ny, nx))
    f, g = orc.init(phi, prm, u=u)
    f, g = orc.step(f, g, prm, t0)
    a0 = _project(orc.macros(f, g, prm)["u"][0, 0, :, 0], 1, ny)
    f, g = orc.step(f, g, prm, t1 - t0)
    a1 = _project(orc.macros(f, g, prm)["u"][0, 0, :, 0], 1, ny)
    return math.log(a0 / a1) / (t1 - t0)


@pytest.mark.parametrize("tau_f", [0.6, 1.0, 1.5])
def test_shear_wave_viscosity(orc, tau_f):
    """Transverse wave decays at nu k^2 with nu = (tau_f - 1/2)/3 (catches a
    wrong relaxation time or a collision without 1/tau)."""
    ny = 64
    k = 2 * math.pi / ny
    nu = (tau_f - 0.5) / 3.0
    rate = _shear_rate(orc, ny, tau_f)
    assert abs(rate / (nu * k * k) - 1.0) < 0.01
    if tau_f == 1.0:
        # error is second order in k: halving k cuts it by ~4
        assert golden_constants()["nu"] == pytest.approx(nu, rel=1e-15)
        e64 = abs(rate / (nu * k * k) - 1.0)
        rate32 = _shear_rate(orc, 32, tau_f)
        e32 = abs(rate32 / (nu * (2 * math.pi / 32) ** 2) - 1.0)
        assert e32 / max(e64, 1e-12) > 3.0


def test_linear_spinodal_growth_rate(orc):
    """A small sine mode of phi grows at omega = M lambda (-A - kappa lambda),
    M = Gamma (tau_g - 1/2), lambda = 2(1 - cos k) (catches a wrong mobility,
    a wrong Gamma mu term in g_eq, a wrong sign of A or kappa)."""
    const = golden_constants()
    prm = orc.param_vector()
    A, kappa = prm[0], prm[2]
    nx = 32
    k = 2 * math.pi / nx
    lam = 2.0 * (1.0 - math.cos(k))
    M = const["M"]
    omega = M * lam * (-A - kappa * lam)
    phi = inputs.sine_phi(nx, 1, 1, 1e-4)
    f, g = orc.init(phi, prm)
    f, g = orc.step(f, g, prm, 200)
    a0 = _project(g.sum(0)[0, 0, :], 1, nx)
    f, g = orc.step(f, g, prm, 800)
    a1 = _project(g.sum(0)[0, 0, :], 1, nx)
    rate = math.log(a1 / a0) / 800
    assert abs(rate / omega - 1.0) < 0.03


def test_phi_advected_by_uniform_flow(orc):
    """With a uniform velocity U the phi pattern moves U sites per step
    (catches a wrong phi u term in g_eq or u missing from it)."""
    prm = orc.param_vector(A=0.0, B=0.0, kappa=0.0)
    nx = 64
    U = 0.05
    phi = inputs.sine_phi(nx, 1, 1, 1e-3)
    u = np.zeros((3, 1, 1, nx))
    u[0] = U
    f, g = orc.init(phi, prm, u=u)
    t = 200
    f, g = orc.step(f, g, prm, t)
    prof = g.sum(0)[0, 0, :]
    phase = np.angle(np.fft.fft(prof)[1])
    # sin(kx - k U t) has FFT phase -pi/2 - k U t
    shift = -(phase + math.pi / 2) / (2 * math.pi / nx)
    assert abs(shift - U * t) < 0.01 * U * t


def _relaxed_tanh_slab(orc, kappa, B, steps=400, nx=64):
    prm = orc.param_vector(kappa=kappa, B=B)
    A = prm[0]
    xi = math.sqrt(-2.0 * kappa / A)
    phi0 = math.sqrt(-A / B)
    x = np.arange(nx)
    prof = phi0 * np.tanh((x - 15.5) / xi) * np.tanh((47.5 - x) / xi)
    f, g = orc.init(prof[None, None, :].copy(), prm)
    f, g = orc.step(f, g, prm, steps)
    return xi, phi0, orc.macros(f, g, prm)


@pytest.mark.parametrize("B", [0.0625, 0.125])
def test_flat_interface_bulk_and_width(orc, B):
    """Two flat interfaces (normal to x) relax to bulk values +-phi0,
    phi0 = sqrt(-A/B), with a tanh profile of width xi = sqrt(-2 kappa/A).
    The width of the discrete profile approaches xi with a gap of second
    order in h/xi (h = 1 site), bounded here by 0.25 (h/xi)^2; the gap must
    shrink when kappa is doubled (catches a wrong A, B or kappa in mu, a
    wrong Laplacian, a force of the wrong sign).

    The interface is started from the continuum profile and measured after
    400 steps: the 1-D flat interface of this discretisation slowly grows a
    checkerboard velocity mode (k = pi), so it is not run to a late steady
    state."""
    gaps = []
    for kappa in (0.04, 0.08):
        xi, phi0, m = _relaxed_tanh_slab(orc, kappa, B)
        p = m["phi"][0, 0, :]
        bulk_in, bulk_out = p[31], p[0]
        assert abs(bulk_in - phi0) < 1e-3 * phi0
        assert abs(bulk_out + phi0) < 1e-3 * phi0
        # sites 15 and 16 straddle the interface centre at 15.5
        xi_fit = 0.5 / math.atanh(p[16] / bulk_in)
        gap = abs(xi_fit / xi - 1.0)
        assert gap < 0.25 / xi ** 2
        gaps.append(gap)
        assert np.abs(m["u"]).max() < 5e-3
    assert gaps[1] < gaps[0] / 1.5


# --------------------------------------------------------------------------
# Tangent-linear model against central finite differences of the plain
# double path (catches a wrong derivative rule in the dual numbers).


@pytest.mark.parametrize("stencil", [7, 19])
def test_tangent_linear_matches_finite_differences(orc, stencil):
    nz, ny, nx = 5, 6, 4
    prm = orc.param_vector(tau_f=0.9, stencil=stencil)
    phi0 = inputs.spinodal_phi(nx, ny, nz, seed=21, amplitude=0.3)
    target = inputs.spinodal_phi(nx, ny, nz, seed=22, amplitude=0.3)
    rng = np.random.default_rng(5)
    dphi = rng.standard_normal(phi0.shape)
    dprm = np.zeros(len(prm))  # the selector entries are not differentiated
    dprm[2] = 0.3  # kappa
    dprm[4] = -0.7  # tau_f
    steps = 6
    L, dL = orc.loss_jvp(phi0, target, prm, steps, dphi0=dphi, dprm=dprm)
    assert L == pytest.approx(orc.loss(phi0, target, prm, steps), rel=1e-13)
    h = 1e-5
    lp = orc.loss(phi0 + h * dphi, target, prm + h * dprm, steps)
    lm = orc.loss(phi0 - h * dphi, target, prm - h * dprm, steps)
    fd = (lp - lm) / (2 * h)
    assert dL == pytest.approx(fd, rel=1e-7)


# --------------------------------------------------------------------------
# 19-point isotropic stencils (catches weights swapped between axis and
# diagonal neighbours, a missing or doubled neighbour, a sign error in the
# gradient, an axis mix-up, and any form whose leading error is anisotropic).


def _axis_field(shape, axis, seed):
    """Random values along one axis, constant across the other two."""
    rng = np.random.default_rng(seed)
    line = rng.standard_normal(shape[axis])
    view = [1, 1, 1]
    view[axis] = shape[axis]
    return np.broadcast_to(line.reshape(view), shape).copy()


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_isotropic_stencils_reduce_to_1d_forms(orc, axis):
    """On a field that varies along one axis only, every diagonal neighbour
    of the 19-point forms sees the same value as an axis neighbour, and the
    sums collapse to the 1-D second difference and central difference: the
    7-point results, to rounding."""
    phi = _axis_field((6, 7, 8), axis, seed=axis)
    assert np.abs(orc.laplacian(phi, 19) - orc.laplacian(phi, 7)).max() < 1e-14
    assert np.abs(orc.gradient(phi, 19) - orc.gradient(phi, 7)).max() < 1e-14


def test_isotropic_stencils_on_constants_and_sums(orc):
    rng = np.random.default_rng(4)
    phi = rng.standard_normal((5, 6, 7))
    assert np.abs(orc.laplacian(np.full((5, 6, 7), 0.7), 19)).max() < 1e-15
    assert np.abs(orc.gradient(np.full((5, 6, 7), 0.7), 19)).max() < 1e-15
    # periodic sums of differences telescope
    assert abs(orc.laplacian(phi, 19).sum()) < 1e-12
    assert np.abs(orc.gradient(phi, 19).reshape(3, -1).sum(1)).max() < 1e-12


def _modes(n):
    z, y, x = np.meshgrid(np.arange(4), np.arange(n), np.arange(n), indexing="ij")
    return x, y, z


@pytest.mark.parametrize("m", [(5, 0, 0), (3, 4, 0), (0, 4, 3)])
def test_isotropic_laplacian_symbol(orc, m):
    """Both Laplacians have the discrete Fourier modes as eigenfunctions. For
    the 19-point form, sum_i w_i c c c c is isotropic on D3Q19, so its symbol
    is -|k|^2 + |k|^4/12 + O(k^6) in every direction; the 7-point symbol's k^4
    term is sum_a k_a^4/12, which depends on the direction."""
    n = 64
    x, y, _ = _modes(n)
    k = np.array(m[:2]) * 2 * math.pi / n if m[2] == 0 else None
    if k is None:  # (0, 4, 3): along y and z needs nz = 64
        z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(4), indexing="ij")
        kv = np.array([0.0, 4.0, 3.0]) * 2 * math.pi / n
        arg = kv[1] * y + kv[2] * z + 0.3
    else:
        kv = np.array([k[0], k[1], 0.0])
        arg = kv[0] * x + kv[1] * y + 0.3
    phi = np.cos(arg)
    kk = float(kv @ kv)
    s19 = float((orc.laplacian(phi, 19) * phi).sum() / (phi * phi).sum())
    s7 = float((orc.laplacian(phi, 7) * phi).sum() / (phi * phi).sum())
    assert abs(s19 - (-kk + kk * kk / 12)) < 1e-4
    aniso7 = sum(ka ** 4 for ka in kv) / 12 - kk * kk / 12  # 7-point k^4 term minus the isotropic one
    assert abs((s7 - s19) - aniso7) < 2e-4


def test_isotropic_gradient_follows_k(orc):
    """grad of sin(k.x) is G(k) cos(k.x). For the 19-point form G is k (1 -
    |k|^2/6 + ...): parallel to k to O(k^5). The central difference gives
    sin(k_a), whose direction departs from k at O(k^3)."""
    n = 64
    x, y, _ = _modes(n)
    kv = np.array([3.0, 4.0, 0.0]) * 2 * math.pi / n
    arg = kv[0] * x + kv[1] * y
    h, cs = np.sin(arg), np.cos(arg)

    def symbol(st):
        gr = orc.gradient(h, st)
        return np.array([(gr[a] * cs).sum() / (cs * cs).sum() for a in range(3)])

    def angle(g):
        return math.acos(min(1.0, float(g @ kv) / (np.linalg.norm(g) * np.linalg.norm(kv))))

    g19, g7 = symbol(19), symbol(7)
    kk = float(kv @ kv)
    assert angle(g19) < 1e-4 < 1e-3 < angle(g7)
    assert np.abs(g19 - kv * (1 - kk / 6)).max() < 1e-3
    assert np.abs(g7 - np.sin(kv)).max() < 1e-14


def test_isotropic_spinodal_growth_rate(orc):
    """With the 19-point stencils a diagonal mode (k along (3, 4, 0)) grows at
    omega = M lambda (-A - kappa lambda) with lambda = |k|^2 - |k|^4/12 (the
    isotropic symbol above), at the same |k| = 2 pi / 32 as the axis-mode pin
    above: the step uses the selected stencil in mu."""
    const = golden_constants()
    prm = orc.param_vector(stencil=19)
    A, kappa = prm[0], prm[2]
    n = 160
    kv = np.array([3.0, 4.0]) * 2 * math.pi / n  # |k| = 5 (2 pi / 160) = 2 pi / 32
    kk = float(kv @ kv)
    lam = kk - kk * kk / 12
    omega = const["M"] * lam * (-A - kappa * lam)
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    basis = np.cos(kv[0] * x + kv[1] * y)[None]
    f, g = orc.init(1e-4 * basis, prm)
    f, g = orc.step(f, g, prm, 200)
    a0 = float((g.sum(0) * basis).sum())
    f, g = orc.step(f, g, prm, 800)
    a1 = float((g.sum(0) * basis).sum())
    rate = math.log(a1 / a0) / 800
    assert abs(rate / omega - 1.0) < 0.03


@pytest.mark.parametrize("stencil", [7, 19])
def test_step_uses_selected_stencils(orc, stencil):
    """mu, the force and grad(phi) of the macroscopic output are built from
    the stencil pair the parameters select (each pinned above): a step that
    ignored the selection would fail one of the two cases."""
    prm = orc.param_vector(stencil=stencil, kappa=0.07)
    A, B, kappa = prm[0], prm[1], prm[2]
    phi = inputs.spinodal_phi(9, 8, 7, seed=31, amplitude=0.4)
    f, g = orc.init(phi, prm)
    m = orc.macros(f, g, prm)
    phi = m["phi"]  # sum of g, within rounding of the input
    mu = A * phi + B * phi ** 3 - kappa * orc.laplacian(phi, stencil)
    assert np.abs(m["mu"] - mu).max() < 1e-15
    assert np.abs(m["force"] + phi * orc.gradient(m["mu"], stencil)).max() < 1e-16
    assert np.abs(m["grad_phi"] - orc.gradient(phi, stencil)).max() < 1e-16
    other = 19 if stencil == 7 else 7
    assert np.abs(m["mu"] - (A * phi + B * phi ** 3 - kappa * orc.laplacian(phi, other))).max() > 1e-4


# --------------------------------------------------------------------------
# Force as the divergence of the chemical stress (catches a wrong bulk
# pressure, a missing -kappa phi lap(phi) or -kappa/2 |grad phi|^2 term, a
# transposed or non-symmetric stress, a divergence taken over the wrong
# index, and a step that ignores the force selection).


def test_stress_of_uniform_phi(orc):
    """No gradients: P = p_b I with the bulk pressure p_b = phi f'(phi) - f
    of f = A phi^2/2 + B phi^4/4, i.e. A phi^2/2 + 3 B phi^4/4."""
    prm = orc.param_vector(A=-0.07, B=0.09)
    A, B = prm[0], prm[1]
    phi = np.full((4, 5, 6), 0.61)
    P = orc.stress(phi, prm)
    pb = 0.5 * A * 0.61 ** 2 + 0.75 * B * 0.61 ** 4
    for c in range(3):
        assert np.abs(P[c] - pb).max() < 1e-16
    assert np.abs(P[3:]).max() == 0.0


@pytest.mark.parametrize("stencil", [7, 19])
def test_stress_of_a_field_varying_along_x(orc, stencil):
    """phi(x) only: the off-diagonal stress vanishes, P_yy = P_zz, and
    P_xx - P_yy = kappa (d_x phi)^2 with the selected gradient."""
    prm = orc.param_vector(kappa=0.06, stencil=stencil)
    phi = _axis_field((5, 6, 16), 2, seed=8)
    P = orc.stress(phi, prm)
    gx = orc.gradient(phi, stencil)[0]
    assert np.abs(P[3:]).max() < 1e-17
    assert np.abs(P[1] - P[2]).max() < 1e-17
    assert np.abs((P[0] - P[1]) - 0.06 * gx * gx).max() < 1e-15


@pytest.mark.parametrize("stencil", [7, 19])
def test_stress_force_sums_to_zero_and_conserves_momentum(orc, stencil):
    """On a periodic lattice a discrete divergence telescopes: sum_x F = 0,
    so the Guo step conserves total momentum exactly, over many steps. The
    potential form -phi grad(mu) has no such property."""
    nz, ny, nx = 6, 7, 8
    phi = inputs.spinodal_phi(nx, ny, nz, seed=33, amplitude=0.5)
    stress = orc.param_vector(force="stress", stencil=stencil, kappa=0.06)
    pot = orc.param_vector(stencil=stencil, kappa=0.06)
    f, g = orc.init(phi, stress)
    m = orc.macros(f, g, stress)
    assert np.abs(m["force"].reshape(3, -1).sum(1)).max() < 1e-15
    mp = orc.macros(*orc.init(phi, pot), pot)
    assert np.abs(mp["force"].reshape(3, -1).sum(1)).max() > 1e-6
    j0 = m["totals"][2:].copy()
    f, g = orc.step(f, g, stress, 50)
    j1 = orc.macros(f, g, stress)["totals"][2:]
    assert np.abs(j1 - j0).max() < 1e-13


def test_stress_force_converges_to_potential_form(orc):
    """div P = phi grad(mu) in the continuum (Gibbs-Duhem): for the same smooth
    field sampled twice as finely (kappa and the lattice spacing scaled
    together), the difference of the two discrete forces falls by about 4."""
    def gap(n):
        prm_s = orc.param_vector(force="stress", kappa=0.04 * (n / 32) ** 2)
        prm_p = orc.param_vector(kappa=0.04 * (n / 32) ** 2)
        z, y, x = np.meshgrid(np.arange(4), np.arange(n), np.arange(n), indexing="ij")
        phi = 0.6 * np.sin(2 * math.pi * x / n) * np.cos(2 * math.pi * y / n)
        fs = orc.macros(*orc.init(phi, prm_s), prm_s)["force"]
        fp = orc.macros(*orc.init(phi, prm_p), prm_p)["force"]
        return np.abs(fs - fp).max() / np.abs(fp).max()
    g32, g64 = gap(32), gap(64)
    assert g32 < 0.05
    assert 3.0 < g32 / g64 < 5.0


def test_tangent_linear_with_stress_force(orc):
    nz, ny, nx = 5, 6, 4
    prm = orc.param_vector(tau_f=0.9, force="stress")
    phi0 = inputs.spinodal_phi(nx, ny, nz, seed=21, amplitude=0.3)
    target = inputs.spinodal_phi(nx, ny, nz, seed=22, amplitude=0.3)
    dphi = np.random.default_rng(6).standard_normal(phi0.shape)
    dprm = np.zeros(len(prm))
    dprm[2], dprm[4] = 0.3, -0.7
    steps = 6
    _, dL = orc.loss_jvp(phi0, target, prm, steps, dphi0=dphi, dprm=dprm)
    h = 1e-5
    fd = (orc.loss(phi0 + h * dphi, target, prm + h * dprm, steps) -
          orc.loss(phi0 - h * dphi, target, prm - h * dprm, steps)) / (2 * h)
    assert dL == pytest.approx(fd, rel=1e-7)


# --------------------------------------------------------------------------
# Two-relaxation-time collision of f (catches a wrong even/odd split of f,
# feq or the Guo source, a wrong prefactor on either part, a tau- that moves
# the shear viscosity, and any loss of mass or momentum).


def test_trt_with_equal_rates_is_bgk(orc):
    """Lambda = (tau - 1/2)^2 makes tau- = tau+: the two-rate collision is
    the one-rate one, to rounding."""
    tau = 0.8
    bgk = orc.param_vector(tau_f=tau)
    trt = orc.param_vector(tau_f=tau, collision="trt", magic=(tau - 0.5) ** 2)
    phi = inputs.spinodal_phi(6, 5, 4, seed=12, amplitude=0.5)
    rng = np.random.default_rng(2)
    u = 0.05 * rng.standard_normal((3,) + phi.shape)
    fa, ga = orc.step(*orc.init(phi, bgk, u=u), bgk, 10)
    fb, gb = orc.step(*orc.init(phi, trt, u=u), trt, 10)
    assert np.abs(fa - fb).max() < 1e-14
    assert np.abs(ga - gb).max() < 1e-15


@pytest.mark.parametrize("magic", [0.1875, 0.25, 1.0])
def test_trt_shear_viscosity_depends_on_tau_plus_only(orc, magic):
    """The shear wave decays at nu k^2 with nu = (tau_f - 1/2)/3 whatever the
    odd-part rate (the magic parameter moves only higher-order terms)."""
    tau, ny = 0.7, 64
    k = 2 * math.pi / ny
    nu = (tau - 0.5) / 3.0
    prm = orc.param_vector(tau_f=tau, collision="trt", magic=magic)
    rate = _shear_rate(orc, ny, tau, prm=prm)
    assert abs(rate / (nu * k * k) - 1.0) < 0.01


def test_trt_conserves_mass_and_adds_the_force(orc):
    prm = orc.param_vector(tau_f=0.9, collision="trt", magic=0.25, kappa=0.06)
    phi = inputs.spinodal_phi(7, 6, 5, seed=14, amplitude=0.5)
    f, g = orc.init(phi, prm)
    m = orc.macros(f, g, prm)
    t0 = m["totals"].copy()
    force = m["force"].reshape(3, -1).sum(1)
    f1, g1 = orc.step(f, g, prm, 1)
    t1 = orc.macros(f1, g1, prm)["totals"]
    assert abs(t1[0] - t0[0]) < 1e-13 * phi.size
    assert abs(t1[1] - t0[1]) < 1e-13 * phi.size
    assert np.abs((t1[2:] - t0[2:]) - force).max() < 1e-14


def test_trt_uniform_equilibrium_is_fixed_point(orc):
    prm = orc.param_vector(tau_f=0.7, collision="trt", magic=0.1875)
    phi = np.full((4, 4, 4), 0.3)
    u = np.zeros((3, 4, 4, 4))
    u[0], u[2] = 0.02, -0.01
    f, g = orc.init(phi, prm, u=u)
    f1, g1 = orc.step(f, g, prm, 1)
    eps = np.finfo(np.float64).eps
    assert np.abs(f1 - f).max() <= 4 * eps * np.abs(f).max()
    assert np.abs(g1 - g).max() <= 4 * eps * np.abs(g).max()


def test_tangent_linear_with_trt(orc):
    nz, ny, nx = 5, 6, 4
    prm = orc.param_vector(tau_f=0.9, collision="trt", magic=0.25)
    phi0 = inputs.spinodal_phi(nx, ny, nz, seed=21, amplitude=0.3)
    target = inputs.spinodal_phi(nx, ny, nz, seed=22, amplitude=0.3)
    dphi = np.random.default_rng(6).standard_normal(phi0.shape)
    dprm = np.zeros(len(prm))
    dprm[2], dprm[4] = 0.3, -0.7
    steps = 6
    _, dL = orc.loss_jvp(phi0, target, prm, steps, dphi0=dphi, dprm=dprm)
    h = 1e-5
    fd = (orc.loss(phi0 + h * dphi, target, prm + h * dprm, steps) -
          orc.loss(phi0 - h * dphi, target, prm - h * dprm, steps)) / (2 * h)
    assert dL == pytest.approx(fd, rel=1e-7)


# --------------------------------------------------------------------------
# The discrete flat interface: the 1-D solution of the discrete equilibrium
# condition is an exact fixed point of the whole step.


def _discrete_interface(n, A, B, kappa, guess):
    """Newton solve of A phi + B phi^3 - kappa (phi(x+1) + phi(x-1) - 2 phi)
    = mu_c on a periodic 1-D lattice of n sites, with mu_c unknown and the
    total of phi fixed to that of the guess. Returns (phi, mu_c)."""
    phi = guess.astype(np.float64).copy()
    total = phi.sum()
    mu = 0.0
    eye = np.eye(n)
    shift = np.roll(eye, 1, axis=1) + np.roll(eye, -1, axis=1)
    for _ in range(60):
        lap = np.roll(phi, 1) + np.roll(phi, -1) - 2 * phi
        r = np.concatenate([A * phi + B * phi ** 3 - kappa * lap - mu, [phi.sum() - total]])
        if np.abs(r).max() < 1e-15:
            break
        J = np.zeros((n + 1, n + 1))
        J[:n, :n] = np.diag(A + 3 * B * phi ** 2 + 2 * kappa) - kappa * shift
        J[:n, n] = -1.0
        J[n, :n] = 1.0
        d = np.linalg.solve(J, -r)
        phi += d[:n]
        mu += d[n]
    return phi, mu


@pytest.mark.parametrize("kappa", [0.04, 0.08])
@pytest.mark.parametrize("taus", [(1.0, 1.0), (0.8, 1.3)])
@pytest.mark.parametrize("stencil", [7, 19])
def test_discrete_flat_interface_is_a_fixed_point(orc, kappa, taus, stencil):
    """The discrete 1-D equilibrium (uniform mu with the 7-point Laplacian,
    two interfaces normal to x, solved by Newton here) is left unchanged by
    every step to 1e-12, with u = 0: mu uniform makes F = 0, and for a
    profile along x the propagated parts of g^eq from the axis and the
    diagonal directions cancel in phi for any shift (the rest, axis and
    diagonal weights of g^eq at u = 0 are 5/6, 1/18, -1/72 per unit phi), so
    phi never moves whatever the relaxation times. Catches a wrong
    coefficient in mu or g^eq, a wrong Laplacian or propagation; a profile
    solved with kappa off by 1 % moves by more than 1e-4. On a profile along
    x the 19-point Laplacian equals the 7-point one (1/3 of the axis pair
    plus 4 x 1/6 of the diagonal pairs), so the same solution serves both."""
    A, B = -0.0625, 0.0625
    n = 64
    x = np.arange(n)
    xi = math.sqrt(-2 * kappa / A)
    guess = np.tanh((x - 15.5) / xi) * np.tanh((47.5 - x) / xi)
    phi1, mu_c = _discrete_interface(n, A, B, kappa, guess)
    assert abs(phi1.max() - 1.0) < 1e-3 and abs(phi1.min() + 1.0) < 1e-3  # the two bulk phases
    prm = orc.param_vector(kappa=kappa, tau_f=taus[0], tau_g=taus[1], stencil=stencil)
    phi3 = np.broadcast_to(phi1, (4, 4, n)).copy()
    f, g = orc.init(phi3, prm)
    f, g = orc.step(f, g, prm, 20)
    m = orc.macros(f, g, prm)
    assert np.abs(m["phi"] - phi3).max() < 1e-12
    assert np.abs(m["u"]).max() < 1e-13
    assert np.abs(m["mu"] - mu_c).max() < 1e-12
    # teeth: the solution for a kappa 1 % off is not a fixed point
    phi_off, _ = _discrete_interface(n, A, B, 1.01 * kappa, guess)
    f, g = orc.init(np.broadcast_to(phi_off, (4, 4, n)).copy(), prm)
    f, g = orc.step(f, g, prm, 20)
    assert np.abs(orc.macros(f, g, prm)["phi"] - phi_off).max() > 1e-4
