"""Pins of the liquid-crystal oracle (oracle/lc_oracle.cpp) against what the
Landau-de Gennes free energy and the Beris-Edwards equation fix independently
of the oracle's code:

- the molecular field of a uniform uniaxial Q = S (n n - I/3) equals the
  closed form -(3/2) df_b/dS (n n - I/3) derived from the scalar bulk free
  energy f_b(S), and vanishes at the bulk order S = q0(gamma) =
  1/4 + 3/4 sqrt(1 - 8/(3 gamma)) for any director;
- such a uniform equilibrium, at rest, is a fixed point of the coupled step;
- in the isotropic phase a small mode relaxes at the linear rate
  Gamma (A0 (1 - gamma/3) + kappa lambda), lambda the 7-point eigenvalue;
- the co-rotation term: a rigid rotation (antisymmetric W) gives the
  commutator Om Q - Q Om for any xi; a pure strain D on the isotropic state
  gives 2 xi D / 3; no flow gives 0;
- upwind advection with Courant number 1 shifts Q by one site (to the
  rounding of one difference), with Courant 1/2 it averages the site and its
  upwind neighbour;
- the force is the divergence of a stress: it sums to zero, and the coupled
  step conserves mass and total momentum;
- Onsager reciprocity of the flow coupling: for any traceless velocity
  gradient W, the stress does work sigma : W = -H : S(W, Q) (the reactive
  stress and the co-rotation term are partners), checked on uniform random
  Q with xi = 0.7, which ties the xi and commutator terms of the stress to
  the co-rotation term;
- Gibbs-Duhem: for xi = 0 the divergence of the chemical stress equals
  -H : d_a Q + d_b (Q H - H Q)_ab, the continuum identity of this free
  energy, to second order in the lattice spacing.
"""

import math

import numpy as np
import pytest

import oracle

A0, GAMMA_NEM, KAPPA = 0.01, 3.0, 0.01


def q5(Q):
    """Five stored components of a full symmetric traceless tensor (..., 3, 3)."""
    return np.stack([Q[..., 0, 0], Q[..., 0, 1], Q[..., 0, 2], Q[..., 1, 1], Q[..., 1, 2]])


def full(q):
    """Full tensor (..., 3, 3) from the five components (5, ...)."""
    xx, xy, xz, yy, yz = q
    return np.stack([np.stack([xx, xy, xz], -1), np.stack([xy, yy, yz], -1), np.stack([xz, yz, -xx - yy], -1)], -2)


def uniform(Q, shape):
    return np.broadcast_to(q5(Q)[(...,) + (None,) * 3], (5,) + shape).copy()


def uniaxial(S, n):
    n = np.asarray(n, dtype=float)
    n = n / np.linalg.norm(n)
    return S * (np.outer(n, n) - np.eye(3) / 3.0)


def q0(gamma):
    return 0.25 + 0.75 * math.sqrt(1.0 - 8.0 / (3.0 * gamma))


def bulk_h_closed_form(S, gamma):
    """Coefficient h of H = h (n n - I/3) for uniform uniaxial Q = S (n n - I/3):
    f_b(S) = A0/3 (1 - gamma/3) S^2 - 2 A0 gamma/27 S^3 + A0 gamma/9 S^4, and
    H : (n n - I/3) = -df_b/dS with (n n - I/3):(n n - I/3) = 2/3."""
    dfds = 2 * A0 / 3 * (1 - gamma / 3) * S - 2 * A0 * gamma / 9 * S ** 2 + 4 * A0 * gamma / 9 * S ** 3
    return -1.5 * dfds


@pytest.mark.parametrize("S", [0.1, 0.3, 0.5, 0.7])
def test_molecular_field_of_uniform_uniaxial_order(S):
    prm = oracle.lc_param_vector(A0=A0, gamma=GAMMA_NEM, kappa=KAPPA)
    rng = np.random.default_rng(int(S * 100))
    n = rng.standard_normal(3)
    shape = (3, 4, 5)
    h, _ = oracle.lc_field(uniform(uniaxial(S, n), shape), prm)
    want = bulk_h_closed_form(S, GAMMA_NEM) * (np.outer(n, n) / n.dot(n) - np.eye(3) / 3)
    assert np.allclose(full(h), want, rtol=0, atol=1e-16)


def test_bulk_order_is_an_equilibrium_and_a_fixed_point():
    gamma = 3.2
    prm = oracle.lc_param_vector(A0=A0, gamma=gamma, kappa=KAPPA)
    S = q0(gamma)
    assert abs(bulk_h_closed_form(S, gamma)) < 1e-17
    shape = (4, 4, 4)
    Q = uniform(uniaxial(S, [1.0, 2.0, -0.5]), shape)
    h, _ = oracle.lc_field(Q, prm)
    assert np.abs(h).max() < 1e-17
    f = oracle.lc_init(shape, prm)
    f1, Q1 = oracle.lc_step(f, Q, prm, 5)
    assert np.abs(Q1 - Q).max() < 1e-16 and np.abs(f1 - f).max() < 1e-16


@pytest.mark.parametrize("kappa", [0.0, 0.02])
def test_isotropic_mode_relaxes_at_the_linear_rate(kappa):
    gamma, Gamma, eps, nx = 2.0, 0.3, 1e-9, 16
    prm = oracle.lc_param_vector(A0=A0, gamma=gamma, kappa=kappa, Gamma=Gamma)
    k = 2 * math.pi * 2 / nx
    M = np.array([[0.3, 0.1, -0.2], [0.1, -0.5, 0.4], [-0.2, 0.4, 0.2]])
    x = np.arange(nx)
    amp = eps * np.sin(k * x)[None, None, :]
    Q = q5(M)[:, None, None, None] * amp[None]
    Q = np.broadcast_to(Q, (5, 3, 3, nx)).copy()
    h, _ = oracle.lc_field(Q, prm)
    Q1 = oracle.lc_update(Q, np.zeros((3,) + Q.shape[1:]), h, prm)
    lam = 2 * (1 - math.cos(k))
    factor = 1 - Gamma * (A0 * (1 - gamma / 3) + kappa * lam)
    mask = np.abs(amp[0, 0]) > 0.5 * eps
    ratio = Q1[..., mask] / Q[..., mask]
    assert np.allclose(ratio, factor, rtol=0, atol=1e-10)  # quadratic terms: ~A0 gamma eps ~ 1e-11


def test_corotation_closed_forms():
    prm = oracle.lc_param_vector(xi=0.7)
    rng = np.random.default_rng(3)
    A = rng.standard_normal((3, 3))
    Q = A + A.T
    Q -= np.trace(Q) / 3 * np.eye(3)
    Om = rng.standard_normal((3, 3))
    Om = 0.5 * (Om - Om.T)
    assert np.allclose(oracle.lc_corotation(Om, Q, prm), Om @ Q - Q @ Om, atol=1e-15)
    D = rng.standard_normal((3, 3))
    D = D + D.T
    D -= np.trace(D) / 3 * np.eye(3)
    assert np.allclose(oracle.lc_corotation(D, np.zeros((3, 3)), prm), 2 * 0.7 * D / 3, atol=1e-15)
    assert np.allclose(oracle.lc_corotation(np.zeros((3, 3)), Q, prm), 0.0, atol=0)


@pytest.mark.parametrize("courant", [1.0, -1.0, 0.5])
def test_upwind_advection(courant):
    prm = oracle.lc_param_vector(Gamma=0.0, xi=0.7)
    rng = np.random.default_rng(5)
    Q = 0.1 * rng.standard_normal((5, 3, 4, 8))
    u = np.zeros((3,) + Q.shape[1:])
    u[0] = courant
    Q1 = oracle.lc_update(Q, u, np.zeros_like(Q), prm)
    # Q - c (Q - Q_upwind): the upwind value to the rounding of one difference
    if courant == 1.0:
        assert np.allclose(Q1, np.roll(Q, 1, axis=3), rtol=0, atol=1e-16)
    elif courant == -1.0:
        assert np.allclose(Q1, np.roll(Q, -1, axis=3), rtol=0, atol=1e-16)
    else:
        assert np.allclose(Q1, 0.5 * (Q + np.roll(Q, 1, axis=3)), rtol=0, atol=1e-16)


def test_force_sums_to_zero_and_momentum_is_conserved():
    prm = oracle.lc_param_vector(A0=A0, gamma=GAMMA_NEM, kappa=KAPPA, xi=0.7)
    rng = np.random.default_rng(7)
    shape = (6, 5, 8)
    Q = 0.2 * rng.standard_normal((5,) + shape)
    f = oracle.lc_init(shape, prm, rho=1 + 0.01 * rng.standard_normal(shape))
    m = oracle.lc_macros(f, Q, prm)
    assert np.abs(m["force"].sum(axis=(1, 2, 3))).max() < 1e-15
    c, _ = oracle.lattice()
    mom0 = np.einsum("ia,i...->a...", c, f).reshape(3, -1).sum(axis=1)
    mass0 = f.sum()
    f1, Q1 = oracle.lc_step(f, Q, prm, 10)
    assert abs(f1.sum() - mass0) < 1e-12
    assert np.abs(np.einsum("ia,i...->a...", c, f1).reshape(3, -1).sum(axis=1) - mom0).max() < 1e-13


def _gibbs_duhem_gap(n):
    """Max |div sigma - (-H:d_a Q + d_b (QH - HQ)_ab)| for a smooth field on an
    n^3 lattice (one period in each direction), with kappa scaled so the
    field's elastic and bulk terms keep their ratio as the spacing halves."""
    scale = n / 16
    prm = oracle.lc_param_vector(A0=A0, gamma=GAMMA_NEM, kappa=KAPPA * scale ** 2, xi=0.0)
    x = 2 * math.pi * np.arange(n) / n
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    X, Y, Z = X.transpose(2, 1, 0), Y.transpose(2, 1, 0), Z.transpose(2, 1, 0)  # (z, y, x) order
    theta = 0.6 * np.sin(X) + 0.4 * np.cos(Y + Z)
    phi = 0.5 * np.cos(Z) + 0.3 * np.sin(X - Y)
    nvec = np.stack([np.cos(theta) * np.cos(phi), np.sin(theta) * np.cos(phi), np.sin(phi)])
    S = 0.4 + 0.1 * np.sin(X + Y)
    Qf = S[..., None, None] * (np.einsum("a...,b...->...ab", nvec, nvec) - np.eye(3) / 3)
    q = q5(Qf)
    h, _ = oracle.lc_field(q, prm)
    f = oracle.lc_init(q.shape[1:], prm)
    F = oracle.lc_macros(f, q, prm)["force"]
    H = full(h)

    def d(a, arr):  # central difference along axis a (0 = x) of (..., z, y, x) arrays
        ax = {0: -1, 1: -2, 2: -3}[a]
        return 0.5 * (np.roll(arr, -1, axis=ax) - np.roll(arr, 1, axis=ax))

    Qm = Qf
    comm = np.einsum("...ac,...cb->...ab", Qm, H) - np.einsum("...ac,...cb->...ab", H, Qm)
    want = np.zeros((3,) + q.shape[1:])
    for a in range(3):
        dQa = d(a, np.moveaxis(Qm, (-2, -1), (0, 1)))  # (3, 3, z, y, x)
        want[a] = -np.einsum("cd...,...cd->...", dQa, H)
        for b in range(3):
            want[a] += d(b, comm[..., a, b])
    # in the field's own units the force is F / h, h = 1/scale: a second-order
    # gap shrinks 4x per halving of h
    return np.abs(F - want).max() * scale


def test_gibbs_duhem_identity_to_second_order():
    g1, g2, g3 = _gibbs_duhem_gap(16), _gibbs_duhem_gap(32), _gibbs_duhem_gap(64)
    assert g1 > 0 and g2 < g1 / 3 and g3 < g2 / 3.5, (g1, g2, g3)


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_stress_and_corotation_are_onsager_partners(seed):
    prm = oracle.lc_param_vector(A0=A0, gamma=GAMMA_NEM, kappa=KAPPA, xi=0.7)
    rng = np.random.default_rng(seed)
    A = 0.3 * rng.standard_normal((3, 3))
    Qm = A + A.T
    Qm -= np.trace(Qm) / 3 * np.eye(3)
    h, sigma = oracle.lc_field(uniform(Qm, (3, 3, 3)), prm)
    H = full(h)[0, 0, 0]
    Sg = sigma[:, 0, 0, 0].reshape(3, 3)
    W = rng.standard_normal((3, 3))
    W -= np.trace(W) / 3 * np.eye(3)
    S = oracle.lc_corotation(W, Qm, prm)
    lhs, rhs = np.sum(Sg * W), -np.sum(H * S)
    assert abs(lhs - rhs) <= 1e-15 * max(1.0, abs(lhs)), (lhs, rhs)
    assert abs(lhs) > 1e-6  # not trivially zero
