"""Brute-force pin of the FP64 oracle on tiny lattices: the same timestep
evaluated site by site in 40-digit arithmetic (mpmath), written as a pull
(gather) update with explicit modular neighbour indices rather than the
oracle's push over whole planes, and compared with the oracle after three
steps. The velocity set and weights come from the golden lattice file.

This catches implementation slips in the oracle's C++ that an invariant can
miss: a wrong neighbour index or periodic wrap, a direction paired with the
wrong weight, a term dropped in one direction only, an option (19-point
stencils, the stress force, the two-relaxation-time collision) wired to the
wrong branch. It does not replace the physical pins, which check the
formulas themselves (a misreading shared by both transcriptions passes
here).

The step, per site x (Sec. 2.1.1's components in their binary-fluid form):
  rho = sum f_i, j = sum f_i c_i, phi = sum g_i;
  mu = A phi + B phi^3 - kappa lap(phi);  F = -phi grad(mu)  or  F = -div P;
  u = (j + F/2)/rho;
  f*_i, g*_i by the BGK (or TRT) collision with Guo forcing;
  f_i(x, t+1) = f*_i(x - c_i, t).
"""

import os

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")
oracle = pytest.importorskip("oracle")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
mp = mpmath.mp


def _lattice():
    c, w = [], []
    with open(os.path.join(GOLDEN, "d3q19_lattice.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                parts = line.split()
                c.append(tuple(int(v) for v in parts[1:4]))
                num, den = parts[4].split("/")
                w.append(mpmath.mpf(int(num)) / int(den))
    return c, w


class Brute:
    """One lattice in 40-digit arithmetic; fields are dicts keyed by (x, y, z)."""

    def __init__(self, shape, prm):
        self.nx, self.ny, self.nz = shape
        self.c, self.w = _lattice()
        self.opp = [self.c.index((-a, -b, -d)) for (a, b, d) in self.c]
        self.sites = [(x, y, z) for z in range(self.nz) for y in range(self.ny) for x in range(self.nx)]
        names = ("A", "B", "kappa", "Gamma", "tau_f", "tau_g", "rho0")
        self.p = {k: mpmath.mpf(float(prm[i])) for i, k in enumerate(names)}
        self.stencil = int(prm[7])
        self.stress = int(prm[8]) == 1
        self.trt = int(prm[9]) == 1
        self.magic = mpmath.mpf(float(prm[10]))

    def at(self, x, y, z, d):
        return ((x + d[0]) % self.nx, (y + d[1]) % self.ny, (z + d[2]) % self.nz)

    # Finite differences on the D3Q19 neighbourhood.
    def lap(self, h, s):
        if self.stencil == 1:  # sum_i 6 w_i (h(x + c_i) - h(x))
            return sum(6 * self.w[i] * (h[self.at(*s, self.c[i])] - h[s]) for i in range(1, 19))
        axes = ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1))
        return sum(h[self.at(*s, e)] for e in axes) - 6 * h[s]

    def grad(self, h, s):
        if self.stencil == 1:  # sum_i 3 w_i c_i h(x + c_i)
            out = [mpmath.mpf(0)] * 3
            for i in range(1, 19):
                v = 3 * self.w[i] * h[self.at(*s, self.c[i])]
                out = [out[a] + self.c[i][a] * v for a in range(3)]
            return out
        out = []
        for a in range(3):
            e = [0, 0, 0]
            e[a] = 1
            em = [-v for v in e]
            out.append((h[self.at(*s, e)] - h[self.at(*s, em)]) / 2)
        return out

    def mu_field(self, phi):
        p = self.p
        return {s: p["A"] * phi[s] + p["B"] * phi[s] ** 3 - p["kappa"] * self.lap(phi, s) for s in self.sites}

    def feq(self, rho, u):
        uu = sum(v * v for v in u)
        out = []
        for i in range(19):
            cu = sum(self.c[i][a] * u[a] for a in range(3))
            out.append(self.w[i] * rho * (1 + 3 * cu + mpmath.mpf(9) / 2 * cu * cu - mpmath.mpf(3) / 2 * uu))
        return out

    def geq(self, phi, u, mu):
        uu = sum(v * v for v in u)
        dev = self.p["Gamma"] * mu - phi / 3
        out = []
        for i in range(19):
            cu = sum(self.c[i][a] * u[a] for a in range(3))
            c2 = sum(v * v for v in self.c[i])
            out.append(self.w[i] * (phi + 3 * phi * cu + mpmath.mpf(9) / 2 * dev * (c2 - 1)
                                    + mpmath.mpf(9) / 2 * phi * cu * cu - mpmath.mpf(3) / 2 * phi * uu))
        return out

    def guo_bare(self, u, F):
        out = []
        for i in range(19):
            ci = self.c[i]
            cu = sum(ci[a] * u[a] for a in range(3))
            out.append(self.w[i] * sum((3 * (ci[a] - u[a]) + 9 * cu * ci[a]) * F[a] for a in range(3)))
        return out

    def init(self, phi, rho, u):
        mu = self.mu_field(phi)
        f = {s: self.feq(rho[s], u[s]) for s in self.sites}
        g = {s: self.geq(phi[s], u[s], mu[s]) for s in self.sites}
        return f, g

    def force(self, phi, mu):
        if not self.stress:
            return {s: [-phi[s] * v for v in self.grad(mu, s)] for s in self.sites}
        p = self.p
        # P_ab = [A phi^2/2 + 3B phi^4/4 - kappa phi lap - kappa/2 |grad phi|^2] delta_ab + kappa d_a phi d_b phi
        P = {}
        for s in self.sites:
            gp = self.grad(phi, s)
            iso = (p["A"] / 2 * phi[s] ** 2 + 3 * p["B"] / 4 * phi[s] ** 4 - p["kappa"] * phi[s] * self.lap(phi, s)
                   - p["kappa"] / 2 * sum(v * v for v in gp))
            P[s] = [[(iso if a == b else 0) + p["kappa"] * gp[a] * gp[b] for b in range(3)] for a in range(3)]
        F = {}
        for s in self.sites:
            F[s] = [-sum(self.grad({t: P[t][a][b] for t in self.sites}, s)[b] for b in range(3)) for a in range(3)]
        return F

    def step(self, f, g):
        p = self.p
        rho = {s: sum(f[s]) for s in self.sites}
        j = {s: [sum(self.c[i][a] * f[s][i] for i in range(19)) for a in range(3)] for s in self.sites}
        phi = {s: sum(g[s]) for s in self.sites}
        mu = self.mu_field(phi)
        F = self.force(phi, mu)
        fs, gs = {}, {}
        for s in self.sites:
            u = [(j[s][a] + F[s][a] / 2) / rho[s] for a in range(3)]
            feq = self.feq(rho[s], u)
            bare = self.guo_bare(u, F[s])
            if self.trt:
                tau_m = mpmath.mpf(1) / 2 + self.magic / (p["tau_f"] - mpmath.mpf(1) / 2)
                pre_p, pre_m = 1 - 1 / (2 * p["tau_f"]), 1 - 1 / (2 * tau_m)
                out = []
                for i in range(19):
                    o = self.opp[i]
                    even = (f[s][i] + f[s][o] - feq[i] - feq[o]) / 2
                    odd = (f[s][i] - f[s][o] - feq[i] + feq[o]) / 2
                    out.append(f[s][i] - even / p["tau_f"] - odd / tau_m
                               + pre_p * (bare[i] + bare[o]) / 2 + pre_m * (bare[i] - bare[o]) / 2)
                fs[s] = out
            else:
                pre = 1 - 1 / (2 * p["tau_f"])
                fs[s] = [f[s][i] - (f[s][i] - feq[i]) / p["tau_f"] + pre * bare[i] for i in range(19)]
            geq = self.geq(phi[s], u, mu[s])
            gs[s] = [g[s][i] - (g[s][i] - geq[i]) / p["tau_g"] for i in range(19)]
        # pull: f_i(x) <- f*_i(x - c_i)
        fn, gn = {}, {}
        for s in self.sites:
            fn[s] = [fs[self.at(*s, [-v for v in self.c[i]])][i] for i in range(19)]
            gn[s] = [gs[self.at(*s, [-v for v in self.c[i]])][i] for i in range(19)]
        return fn, gn

    def to_array(self, d):
        out = np.zeros((19, self.nz, self.ny, self.nx))
        for (x, y, z), v in d.items():
            out[:, z, y, x] = [float(e) for e in v]
        return out


CASES = {
    "bgk-7": ((4, 4, 4), dict()),
    "bgk-19": ((5, 6, 7), dict(stencil=19)),
    "stress-7": ((5, 4, 6), dict(force="stress")),
    "stress-19": ((4, 5, 4), dict(force="stress", stencil=19)),
    "trt-7": ((6, 5, 4), dict(collision="trt", magic=0.25)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_oracle_matches_40_digit_brute_force(case):
    """Three steps from a non-trivial start (rho, u and phi all varying,
    tau_f and tau_g away from 1 so that the relaxation terms are live): the
    oracle's f and g agree with the 40-digit evaluation to within 36 FP64
    ulps (4e-15) of the largest value."""
    (nx, ny, nz), opts = CASES[case]
    prm = oracle.param_vector(tau_f=0.8, tau_g=1.3, kappa=0.04, **opts)
    rng = np.random.default_rng(7)
    phi = 0.8 * (2 * rng.random((nz, ny, nx)) - 1)
    rho = 1.0 + 0.05 * (2 * rng.random((nz, ny, nx)) - 1)
    u = 0.03 * (2 * rng.random((3, nz, ny, nx)) - 1)

    mp.dps = 40
    b = Brute((nx, ny, nz), prm)
    key = lambda s: (s[2], s[1], s[0])  # noqa: E731  (z, y, x) index of site (x, y, z)
    fb, gb = b.init({s: mpmath.mpf(float(phi[key(s)])) for s in b.sites},
                    {s: mpmath.mpf(float(rho[key(s)])) for s in b.sites},
                    {s: [mpmath.mpf(float(u[a][key(s)])) for a in range(3)] for s in b.sites})
    f0, g0 = oracle.init(phi, prm, rho=rho, u=u)
    # the initial state itself
    np.testing.assert_allclose(f0, b.to_array(fb), rtol=0, atol=4e-16 * np.abs(f0).max())
    np.testing.assert_allclose(g0, b.to_array(gb), rtol=0, atol=4e-16 * np.abs(g0).max())

    for _ in range(3):
        fb, gb = b.step(fb, gb)
    f3, g3 = oracle.step(f0, g0, prm, nsteps=3)
    fe, ge = b.to_array(fb), b.to_array(gb)
    err_f = np.abs(f3 - fe).max() / np.abs(fe).max()
    err_g = np.abs(g3 - ge).max() / np.abs(ge).max()
    # measured about 1e-15 (5-10 ulps of the largest value) in every case
    assert err_f < 4e-15 and err_g < 4e-15, (err_f, err_g)
    # and the state moved: the comparison is not between two copies of the start
    assert np.abs(fe - b.to_array(b.init(*[{s: mpmath.mpf(float(a[key(s)])) for s in b.sites}
                                           for a in (phi, rho)],
                                         {s: [mpmath.mpf(float(u[a][key(s)])) for a in range(3)]
                                          for s in b.sites})[0])).max() > 1e-4


def test_brute_force_is_sensitive_to_a_planted_slip():
    """The comparison has teeth: a copy of the brute force with the weight of
    one diagonal pair swapped against an axis weight disagrees with the
    oracle far beyond the tolerance."""
    prm = oracle.param_vector(tau_f=0.8, tau_g=1.3)
    rng = np.random.default_rng(8)
    nx = ny = nz = 4
    phi = 0.8 * (2 * rng.random((nz, ny, nx)) - 1)
    mp.dps = 40
    b = Brute((nx, ny, nz), prm)
    b.w[7], b.w[1] = b.w[1], b.w[7]
    key = lambda s: (s[2], s[1], s[0])  # noqa: E731
    one = {s: mpmath.mpf(1) for s in b.sites}
    zero = {s: [mpmath.mpf(0)] * 3 for s in b.sites}
    fb, gb = b.init({s: mpmath.mpf(float(phi[key(s)])) for s in b.sites}, one, zero)
    fb, gb = b.step(fb, gb)
    f0, g0 = oracle.init(phi, prm)
    f1, g1 = oracle.step(f0, g0, prm, nsteps=1)
    assert np.abs(g1 - b.to_array(gb)).max() / np.abs(g1).max() > 1e-6
