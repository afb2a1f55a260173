// FP64 CPU oracle for the liquid-crystal timestep: a Landau-de Gennes
// Q-tensor evolved by the Beris-Edwards equation with finite differences,
// coupled to D3Q19 lattice-Boltzmann flow through the divergence of its
// chemical stress.
//
// TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or call
// this file: only the tests and the smoke check (__graft_entry__.smoke) do.
// It shares no code, header, table or helper with the CUDA library.
//
// What it computes. The paper's Ludwig test case is a liquid crystal: a
// symmetric traceless 3x3 order-parameter tensor Q advected and relaxed by
// the Beris-Edwards model with the Landau-de Gennes free energy (Beris &
// Edwards 1994; de Gennes & Prost 1995), whose chemical stress drives the
// lattice-Boltzmann fluid; the timestep's kernels are "Order Parameter
// Gradients", "Chemical stress", "Collision", "Propagation", "LC Update" and
// "Advection" (Sec. 2.1.1). The paper prints none of the equations; the
// forms here are the standard ones of that model, one elastic constant:
//   free energy   f = A0/2 (1 - gamma/3) Q_ab Q_ab - A0 gamma/3 Q_ab Q_bc Q_ca
//                     + A0 gamma/4 (Q_ab Q_ab)^2 + kappa/2 (d_c Q_ab)^2
//   molecular field H_ab = -A0 (1 - gamma/3) Q_ab + A0 gamma (Q_ac Q_cb - delta_ab Q_cd Q_cd / 3)
//                     - A0 gamma (Q_cd Q_cd) Q_ab + kappa lap(Q_ab)
//   Beris-Edwards  dQ/dt + u.grad(Q) = S(W, Q) + Gamma H,  W_ab = d_b u_a,
//     S = (xi D + Om)(Q + I/3) + (Q + I/3)(xi D - Om) - 2 xi (Q + I/3) tr(Q W),
//     D = (W + W^T)/2, Om = (W - W^T)/2
//   stress (added to the fluid's own ideal-gas pressure)
//     sigma_ab = f delta_ab - kappa d_a Q_cd d_b Q_cd - xi H_ac (Q_cb + delta_cb/3)
//                - xi (Q_ac + delta_ac/3) H_cb + 2 xi (Q_ab + delta_ab/3) Q_cd H_cd
//                + Q_ac H_cb - H_ac Q_cb
//   force on the fluid F_a = d_b sigma_ab; BGK collision of f with the Guo
//   forcing and u = (j + F/2)/rho, then propagation, as in the binary fluid.
// Discretisation (the readings): d_c is the 2-point central difference,
// lap the 7-point Laplacian, the divergence of sigma central differences of
// the per-site sigma, W central differences of the per-site u; advection is
// first-order upwind on the sign of each velocity component at the site;
// dt = 1. One step, all fields of the same time level t:
//   rho, j from f(t); H(t), sigma(t) from Q(t); F(t) = div sigma(t);
//   u(t) = (j + F/2)/rho; f(t+1) = propagate(collide(f(t), u, F));
//   Q(t+1) = Q(t) + Gamma H(t) + S(W(t), Q(t)) - u(t).grad(Q(t)).
// Q is held as its five independent components (xx, xy, xz, yy, yz; zz =
// -xx - yy), so the update keeps it symmetric and traceless; the trace of S
// (2 xi div(u)/3, from the lattice fluid's slight compressibility) is dropped.
//
// Layout: site s = x + nx*(y + ny*z) (x fastest); component k of site s at
// [k*N + s]: f has 19 components, Q and H 5, u 3, sigma 9 (row-major ab).

#include <cmath>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

const int kQ = 19;
const int kCx[kQ] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
const int kCy[kQ] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
const int kCz[kQ] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
double weight(int i) { return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }

struct LcParams {
    double A0, gamma, kappa, Gamma, xi, tau_f, rho0;
};
LcParams params_of(const double* p) { return LcParams{p[0], p[1], p[2], p[3], p[4], p[5], p[6]}; }

struct Lattice {
    int nx, ny, nz;
    long n;
    long site(int x, int y, int z) const {
        x = (x % nx + nx) % nx;
        y = (y % ny + ny) % ny;
        z = (z % nz + nz) % nz;
        return x + (long)nx * (y + (long)ny * z);
    }
    void coords(long s, int& x, int& y, int& z) const {
        x = (int)(s % nx);
        y = (int)((s / nx) % ny);
        z = (int)(s / ((long)nx * ny));
    }
};

typedef double Mat[3][3];

// The full tensor from the five stored components of site s.
void full_q(const double* q, long n, long s, Mat Q) {
    const double xx = q[0 * n + s], xy = q[1 * n + s], xz = q[2 * n + s], yy = q[3 * n + s], yz = q[4 * n + s];
    Q[0][0] = xx; Q[0][1] = xy; Q[0][2] = xz;
    Q[1][0] = xy; Q[1][1] = yy; Q[1][2] = yz;
    Q[2][0] = xz; Q[2][1] = yz; Q[2][2] = -xx - yy;
}

const int kCompA[5] = {0, 0, 0, 1, 1};
const int kCompB[5] = {0, 1, 2, 1, 2};

// Gradient dQ[c] (central difference along axis c) and 7-point Laplacian of
// the full tensor at site (x, y, z).
void q_derivatives(const Lattice& L, const double* q, int x, int y, int z, Mat dQ[3], Mat lapQ) {
    Mat Qc, Qp, Qm;
    full_q(q, L.n, L.site(x, y, z), Qc);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) lapQ[a][b] = -6.0 * Qc[a][b];
    const int e[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int c = 0; c < 3; ++c) {
        full_q(q, L.n, L.site(x + e[c][0], y + e[c][1], z + e[c][2]), Qp);
        full_q(q, L.n, L.site(x - e[c][0], y - e[c][1], z - e[c][2]), Qm);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                dQ[c][a][b] = 0.5 * (Qp[a][b] - Qm[a][b]);
                lapQ[a][b] += Qp[a][b] + Qm[a][b];
            }
    }
}

// Molecular field H (full tensor) from Q and its Laplacian.
void molecular_field(const LcParams& p, const Mat Q, const Mat lapQ, Mat H) {
    double tr2 = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) tr2 += Q[a][b] * Q[a][b];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double qq = 0.0;
            for (int c = 0; c < 3; ++c) qq += Q[a][c] * Q[c][b];
            const double delta = a == b ? 1.0 : 0.0;
            H[a][b] = -p.A0 * (1.0 - p.gamma / 3.0) * Q[a][b] + p.A0 * p.gamma * (qq - delta * tr2 / 3.0) -
                      p.A0 * p.gamma * tr2 * Q[a][b] + p.kappa * lapQ[a][b];
        }
}

// Free energy density (bulk + one-constant gradient) at a site.
double free_energy(const LcParams& p, const Mat Q, const Mat dQ[3]) {
    double tr2 = 0.0, tr3 = 0.0, grad2 = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            tr2 += Q[a][b] * Q[a][b];
            for (int c = 0; c < 3; ++c) tr3 += Q[a][b] * Q[b][c] * Q[c][a];
        }
    for (int c = 0; c < 3; ++c)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) grad2 += dQ[c][a][b] * dQ[c][a][b];
    return 0.5 * p.A0 * (1.0 - p.gamma / 3.0) * tr2 - p.A0 * p.gamma / 3.0 * tr3 + 0.25 * p.A0 * p.gamma * tr2 * tr2 +
           0.5 * p.kappa * grad2;
}

// Chemical stress sigma (full tensor) at a site.
void chemical_stress(const LcParams& p, const Mat Q, const Mat dQ[3], const Mat H, Mat sigma) {
    const double fe = free_energy(p, Q, dQ);
    double qh = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) qh += Q[a][b] * H[a][b];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const double dab = a == b ? 1.0 : 0.0;
            double s = fe * dab;
            double grad = 0.0;
            for (int c = 0; c < 3; ++c)
                for (int d = 0; d < 3; ++d) grad += dQ[a][c][d] * dQ[b][c][d];
            s -= p.kappa * grad;
            for (int c = 0; c < 3; ++c) {
                const double dcb = c == b ? 1.0 : 0.0, dac = a == c ? 1.0 : 0.0;
                s -= p.xi * H[a][c] * (Q[c][b] + dcb / 3.0);
                s -= p.xi * (Q[a][c] + dac / 3.0) * H[c][b];
                s += Q[a][c] * H[c][b] - H[a][c] * Q[c][b];
            }
            s += 2.0 * p.xi * (Q[a][b] + dab / 3.0) * qh;
            sigma[a][b] = s;
        }
}

// H (5 components) and sigma (9) of every site.
void field_and_stress(const Lattice& L, const LcParams& p, const double* q, double* h, double* sigma) {
#pragma omp parallel for schedule(static)
    for (long s = 0; s < L.n; ++s) {
        int x, y, z;
        L.coords(s, x, y, z);
        Mat Q, dQ[3], lapQ, H, sg;
        full_q(q, L.n, s, Q);
        q_derivatives(L, q, x, y, z, dQ, lapQ);
        molecular_field(p, Q, lapQ, H);
        chemical_stress(p, Q, dQ, H, sg);
        for (int k = 0; k < 5; ++k) h[k * L.n + s] = H[kCompA[k]][kCompB[k]];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) sigma[(3 * a + b) * L.n + s] = sg[a][b];
    }
}

// Force F_a = sum_b D_b sigma_ab (central differences), the Guo velocity
// u = (j + F/2)/rho, and rho, from f and sigma.
void force_and_velocity(const Lattice& L, const double* f, const double* sigma, double* rho, double* u,
                        double* F) {
#pragma omp parallel for schedule(static)
    for (long s = 0; s < L.n; ++s) {
        int x, y, z;
        L.coords(s, x, y, z);
        double Fa[3] = {0.0, 0.0, 0.0};
        const int e[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
        for (int b = 0; b < 3; ++b) {
            const long sp = L.site(x + e[b][0], y + e[b][1], z + e[b][2]);
            const long sm = L.site(x - e[b][0], y - e[b][1], z - e[b][2]);
            for (int a = 0; a < 3; ++a)
                Fa[a] += 0.5 * (sigma[(3 * a + b) * L.n + sp] - sigma[(3 * a + b) * L.n + sm]);
        }
        double r = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < kQ; ++i) {
            const double fi = f[i * L.n + s];
            r += fi;
            j[0] += kCx[i] * fi;
            j[1] += kCy[i] * fi;
            j[2] += kCz[i] * fi;
        }
        rho[s] = r;
        for (int a = 0; a < 3; ++a) {
            u[a * L.n + s] = (j[a] + 0.5 * Fa[a]) / r;
            F[a * L.n + s] = Fa[a];
        }
    }
}

// BGK + Guo collision of f at every site, then propagation (push).
void collide_propagate(const Lattice& L, const LcParams& p, const double* f, const double* rho, const double* u,
                       const double* F, double* out) {
    const double omega = 1.0 / p.tau_f, pre = 1.0 - 0.5 / p.tau_f;
#pragma omp parallel for schedule(static)
    for (long s = 0; s < L.n; ++s) {
        int x, y, z;
        L.coords(s, x, y, z);
        const double ux = u[s], uy = u[L.n + s], uz = u[2 * L.n + s];
        const double Fx = F[s], Fy = F[L.n + s], Fz = F[2 * L.n + s];
        const double uu = ux * ux + uy * uy + uz * uz, uF = ux * Fx + uy * Fy + uz * Fz;
        for (int i = 0; i < kQ; ++i) {
            const double cu = kCx[i] * ux + kCy[i] * uy + kCz[i] * uz;
            const double cF = kCx[i] * Fx + kCy[i] * Fy + kCz[i] * Fz;
            const double feq = weight(i) * rho[s] * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
            const double src = pre * weight(i) * (3.0 * (cF - uF) + 9.0 * cu * cF);
            const double fi = f[i * L.n + s];
            out[i * L.n + L.site(x + kCx[i], y + kCy[i], z + kCz[i])] = fi - omega * (fi - feq) + src;
        }
    }
}

// S(W, Q) (full tensor) for the velocity gradient W_ab = d_b u_a.
void co_rotation(const LcParams& p, const Mat W, const Mat Q, Mat S) {
    Mat D, Om, Qp;
    double trQW = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            D[a][b] = 0.5 * (W[a][b] + W[b][a]);
            Om[a][b] = 0.5 * (W[a][b] - W[b][a]);
            Qp[a][b] = Q[a][b] + (a == b ? 1.0 / 3.0 : 0.0);
            trQW += Q[a][b] * W[b][a];
        }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int c = 0; c < 3; ++c)
                s += (p.xi * D[a][c] + Om[a][c]) * Qp[c][b] + Qp[a][c] * (p.xi * D[c][b] - Om[c][b]);
            S[a][b] = s - 2.0 * p.xi * Qp[a][b] * trQW;
        }
}

// Q(t+1) = Q + Gamma H + S(W, Q) - u.grad(Q) (first-order upwind), dt = 1.
void q_update(const Lattice& L, const LcParams& p, const double* q, const double* u, const double* h, double* qn) {
#pragma omp parallel for schedule(static)
    for (long s = 0; s < L.n; ++s) {
        int x, y, z;
        L.coords(s, x, y, z);
        const int e[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
        Mat W, Q, S;
        double us[3];
        for (int a = 0; a < 3; ++a) us[a] = u[a * L.n + s];
        for (int b = 0; b < 3; ++b) {
            const long sp = L.site(x + e[b][0], y + e[b][1], z + e[b][2]);
            const long sm = L.site(x - e[b][0], y - e[b][1], z - e[b][2]);
            for (int a = 0; a < 3; ++a) W[a][b] = 0.5 * (u[a * L.n + sp] - u[a * L.n + sm]);
        }
        full_q(q, L.n, s, Q);
        co_rotation(p, W, Q, S);
        for (int k = 0; k < 5; ++k) {
            const int a = kCompA[k], b = kCompB[k];
            const double qc = q[k * L.n + s];
            double adv = 0.0;
            for (int c = 0; c < 3; ++c) {
                const long up = us[c] >= 0.0 ? L.site(x - e[c][0], y - e[c][1], z - e[c][2])
                                              : L.site(x + e[c][0], y + e[c][1], z + e[c][2]);
                const double diff = us[c] >= 0.0 ? qc - q[k * L.n + up] : q[k * L.n + up] - qc;
                adv += us[c] * diff;
            }
            qn[k * L.n + s] = qc + p.Gamma * h[k * L.n + s] + S[a][b] - adv;
        }
    }
}

}  // namespace

extern "C" {

// H (5 components) and sigma (9, row-major) of the Q field.
int orc_lc_field(int nx, int ny, int nz, const double* prm, const double* q, double* h, double* sigma) {
    if (nx < 3 || ny < 3 || nz < 3) return -1;
    Lattice L{nx, ny, nz, (long)nx * ny * nz};
    field_and_stress(L, params_of(prm), q, h, sigma);
    return 0;
}

// S(W, Q) at one site: W and Q full 3x3 (row-major), S out.
void orc_lc_corotation(const double* prm, const double* W, const double* Q, double* S) {
    Mat w, qq, s;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            w[a][b] = W[3 * a + b];
            qq[a][b] = Q[3 * a + b];
        }
    co_rotation(params_of(prm), w, qq, s);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) S[3 * a + b] = s[a][b];
}

// One Q update with a given velocity field u (3 components) and H (5).
int orc_lc_update(int nx, int ny, int nz, const double* prm, const double* q, const double* u, const double* h,
                  double* qn) {
    if (nx < 3 || ny < 3 || nz < 3) return -1;
    Lattice L{nx, ny, nz, (long)nx * ny * nz};
    q_update(L, params_of(prm), q, u, h, qn);
    return 0;
}

// rho, u = (j + F/2)/rho and F = div sigma of the state (f, Q).
int orc_lc_macros(int nx, int ny, int nz, const double* prm, const double* f, const double* q, double* rho,
                  double* u, double* F) {
    if (nx < 3 || ny < 3 || nz < 3) return -1;
    Lattice L{nx, ny, nz, (long)nx * ny * nz};
    std::vector<double> h(5 * L.n), sigma(9 * L.n);
    field_and_stress(L, params_of(prm), q, h.data(), sigma.data());
    force_and_velocity(L, f, sigma.data(), rho, u, F);
    return 0;
}

// f = feq(rho, u) with rho = rho0 (or the given field) and u = 0 (or given).
int orc_lc_init(int nx, int ny, int nz, const double* prm, const double* rho, const double* u, double* f) {
    if (nx < 3 || ny < 3 || nz < 3) return -1;
    const LcParams p = params_of(prm);
    const long n = (long)nx * ny * nz;
    for (long s = 0; s < n; ++s) {
        const double r = rho ? rho[s] : p.rho0;
        const double ux = u ? u[s] : 0.0, uy = u ? u[n + s] : 0.0, uz = u ? u[2 * n + s] : 0.0;
        const double uu = ux * ux + uy * uy + uz * uz;
        for (int i = 0; i < kQ; ++i) {
            const double cu = kCx[i] * ux + kCy[i] * uy + kCz[i] * uz;
            f[i * n + s] = weight(i) * r * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
        }
    }
    return 0;
}

// nsteps coupled steps of (f, Q), in place.
int orc_lc_step(int nx, int ny, int nz, const double* prm, double* f, double* q, int nsteps) {
    if (nx < 3 || ny < 3 || nz < 3 || nsteps < 0) return -1;
    Lattice L{nx, ny, nz, (long)nx * ny * nz};
    const LcParams p = params_of(prm);
    std::vector<double> h(5 * L.n), sigma(9 * L.n), rho(L.n), u(3 * L.n), F(3 * L.n), fn(kQ * L.n), qn(5 * L.n);
    for (int t = 0; t < nsteps; ++t) {
        field_and_stress(L, p, q, h.data(), sigma.data());
        force_and_velocity(L, f, sigma.data(), rho.data(), u.data(), F.data());
        collide_propagate(L, p, f, rho.data(), u.data(), F.data(), fn.data());
        q_update(L, p, q, u.data(), h.data(), qn.data());
        std::memcpy(f, fn.data(), sizeof(double) * kQ * L.n);
        std::memcpy(q, qn.data(), sizeof(double) * 5 * L.n);
    }
    return 0;
}

}  // extern "C"
