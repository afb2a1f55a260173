// FP64 CPU oracle for the binary-fluid D3Q19 lattice-Boltzmann timestep.
//
// TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or call
// this file: only the tests, the smoke check and the CPU-baseline leg of the
// benchmark do. It shares no code, header, table or helper with the CUDA
// library; the two are independent statements of the same method.
//
// What it computes. The paper (Gray & Stratford, "A Lightweight Approach to
// Performance Portability with targetDP", Sec. 2.1.1) names the kernels of one
// Ludwig timestep -- "Collision", "Propagation", "Chemical stress" and
// "Order Parameter Gradients" -- but prints none of their equations. The
// binary-fluid instance computed here is the standard one those names stand
// for:
//   * the D3Q19 velocity set and weights (Qian, d'Humieres & Lallemand 1992);
//   * BGK collision of f with the Guo-Zheng-Shi (2002) forcing term and the
//     half-force velocity u = (j + F/2)/rho; optionally (collision = 1) the
//     two-relaxation-time form: the even and odd parts of each opposite pair,
//     f+- = (f_i +- f_-i)/2 (and likewise feq and the Guo source), relax with
//     omega+ = 1/tau_f and omega- = 1/tau-, tau- = 1/2 + Lambda/(tau_f - 1/2),
//     the source parts scaled by (1 - omega+/2) and (1 - omega-/2);
//   * BGK collision of g towards an equilibrium whose zeroth, first and second
//     moments are phi, phi*u and Gamma*mu*I + phi*u*u;
//   * the symmetric phi^4 free energy: mu = A phi + B phi^3 - kappa lap(phi),
//     force F = -phi * grad(mu), with one of two stencil pairs: the 7-point
//     Laplacian and the 2-point central difference (the default), or the
//     19-point isotropic forms on the D3Q19 neighbourhood,
//       lap h = sum_i 6 w_i (h(x + c_i) - h(x)),
//       grad h = sum_i 3 w_i c_i h(x + c_i),
//     whose leading truncation errors are isotropic (sum_i w_i c c c c is);
//   * optionally (force = 1) the force as the divergence of the chemical
//     stress of the same free energy, F = -div P with
//       P_ab = [p_b - kappa phi lap(phi) - kappa/2 |grad phi|^2] delta_ab
//              + kappa d_a phi d_b phi,   p_b = A phi^2/2 + 3 B phi^4/4,
//     equal to -phi grad(mu) in the continuum and conserving total momentum
//     exactly on the lattice (a discrete divergence telescopes);
//   * propagation: f_i(x + c_i, t+1) = f*_i(x, t) on a periodic lattice.
// One step is: moments -> phi stencil and mu -> force and velocity ->
// collide f -> collide g -> propagate, all stencils on fields of the same
// time level. The state between steps is the post-propagation
// (pre-collision) pair f, g.
//
// Layout: site s = x + nx*(y + ny*z) (x fastest); distribution component i of
// site s at [i*N + s]; vector fields (u, grad phi, F) as [a*N + s].
// Arithmetic is plain double; the build passes -ffp-contract=off so that no
// fused multiply-add changes the rounding of what is written here.
//
// The whole scheme is templated on the scalar type: with T = double it is the
// oracle; with T = Dual (value + one directional derivative) the same source
// is the tangent-linear model used to check the adjoint.
//
// Every function carries a pin in tests/test_oracle_pins.py; none is
// "parity unpinned".

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------------------
// D3Q19 velocity set (Qian, d'Humieres & Lallemand 1992). Order: rest; the six
// axis vectors +x,-x,+y,-y,+z,-z; then the twelve face diagonals in pairs
// (v, -v). The opposite of an odd index i is i+1.
const int kQ = 19;
const int kCx[kQ] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
const int kCy[kQ] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
const int kCz[kQ] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

double weight(int i) {
    if (i == 0) return 1.0 / 3.0;
    if (i <= 6) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

// Index of -c_i (odd i pairs with i + 1).
int opposite(int i) { return i == 0 ? 0 : (i % 2 ? i + 1 : i - 1); }

// ---------------------------------------------------------------------------
// Dual number: value and one directional derivative (forward-mode AD).
struct Dual {
    double v, d;
    Dual() : v(0.0), d(0.0) {}
    Dual(double value) : v(value), d(0.0) {}
    Dual(double value, double deriv) : v(value), d(deriv) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
    return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual operator+(Dual a, double b) { return Dual(a.v + b, a.d); }
inline Dual operator+(double a, Dual b) { return Dual(a + b.v, b.d); }
inline Dual operator-(Dual a, double b) { return Dual(a.v - b, a.d); }
inline Dual operator-(double a, Dual b) { return Dual(a - b.v, -b.d); }
inline Dual operator*(Dual a, double b) { return Dual(a.v * b, a.d * b); }
inline Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
inline Dual operator/(Dual a, double b) { return Dual(a.v / b, a.d / b); }
inline Dual operator/(double a, Dual b) { return Dual(a / b.v, -a * b.d / (b.v * b.v)); }
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }

// ---------------------------------------------------------------------------
template <class T>
struct Params {
    T A, B, kappa, Gamma, tau_f, tau_g, rho0;
    int stencil;  // 0: 7-point / central difference; 1: 19-point isotropic
    int force;    // 0: F = -phi grad(mu); 1: F = -div P (chemical stress)
    int collision;  // 0: BGK; 1: two-relaxation-time with magic parameter lambda
    T lambda;       // (tau_f - 1/2)(tau- - 1/2), collision = 1 only
};

struct Lattice {
    int nx, ny, nz;
    long n;
    Lattice(int x, int y, int z) : nx(x), ny(y), nz(z), n((long)x * y * z) {}
    long site(int x, int y, int z) const { return x + (long)nx * (y + (long)ny * z); }
    // Site reached from (x,y,z) by the displacement (dx,dy,dz), periodic.
    long shifted(int x, int y, int z, int dx, int dy, int dz) const {
        int xs = ((x + dx) % nx + nx) % nx;
        int ys = ((y + dy) % ny + ny) % ny;
        int zs = ((z + dz) % nz + nz) % nz;
        return site(xs, ys, zs);
    }
};

// Equilibrium of f: w_i rho [1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u].
template <class T>
void feq_site(T rho, const T u[3], T out[kQ]) {
    T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < kQ; ++i) {
        T cu = kCx[i] * u[0] + kCy[i] * u[1] + kCz[i] * u[2];
        out[i] = weight(i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

// Equilibrium of g: second-order Hermite form with moments phi, phi u and
// Gamma mu I + phi u u:
//   w_i [phi + 3 phi c.u + 9/2 (Gamma mu - phi/3)(|c|^2 - 1)
//        + 9/2 phi (c.u)^2 - 3/2 phi u.u].
template <class T>
void geq_site(T phi, const T u[3], T mu, T Gamma, T out[kQ]) {
    T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    T pressure_dev = Gamma * mu - phi / 3.0;
    for (int i = 0; i < kQ; ++i) {
        T cu = kCx[i] * u[0] + kCy[i] * u[1] + kCz[i] * u[2];
        int c2 = kCx[i] * kCx[i] + kCy[i] * kCy[i] + kCz[i] * kCz[i];
        out[i] = weight(i) * (phi + 3.0 * phi * cu + 4.5 * pressure_dev * (double)(c2 - 1)
                              + 4.5 * phi * cu * cu - 1.5 * phi * uu);
    }
}

// The Guo source without its prefactor: w_i [3 (c_i - u) + 9 (c_i.u) c_i] . F.
template <class T>
void guo_bare_site(const T u[3], const T F[3], T out[kQ]) {
    for (int i = 0; i < kQ; ++i) {
        T cu = kCx[i] * u[0] + kCy[i] * u[1] + kCz[i] * u[2];
        T ex = 3.0 * (kCx[i] - u[0]) + 9.0 * cu * kCx[i];
        T ey = 3.0 * (kCy[i] - u[1]) + 9.0 * cu * kCy[i];
        T ez = 3.0 * (kCz[i] - u[2]) + 9.0 * cu * kCz[i];
        out[i] = weight(i) * (ex * F[0] + ey * F[1] + ez * F[2]);
    }
}

// Guo-Zheng-Shi (2002) source term, including its (1 - 1/(2 tau)) prefactor:
//   (1 - 1/(2 tau)) w_i [3 (c_i - u) + 9 (c_i.u) c_i] . F.
template <class T>
void guo_site(const T u[3], const T F[3], T tau, T out[kQ]) {
    T pre = 1.0 - 1.0 / (2.0 * tau);
    for (int i = 0; i < kQ; ++i) {
        T cu = kCx[i] * u[0] + kCy[i] * u[1] + kCz[i] * u[2];
        T ex = 3.0 * (kCx[i] - u[0]) + 9.0 * cu * kCx[i];
        T ey = 3.0 * (kCy[i] - u[1]) + 9.0 * cu * kCy[i];
        T ez = 3.0 * (kCz[i] - u[2]) + 9.0 * cu * kCz[i];
        out[i] = pre * weight(i) * (ex * F[0] + ey * F[1] + ez * F[2]);
    }
}

// Coefficients of the 19-point isotropic forms, 6 w_i and 3 w_i, written as
// the exact fractions they are: 1/3 and 1/6 (axis neighbours), 1/6 and 1/12
// (face diagonals).
double lap19_coef(int i) { return i <= 6 ? 1.0 / 3.0 : 1.0 / 6.0; }
double grad19_coef(int i) { return i <= 6 ? 1.0 / 6.0 : 1.0 / 12.0; }

// Laplacian, periodic: 7-point (sum of the six axis neighbours minus 6 h), or
// 19-point isotropic (sum over i = 1..18, in velocity order, of
// 6 w_i (h(x + c_i) - h(x))).
template <class T>
void laplacian(const Lattice& L, const T* phi, T* lap, int stencil = 0) {
#pragma omp parallel for schedule(static)
    for (int z = 0; z < L.nz; ++z)
        for (int y = 0; y < L.ny; ++y)
            for (int x = 0; x < L.nx; ++x) {
                long s = L.site(x, y, z);
                if (stencil == 0) {
                    T sum = phi[L.shifted(x, y, z, 1, 0, 0)] + phi[L.shifted(x, y, z, -1, 0, 0)]
                          + phi[L.shifted(x, y, z, 0, 1, 0)] + phi[L.shifted(x, y, z, 0, -1, 0)]
                          + phi[L.shifted(x, y, z, 0, 0, 1)] + phi[L.shifted(x, y, z, 0, 0, -1)];
                    lap[s] = sum - 6.0 * phi[s];
                } else {
                    T sum = 0.0;
                    for (int i = 1; i < kQ; ++i)
                        sum += lap19_coef(i) * (phi[L.shifted(x, y, z, kCx[i], kCy[i], kCz[i])] - phi[s]);
                    lap[s] = sum;
                }
            }
}

// Gradient, periodic: central difference (h(x+e_a) - h(x-e_a))/2, or the
// 19-point isotropic sum over i = 1..18 (velocity order, terms with c_ia = 0
// left out) of 3 w_i c_ia h(x + c_i).
template <class T>
void gradient(const Lattice& L, const T* h, T* grad, int stencil = 0) {
#pragma omp parallel for schedule(static)
    for (int z = 0; z < L.nz; ++z)
        for (int y = 0; y < L.ny; ++y)
            for (int x = 0; x < L.nx; ++x) {
                long s = L.site(x, y, z);
                if (stencil == 0) {
                    grad[0 * L.n + s] = (h[L.shifted(x, y, z, 1, 0, 0)] - h[L.shifted(x, y, z, -1, 0, 0)]) / 2.0;
                    grad[1 * L.n + s] = (h[L.shifted(x, y, z, 0, 1, 0)] - h[L.shifted(x, y, z, 0, -1, 0)]) / 2.0;
                    grad[2 * L.n + s] = (h[L.shifted(x, y, z, 0, 0, 1)] - h[L.shifted(x, y, z, 0, 0, -1)]) / 2.0;
                } else {
                    T g[3] = {T(0.0), T(0.0), T(0.0)};
                    for (int i = 1; i < kQ; ++i) {
                        const T hi = h[L.shifted(x, y, z, kCx[i], kCy[i], kCz[i])];
                        const int c[3] = {kCx[i], kCy[i], kCz[i]};
                        for (int a = 0; a < 3; ++a)
                            if (c[a] > 0)
                                g[a] += grad19_coef(i) * hi;
                            else if (c[a] < 0)
                                g[a] -= grad19_coef(i) * hi;
                    }
                    for (int a = 0; a < 3; ++a) grad[a * L.n + s] = g[a];
                }
            }
}

// mu = A phi + B phi^3 - kappa lap(phi).
template <class T>
void chemical_potential(const Lattice& L, const Params<T>& p, const T* phi, T* lap, T* mu) {
    laplacian(L, phi, lap, p.stencil);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < L.n; ++s)
        mu[s] = p.A * phi[s] + p.B * phi[s] * phi[s] * phi[s] - p.kappa * lap[s];
}

// Propagation: out_i(x + c_i) = in_i(x) for every component i (a permutation).
template <class T>
void propagate(const Lattice& L, const T* in, T* out) {
    for (int i = 0; i < kQ; ++i) {
#pragma omp parallel for schedule(static)
        for (int z = 0; z < L.nz; ++z)
            for (int y = 0; y < L.ny; ++y)
                for (int x = 0; x < L.nx; ++x)
                    out[i * L.n + L.shifted(x, y, z, kCx[i], kCy[i], kCz[i])] =
                        in[i * L.n + L.site(x, y, z)];
    }
}

// Transpose of propagate: out_i(x) = in_i(x + c_i).
template <class T>
void propagate_reverse(const Lattice& L, const T* in, T* out) {
    for (int i = 0; i < kQ; ++i) {
#pragma omp parallel for schedule(static)
        for (int z = 0; z < L.nz; ++z)
            for (int y = 0; y < L.ny; ++y)
                for (int x = 0; x < L.nx; ++x)
                    out[i * L.n + L.site(x, y, z)] =
                        in[i * L.n + L.shifted(x, y, z, kCx[i], kCy[i], kCz[i])];
    }
}

// Chemical stress of the phi^4 free energy at every site, six components
// [xx, yy, zz, xy, xz, yz] of P (layout [c*N + s]), from grad phi and
// lap(phi) with the selected stencils:
//   iso = A/2 phi^2 + 3B/4 phi^4 - kappa phi lap - kappa/2 |grad phi|^2,
//   P_aa = iso + kappa (d_a phi)^2,  P_ab = kappa d_a phi d_b phi.
template <class T>
void chemical_stress(const Lattice& L, const Params<T>& p, const T* phi, const T* lap, T* P) {
    const long n = L.n;
    std::vector<T> gr(3 * n);
    gradient(L, phi, gr.data(), p.stencil);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < n; ++s) {
        const T ph = phi[s], gx = gr[s], gy = gr[n + s], gz = gr[2 * n + s];
        const T pb = 0.5 * p.A * ph * ph + 0.75 * p.B * ph * ph * ph * ph;
        const T iso = pb - p.kappa * ph * lap[s] - 0.5 * p.kappa * (gx * gx + gy * gy + gz * gz);
        P[0 * n + s] = iso + p.kappa * gx * gx;
        P[1 * n + s] = iso + p.kappa * gy * gy;
        P[2 * n + s] = iso + p.kappa * gz * gz;
        P[3 * n + s] = p.kappa * gx * gy;
        P[4 * n + s] = p.kappa * gx * gz;
        P[5 * n + s] = p.kappa * gy * gz;
    }
}

// F_a = -sum_b D_b P_ab, D the selected gradient stencil, summed in the
// order b = x, y, z.
template <class T>
void stress_force(const Lattice& L, const Params<T>& p, const T* P, T* F) {
    const long n = L.n;
    // component of P for the pair (a, b)
    const int comp[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
    std::vector<T> d(3 * n);
    std::vector<T> acc(3 * n, T(0.0));
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            gradient(L, P + comp[a][b] * n, d.data(), p.stencil);
#pragma omp parallel for schedule(static)
            for (long s = 0; s < n; ++s) acc[a * n + s] = acc[a * n + s] + d[b * n + s];
        }
#pragma omp parallel for schedule(static)
    for (long k = 0; k < 3 * n; ++k) F[k] = -acc[k];
}

// Macroscopic fields of a pre-collision state, in the order the step uses
// them: rho, j, phi; lap(phi) and mu; the force (F = -phi grad(mu), or
// -div P); u = (j + F/2)/rho.
template <class T>
struct Macro {
    std::vector<T> rho, j, phi, lap, mu, gradmu, F, u;
    explicit Macro(long n)
        : rho(n), j(3 * n), phi(n), lap(n), mu(n), gradmu(3 * n), F(3 * n), u(3 * n) {}
};

template <class T>
void macroscopic(const Lattice& L, const Params<T>& p, const T* f, const T* g, Macro<T>& m) {
    const long n = L.n;
#pragma omp parallel for schedule(static)
    for (long s = 0; s < n; ++s) {
        T rho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0, phi = 0.0;
        for (int i = 0; i < kQ; ++i) {
            T fi = f[i * n + s];
            rho += fi;
            jx += kCx[i] * fi;
            jy += kCy[i] * fi;
            jz += kCz[i] * fi;
            phi += g[i * n + s];
        }
        m.rho[s] = rho;
        m.j[0 * n + s] = jx;
        m.j[1 * n + s] = jy;
        m.j[2 * n + s] = jz;
        m.phi[s] = phi;
    }
    chemical_potential(L, p, m.phi.data(), m.lap.data(), m.mu.data());
    gradient(L, m.mu.data(), m.gradmu.data(), p.stencil);
    if (p.force == 1) {
        std::vector<T> P(6 * n);
        chemical_stress(L, p, m.phi.data(), m.lap.data(), P.data());
        stress_force(L, p, P.data(), m.F.data());
    }
#pragma omp parallel for schedule(static)
    for (long s = 0; s < n; ++s)
        for (int a = 0; a < 3; ++a) {
            if (p.force == 0) m.F[a * n + s] = -m.phi[s] * m.gradmu[a * n + s];
            m.u[a * n + s] = (m.j[a * n + s] + m.F[a * n + s] / 2.0) / m.rho[s];
        }
}

// Collision of both distributions at every site (in place on f, g).
template <class T>
void collide(const Lattice& L, const Params<T>& p, const Macro<T>& m, T* f, T* g) {
    const long n = L.n;
#pragma omp parallel for schedule(static)
    for (long s = 0; s < n; ++s) {
        T u[3] = {m.u[s], m.u[n + s], m.u[2 * n + s]};
        T F[3] = {m.F[s], m.F[n + s], m.F[2 * n + s]};
        T feq[kQ], src[kQ], geq[kQ];
        feq_site(m.rho[s], u, feq);
        guo_site(u, F, p.tau_f, src);
        if (p.collision == 0) {
            for (int i = 0; i < kQ; ++i) {
                T fi = f[i * n + s];
                f[i * n + s] = fi - (fi - feq[i]) / p.tau_f + src[i];
            }
        } else {
            const T tau_m = 0.5 + p.lambda / (p.tau_f - 0.5);
            const T pre_p = 1.0 - 1.0 / (2.0 * p.tau_f), pre_m = 1.0 - 1.0 / (2.0 * tau_m);
            T bare[kQ], out[kQ];
            guo_bare_site(u, F, bare);
            for (int i = 0; i < kQ; ++i) {
                const int o = opposite(i);
                const T fi = f[i * n + s], fo = f[o * n + s];
                const T fp = 0.5 * (fi + fo), fm = 0.5 * (fi - fo);
                const T ep = 0.5 * (feq[i] + feq[o]), em = 0.5 * (feq[i] - feq[o]);
                const T sp = 0.5 * (bare[i] + bare[o]), sm = 0.5 * (bare[i] - bare[o]);
                out[i] = fi - (fp - ep) / p.tau_f - (fm - em) / tau_m + pre_p * sp + pre_m * sm;
            }
            for (int i = 0; i < kQ; ++i) f[i * n + s] = out[i];
        }
        geq_site(m.phi[s], u, m.mu[s], p.Gamma, geq);
        for (int i = 0; i < kQ; ++i) {
            T gi = g[i * n + s];
            g[i * n + s] = gi - (gi - geq[i]) / p.tau_g;
        }
    }
}

// One full timestep; tmp holds 19*N scalars.
template <class T>
void step(const Lattice& L, const Params<T>& p, T* f, T* g, T* tmp, Macro<T>& m) {
    macroscopic(L, p, f, g, m);
    collide(L, p, m, f, g);
    const size_t bytes = sizeof(T) * kQ * L.n;
    propagate(L, f, tmp);
    std::memcpy(f, tmp, bytes);
    propagate(L, g, tmp);
    std::memcpy(g, tmp, bytes);
}

// Initial state: f = feq(rho, u); g = geq(phi, u, mu(phi)), no force.
template <class T>
void init_state(const Lattice& L, const Params<T>& p, const T* phi, const T* rho_in,
                const T* u_in, T* f, T* g) {
    const long n = L.n;
    std::vector<T> lap(n), mu(n);
    chemical_potential(L, p, phi, lap.data(), mu.data());
#pragma omp parallel for schedule(static)
    for (long s = 0; s < n; ++s) {
        T rho = rho_in ? rho_in[s] : p.rho0;
        T u[3] = {T(0.0), T(0.0), T(0.0)};
        if (u_in) {
            u[0] = u_in[s];
            u[1] = u_in[n + s];
            u[2] = u_in[2 * n + s];
        }
        T fe[kQ], ge[kQ];
        feq_site(rho, u, fe);
        geq_site(phi[s], u, mu[s], p.Gamma, ge);
        for (int i = 0; i < kQ; ++i) {
            f[i * n + s] = fe[i];
            g[i * n + s] = ge[i];
        }
    }
}

// prm = {A, B, kappa, Gamma, tau_f, tau_g, rho0, stencil, force, collision,
// lambda}; stencil, force and collision are selectors (0 or 1).
Params<double> params_from(const double* prm) {
    return Params<double>{prm[0], prm[1], prm[2], prm[3], prm[4], prm[5], prm[6],
                          prm[7] != 0.0 ? 1 : 0, prm[8] != 0.0 ? 1 : 0, prm[9] != 0.0 ? 1 : 0, prm[10]};
}

Params<Dual> dual_params_from(const double* prm, const double* dprm) {
    Params<Dual> p;
    p.A = Dual(prm[0], dprm[0]);
    p.B = Dual(prm[1], dprm[1]);
    p.kappa = Dual(prm[2], dprm[2]);
    p.Gamma = Dual(prm[3], dprm[3]);
    p.tau_f = Dual(prm[4], dprm[4]);
    p.tau_g = Dual(prm[5], dprm[5]);
    p.rho0 = Dual(prm[6], dprm[6]);
    p.stencil = prm[7] != 0.0 ? 1 : 0;  // selectors, not differentiated
    p.force = prm[8] != 0.0 ? 1 : 0;
    p.collision = prm[9] != 0.0 ? 1 : 0;
    p.lambda = Dual(prm[10], 0.0);  // not differentiated
    return p;
}

bool dims_ok(int nx, int ny, int nz) { return nx >= 1 && ny >= 1 && nz >= 1; }

// Deterministic sum: per-plane partials, then planes in z order.
double plane_ordered_sum(const Lattice& L, const double* a) {
    std::vector<double> part(L.nz, 0.0);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < L.nz; ++z) {
        double acc = 0.0;
        for (long s = (long)z * L.nx * L.ny; s < (long)(z + 1) * L.nx * L.ny; ++s) acc += a[s];
        part[z] = acc;
    }
    double total = 0.0;
    for (int z = 0; z < L.nz; ++z) total += part[z];
    return total;
}

}  // namespace

// ---------------------------------------------------------------------------
// C interface (called from Python through ctypes by the tests only).
// prm = {A, B, kappa, Gamma, tau_f, tau_g, rho0, stencil, force, collision,
// lambda}; the derivative direction dprm has the first seven. Return 0 on
// success, -1 on bad arguments.
extern "C" {

int orc_version() { return 4; }

// Chemical stress P (6 x N, [xx, yy, zz, xy, xz, yz]) of a phi field with the
// stencils and parameters of prm.
int orc_stress(int nx, int ny, int nz, const double* prm, const double* phi, double* P) {
    if (!dims_ok(nx, ny, nz) || !prm || !phi || !P) return -1;
    Lattice L(nx, ny, nz);
    Params<double> p = params_from(prm);
    std::vector<double> lap(L.n);
    laplacian(L, phi, lap.data(), p.stencil);
    chemical_stress(L, p, phi, lap.data(), P);
    return 0;
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

int orc_get_threads() {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_lattice(int* c, double* w) {
    for (int i = 0; i < kQ; ++i) {
        c[3 * i + 0] = kCx[i];
        c[3 * i + 1] = kCy[i];
        c[3 * i + 2] = kCz[i];
        w[i] = weight(i);
    }
}

void orc_feq(double rho, const double* u, double* out) { feq_site(rho, u, out); }

void orc_geq(double phi, const double* u, double mu, double Gamma, double* out) {
    geq_site(phi, u, mu, Gamma, out);
}

void orc_guo(const double* u, const double* F, double tau, double* out) {
    guo_site(u, F, tau, out);
}

int orc_laplacian(int nx, int ny, int nz, int stencil, const double* phi, double* lap) {
    if (!dims_ok(nx, ny, nz) || !phi || !lap || (stencil != 0 && stencil != 1)) return -1;
    laplacian(Lattice(nx, ny, nz), phi, lap, stencil);
    return 0;
}

int orc_gradient(int nx, int ny, int nz, int stencil, const double* h, double* grad) {
    if (!dims_ok(nx, ny, nz) || !h || !grad || (stencil != 0 && stencil != 1)) return -1;
    gradient(Lattice(nx, ny, nz), h, grad, stencil);
    return 0;
}

int orc_propagate(int nx, int ny, int nz, int reverse, const double* in, double* out) {
    if (!dims_ok(nx, ny, nz) || !in || !out || in == out) return -1;
    Lattice L(nx, ny, nz);
    if (reverse)
        propagate_reverse(L, in, out);
    else
        propagate(L, in, out);
    return 0;
}

int orc_init(int nx, int ny, int nz, const double* prm, const double* phi, const double* rho,
             const double* u, double* f, double* g) {
    if (!dims_ok(nx, ny, nz) || !prm || !phi || !f || !g) return -1;
    init_state(Lattice(nx, ny, nz), params_from(prm), phi, rho, u, f, g);
    return 0;
}

int orc_step(int nx, int ny, int nz, const double* prm, double* f, double* g, int nsteps) {
    if (!dims_ok(nx, ny, nz) || !prm || !f || !g || nsteps < 0) return -1;
    Lattice L(nx, ny, nz);
    Params<double> p = params_from(prm);
    std::vector<double> tmp(kQ * L.n);
    Macro<double> m(L.n);
    for (int t = 0; t < nsteps; ++t) step(L, p, f, g, tmp.data(), m);
    return 0;
}

// Macroscopic output of a pre-collision state. Any output pointer may be
// null. totals (if given) = {sum rho, sum phi, sum jx, sum jy, sum jz}.
int orc_macros(int nx, int ny, int nz, const double* prm, const double* f, const double* g,
               double* rho, double* u, double* phi, double* gradphi, double* mu, double* force,
               double* totals) {
    if (!dims_ok(nx, ny, nz) || !prm || !f || !g) return -1;
    Lattice L(nx, ny, nz);
    const long n = L.n;
    Macro<double> m(n);
    macroscopic(L, params_from(prm), f, g, m);
    if (rho) std::memcpy(rho, m.rho.data(), sizeof(double) * n);
    if (u) std::memcpy(u, m.u.data(), sizeof(double) * 3 * n);
    if (phi) std::memcpy(phi, m.phi.data(), sizeof(double) * n);
    if (mu) std::memcpy(mu, m.mu.data(), sizeof(double) * n);
    if (force) std::memcpy(force, m.F.data(), sizeof(double) * 3 * n);
    if (gradphi) gradient(L, m.phi.data(), gradphi, params_from(prm).stencil);
    if (totals) {
        totals[0] = plane_ordered_sum(L, m.rho.data());
        totals[1] = plane_ordered_sum(L, m.phi.data());
        for (int a = 0; a < 3; ++a) totals[2 + a] = plane_ordered_sum(L, m.j.data() + a * n);
    }
    return 0;
}

// Tangent-linear model. Values in f, g; one direction in df, dg; parameter
// direction dprm (same order as prm). Advances both by nsteps.
int orc_step_tl(int nx, int ny, int nz, const double* prm, const double* dprm, double* f,
                double* g, double* df, double* dg, int nsteps) {
    if (!dims_ok(nx, ny, nz) || !prm || !dprm || !f || !g || !df || !dg || nsteps < 0) return -1;
    Lattice L(nx, ny, nz);
    const long nq = kQ * L.n;
    Params<Dual> p = dual_params_from(prm, dprm);
    std::vector<Dual> F(nq), G(nq), tmp(nq);
    for (long k = 0; k < nq; ++k) {
        F[k] = Dual(f[k], df[k]);
        G[k] = Dual(g[k], dg[k]);
    }
    Macro<Dual> m(L.n);
    for (int t = 0; t < nsteps; ++t) step(L, p, F.data(), G.data(), tmp.data(), m);
    for (long k = 0; k < nq; ++k) {
        f[k] = F[k].v;
        df[k] = F[k].d;
        g[k] = G[k].v;
        dg[k] = G[k].d;
    }
    return 0;
}

// Loss L = sum_x (phi_T(x) - phi_target(x))^2 after init from phi0 (rho0,
// u = 0) and nsteps steps, and its directional derivative along (dphi0,
// dprm). dphi0 may be null (zero direction).
int orc_loss_jvp(int nx, int ny, int nz, const double* prm, const double* dprm,
                 const double* phi0, const double* dphi0, const double* phi_target, int nsteps,
                 double* loss, double* dloss) {
    if (!dims_ok(nx, ny, nz) || !prm || !dprm || !phi0 || !phi_target || nsteps < 0 || !loss ||
        !dloss)
        return -1;
    Lattice L(nx, ny, nz);
    const long n = L.n, nq = kQ * n;
    Params<Dual> p = dual_params_from(prm, dprm);
    std::vector<Dual> phi(n), F(nq), G(nq), tmp(nq);
    for (long s = 0; s < n; ++s) phi[s] = Dual(phi0[s], dphi0 ? dphi0[s] : 0.0);
    init_state<Dual>(L, p, phi.data(), nullptr, nullptr, F.data(), G.data());
    Macro<Dual> m(n);
    for (int t = 0; t < nsteps; ++t) step(L, p, F.data(), G.data(), tmp.data(), m);
    double acc = 0.0, dacc = 0.0;
    for (long s = 0; s < n; ++s) {
        Dual ph = 0.0;
        for (int i = 0; i < kQ; ++i) ph += G[i * n + s];
        Dual r = ph - phi_target[s];
        Dual r2 = r * r;
        acc += r2.v;
        dacc += r2.d;
    }
    *loss = acc;
    *dloss = dacc;
    return 0;
}

}  // extern "C"
