// Liquid-crystal timestep on the GPU: a Landau-de Gennes Q-tensor evolved by
// the Beris-Edwards equation, coupled to D3Q19 lattice-Boltzmann flow through
// the divergence of its chemical stress (the paper's Ludwig test case, Sec.
// 2.1.1: "Order Parameter Gradients", "Chemical stress", "Collision",
// "Propagation", "LC Update", "Advection"; one elastic constant):
//   H_ab = -A0 (1 - gamma/3) Q_ab + A0 gamma (Q_ac Q_cb - delta_ab Q_cd Q_cd/3)
//          - A0 gamma (Q_cd Q_cd) Q_ab + kappa lap(Q_ab)
//   sigma_ab = f delta_ab - kappa d_a Q_cd d_b Q_cd - xi H_ac (Q_cb + delta_cb/3)
//          - xi (Q_ac + delta_ac/3) H_cb + 2 xi (Q_ab + delta_ab/3) Q_cd H_cd
//          + Q_ac H_cb - H_ac Q_cb,   f the free energy density (bulk + gradient)
//   F_a = d_b sigma_ab,  u = (j + F/2)/rho,  f collided (BGK + Guo) and pushed
//   Q(t+1) = Q + Gamma H + S(W, Q) - u.grad(Q) (first-order upwind), W_ab = d_b u_a,
//   S = (xi D + Om)(Q + I/3) + (Q + I/3)(xi D - Om) - 2 xi (Q + I/3) tr(Q W).
// d is the 2-point central difference, lap the 7-point Laplacian, dt = 1.
// Two step forms (lc_ctx::kernel):
//   generic, three launches, one thread per site in site order (any lattice):
//     k_lc_field    Q (+ its six neighbours) -> H (5 values), sigma (9)
//     k_lc_collide  sigma (+ neighbours), f -> F, u (3 values stored), f
//                   collided and pushed into the other buffer
//     k_lc_update   Q, H, u (+ neighbours) -> Q of the next step (other buffer)
//   fused, two launches (nx % 32 == 0, ny % 8 == 0): k_lc_fused marches tile
//     columns up z with Q and sigma in shared memory and writes only f and u;
//     k_lc_update then recomputes H from Q (see the comment at k_lc_fused).
// Every form uses the same per-site helpers in the same order, so FP64 gives
// the same bits either way.
// Q is stored as its five independent components (xx, xy, xz, yy, yz; zz =
// -xx - yy): symmetric and traceless by construction (the trace of S, from
// the lattice fluid's slight compressibility, is dropped).
// Template on the arithmetic and storage type T (double or float): FP64 is
// instantiated without FMA contraction (lc_f64.cu), FP32 with it (lc_f32.cu).
#pragma once
#include <cuda_runtime.h>

#include "ld_common.cuh"
#include "lc_internal.h"

namespace lc {
namespace {

using ld::Q;
using ld::cx;
using ld::cy;
using ld::cz;
using ld::wgt;

constexpr int kLcThreads = 128;

// a1 = -A0 (1 - gamma/3), a1n = A0 (1 - gamma/3), a2 = A0 gamma: the bulk
// coefficients of H and of the free energy density (and the products of
// them the helpers use, formed once here in FP64).
// fm: the fluid's BGK + Guo constants (omega_f = 1/tau_f, force_pre =
// 1 - 1/(2 tau_f)) for the binary fluid's collision of f, which is the same
// collision.
template <class T>
struct LcModel {
    T A0, gamma, kappa, Gamma, xi, a1, a1n, a2;
    T a2_3, half_kappa, two_xi, xi2_3, fe_a1, fe_a2;  // a2/3, kappa/2, 2 xi, 2 xi/3, a1n/2, a2/4
    ld::Model<T> fm;
};
template <class T>
LcModel<T> lc_model_of(const lc_params& p) {
    const double a1n = p.A0 * (1.0 - p.gamma / 3.0);
    LcModel<T> m{};
    m.A0 = (T)p.A0;
    m.gamma = (T)p.gamma;
    m.kappa = (T)p.kappa;
    m.Gamma = (T)p.Gamma;
    m.xi = (T)p.xi;
    m.a1 = (T)(-a1n);
    m.a1n = (T)a1n;
    m.a2 = (T)(p.A0 * p.gamma);
    m.a2_3 = (T)(p.A0 * p.gamma / 3.0);
    m.half_kappa = (T)(0.5 * p.kappa);
    m.two_xi = (T)(2.0 * p.xi);
    m.xi2_3 = (T)(2.0 * p.xi / 3.0);
    m.fe_a1 = (T)(0.5 * a1n);
    m.fe_a2 = (T)(0.25 * p.A0 * p.gamma);
    m.fm.omega_f = (T)(1.0 / p.tau_f);
    m.fm.force_pre = (T)(1.0 - 0.5 / p.tau_f);
    m.fm.omega_m = m.fm.omega_f;
    m.fm.force_pre_m = m.fm.force_pre;
    return m;
}

struct LcGeom {
    int nx, ny, nz;
    long long n, npad;
};

// Symmetric tensors are held as their six unique components (xx, xy, xz,
// yy, yz, zz); the stored Q has five, zz = -xx - yy. sym_a/sym_b give the
// index pair of component k, sym_w its multiplicity in a full contraction
// (1 on the diagonal, 2 off it), sym_k the component of (a, b).
__device__ __forceinline__ int sym_a(int k) { return k < 3 ? 0 : (k < 5 ? 1 : 2); }
__device__ __forceinline__ int sym_b(int k) { return k < 3 ? k : (k < 5 ? k - 2 : 2); }
template <class T>
__device__ __forceinline__ T sym_w(int k) {
    return (k == 0 || k == 3 || k == 5) ? T(1) : T(2);
}
__device__ __forceinline__ int sym_k(int a, int b) {
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return lo == 0 ? hi : (lo == 1 ? hi + 2 : 5);
}

// The six components of Q at element offset s of the [5][npad] store.
template <class T>
__device__ __forceinline__ void lc_load6(const T* q, long long npad, long long s, T (&v)[6]) {
#pragma unroll
    for (int k = 0; k < 5; ++k) v[k] = q[k * npad + s];
    v[5] = -v[0] - v[3];
}

// Arithmetic of the stencil helpers below: T itself (float or double), or
// LcF2, two x-adjacent sites in packed FP32 (sm_100 f32x2 instructions: one
// instruction for both sites, each lane rounded as the scalar operation).
struct LcF2 {
    float2 v;
    LcF2() = default;
    __device__ explicit LcF2(float2 a) : v(a) {}
    __device__ explicit LcF2(double a) : v(make_float2((float)a, (float)a)) {}
};
__device__ __forceinline__ LcF2 operator+(LcF2 a, LcF2 b) { return LcF2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ LcF2 operator*(LcF2 a, LcF2 b) { return LcF2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ LcF2 operator-(LcF2 a, LcF2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;"
        : "=l"(r)
        : "l"(*reinterpret_cast<const unsigned long long*>(&a.v)), "l"(*reinterpret_cast<const unsigned long long*>(&b.v)));
    return LcF2(*reinterpret_cast<const float2*>(&r));
}
__device__ __forceinline__ LcF2& operator+=(LcF2& a, LcF2 b) { return a = a + b; }
// a * b + c: one fused operation for the pairs, the plain expression for T
// (contracted in FP32, two roundings in the FP64 unit built without
// contraction).
__device__ __forceinline__ LcF2 lc_fma(LcF2 a, LcF2 b, LcF2 c) { return LcF2(__ffma2_rn(a.v, b.v, c.v)); }
template <class T>
__device__ __forceinline__ T lc_fma(T a, T b, T c) {
    return a * b + c;
}
// zz = -xx - yy of a traceless tensor
__device__ __forceinline__ LcF2 lc_zz(LcF2 xx, LcF2 yy) { return LcF2(-1.0) * xx - yy; }
template <class T>
__device__ __forceinline__ T lc_zz(T xx, T yy) {
    return -xx - yy;
}

// Model constants of the stencil helpers in arithmetic A (broadcast to both
// lanes for LcF2): a1 = -A0 (1 - gamma/3), a2 = A0 gamma, a2_3 = a2/3,
// kappa, xi, two_xi = 2 xi, xi2_3 = 2 xi/3, fe_a1 = a1n/2 and fe_a2 = a2/4 of
// the free energy density.
template <class A>
struct LcCoef {
    A a1, a2, a2_3, kappa, half_kappa, xi, two_xi, xi2_3, fe_a1, fe_a2;
};
template <class A, class T>
__device__ __forceinline__ LcCoef<A> lc_coef(const LcModel<T>& m) {
    LcCoef<A> c;
    c.a1 = A(m.a1);
    c.a2 = A(m.a2);
    c.a2_3 = A(m.a2_3);
    c.kappa = A(m.kappa);
    c.half_kappa = A(m.half_kappa);
    c.xi = A(m.xi);
    c.two_xi = A(m.two_xi);
    c.xi2_3 = A(m.xi2_3);
    c.fe_a1 = A(m.fe_a1);
    c.fe_a2 = A(m.fe_a2);
    return c;
}

// Central-difference gradient dQ[c][k] = d_c Q_k and 7-point Laplacian of
// Q at a site. nb(c, sgn, v) fills v with the six components of the
// neighbour at sgn * e_c.
template <class A, class Nb>
__device__ __forceinline__ void lc_grad_lap(const A (&q)[6], Nb nb, A (&dQ)[3][6], A (&lap)[6]) {
#pragma unroll
    for (int k = 0; k < 6; ++k) lap[k] = A(-6.0) * q[k];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        A qp[6], qm[6];
        nb(c, 1, qp);
        nb(c, -1, qm);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            dQ[c][k] = A(0.5) * (qp[k] - qm[k]);
            lap[k] += qp[k] + qm[k];
        }
    }
}

// The contraction X:Y of two symmetric tensors from their six components
// (off-diagonal products counted twice).
template <class A>
__device__ __forceinline__ A lc_sym_dot(const A (&x)[6], const A (&y)[6]) {
    const A diag = lc_fma(x[5], y[5], lc_fma(x[3], y[3], x[0] * y[0]));
    const A off = lc_fma(x[4], y[4], lc_fma(x[2], y[2], x[1] * y[1]));
    return diag + (off + off);
}

// Molecular field H = -dF/dQ of the Landau-de Gennes free energy with one
// elastic constant, on the six components:
//   H = a1 Q + a2 (QQ - tr2 I/3) - a2 tr2 Q + kappa lap Q;
// also returns tr2 = Q:Q and the square QQ = Q.Q (symmetric) for the stress.
template <class A>
__device__ __forceinline__ void lc_molecular_field(const A (&q)[6], const A (&lap)[6], const LcCoef<A>& m, A& tr2,
                                                   A (&qq)[6], A (&H)[6]) {
    tr2 = lc_sym_dot(q, q);
    const A tr2_3 = tr2 * A(1.0 / 3.0), a2tr2 = m.a2 * tr2;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const int a = sym_a(k), b = sym_b(k);
        A s = q[sym_k(a, 0)] * q[sym_k(0, b)];
        s = lc_fma(q[sym_k(a, 1)], q[sym_k(1, b)], s);
        s = lc_fma(q[sym_k(a, 2)], q[sym_k(2, b)], s);
        qq[k] = s;
        const A dev = a == b ? s - tr2_3 : s;
        H[k] = lc_fma(m.kappa, lap[k], lc_fma(m.a2, dev, (m.a1 - a2tr2) * q[k]));
    }
}

// Chemical stress sigma_ab of a site. With P = Q.H (so H.Q = P^T, Q and H
// being symmetric) the terms of H collapse to
//   -xi (P_ab + P_ba) - (2 xi/3) H_ab + 2 xi (Q_ab + delta_ab/3) Q:H + P_ab - P_ba,
// the elastic term is -kappa G_ab with G_ab = d_a Q_cd d_b Q_cd (symmetric),
// and the free energy density f on the diagonal uses |grad Q|^2 = tr G and
// tr(Q^3) = QQ:Q. out(a, b, value) receives each component.
template <class A, class Out>
__device__ __forceinline__ void lc_stress(const A (&q)[6], const A (&dQ)[3][6], const A (&H)[6], const A (&qq)[6],
                                          A tr2, const LcCoef<A>& m, Out out) {
    const A tr3 = lc_sym_dot(qq, q), qh = lc_sym_dot(q, H);
    A G[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const int a = sym_a(k), b = sym_b(k);
        const A diag = lc_fma(dQ[a][5], dQ[b][5], lc_fma(dQ[a][3], dQ[b][3], dQ[a][0] * dQ[b][0]));
        const A off = lc_fma(dQ[a][4], dQ[b][4], lc_fma(dQ[a][2], dQ[b][2], dQ[a][1] * dQ[b][1]));
        G[k] = diag + (off + off);
    }
    const A grad2 = G[0] + G[3] + G[5];
    // f = a1n/2 tr2 - a2/3 tr3 + a2/4 tr2^2 + kappa/2 |grad Q|^2
    const A fe = lc_fma(m.half_kappa, grad2, lc_fma(m.fe_a2 * tr2, tr2, m.fe_a1 * tr2 - m.a2_3 * tr3));
    A P[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            A s = q[sym_k(a, 0)] * H[sym_k(0, b)];
            s = lc_fma(q[sym_k(a, 1)], H[sym_k(1, b)], s);
            P[a][b] = lc_fma(q[sym_k(a, 2)], H[sym_k(2, b)], s);
        }
    const A tq = m.two_xi * qh;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int k = sym_k(a, b);
            // 2 xi (Q + delta/3) Q:H - (2 xi/3) H - kappa G - xi (P + P^T) + (P - P^T) [+ f]
            A v = lc_fma(tq, a == b ? q[k] + A(1.0 / 3.0) : q[k], (P[a][b] - P[b][a]) - m.xi * (P[a][b] + P[b][a]));
            v = v - lc_fma(m.kappa, G[k], m.xi2_3 * H[k]);
            out(a, b, a == b ? v + fe : v);
        }
}

// Velocity u = (j + F/2)/rho and the BGK + Guo collision of one site's f
// (in place), by the binary fluid's routines (guo_velocity, collide_f: the
// equilibrium and source term on opposite direction pairs); u is returned in
// uv.
template <class T>
__device__ __forceinline__ void lc_moments_u(const T (&fv)[Q], const T (&Fa)[3], T& rho, T (&uv)[3]) {
    T jx = T(0), jy = T(0), jz = T(0);
    rho = T(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        rho += fv[i];
        ld::add_c(i, fv[i], jx, jy, jz);
    }
    ld::guo_velocity(rho, jx, jy, jz, Fa[0], Fa[1], Fa[2], uv[0], uv[1], uv[2]);
}
template <class T>
__device__ __forceinline__ void lc_collide_site(T (&fv)[Q], const T (&Fa)[3], const LcModel<T>& m, T (&uv)[3]) {
    T rho;
    lc_moments_u(fv, Fa, rho, uv);
    ld::collide_f(fv, rho, uv[0], uv[1], uv[2], Fa[0], Fa[1], Fa[2], m.fm);
}

// The Q update of one site: Q + Gamma H + S(W, Q) - u.grad(Q), the
// advection first-order upwind, W_ab = d_b u_a from the central difference
// of u. qnb(k, c, sgn) is component k of Q at the neighbour sgn * e_c.
template <class T, class QNb>
__device__ __forceinline__ void lc_update_site(const T (&q)[6], const T (&H)[6], const T (&us)[3], const T (&W)[3][3],
                                               const LcModel<T>& m, QNb qnb, T (&qn)[5]) {
    T D[3][3], Om[3][3], Qp[3][3];
    T trQW = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            D[a][b] = T(0.5) * (W[a][b] + W[b][a]);
            Om[a][b] = T(0.5) * (W[a][b] - W[b][a]);
            Qp[a][b] = q[sym_k(a, b)] + (a == b ? T(1) / T(3) : T(0));
            trQW += q[sym_k(a, b)] * W[b][a];
        }
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int a = sym_a(k), b = sym_b(k);
        T S = T(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) S += (m.xi * D[a][c] + Om[a][c]) * Qp[c][b] + Qp[a][c] * (m.xi * D[c][b] - Om[c][b]);
        S = S - T(2) * m.xi * Qp[a][b] * trQW;
        const T qc = q[k];
        T adv = T(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const bool fwd = us[c] >= T(0);
            const T diff = fwd ? qc - qnb(k, c, -1) : qnb(k, c, 1) - qc;
            adv += us[c] * diff;
        }
        qn[k] = qc + m.Gamma * H[k] + S - adv;
    }
}

// Site coordinates and the element offsets of its six axis neighbours
// (periodic), for the per-site kernels: nbr[2c] at +e_c, nbr[2c+1] at -e_c.
struct LcSite {
    int s, x, y, z;
    int nbr[6];
};
__device__ __forceinline__ bool lc_site_of(const LcGeom& g, LcSite& t) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.n) return false;  // n < 2^31 (lc_create)
    t.s = (int)s;
    t.x = t.s % g.nx;
    const int r = t.s / g.nx;
    t.y = r % g.ny;
    t.z = r / g.ny;
    const int plane = g.nx * g.ny;
    t.nbr[0] = t.s + (t.x + 1 == g.nx ? 1 - g.nx : 1);
    t.nbr[1] = t.s + (t.x == 0 ? g.nx - 1 : -1);
    t.nbr[2] = t.s + (t.y + 1 == g.ny ? (1 - g.ny) * g.nx : g.nx);
    t.nbr[3] = t.s + (t.y == 0 ? (g.ny - 1) * g.nx : -g.nx);
    t.nbr[4] = t.s + (t.z + 1 == g.nz ? (1 - g.nz) * plane : plane);
    t.nbr[5] = t.s + (t.z == 0 ? (g.nz - 1) * plane : -plane);
    return true;
}
__device__ __forceinline__ int lc_nb(const LcSite& t, int c, int sgn) { return t.nbr[2 * c + (sgn > 0 ? 0 : 1)]; }

template <class T>
__global__ void __launch_bounds__(kLcThreads) k_lc_field(LcGeom g, LcModel<T> m, const T* __restrict__ q,
                                                         T* __restrict__ h, T* __restrict__ sigma) {
    LcSite t;
    if (!lc_site_of(g, t)) return;
    const LcCoef<T> cf = lc_coef<T>(m);
    T q6[6], dQ[3][6], lap[6], H[6], qq[6], tr2;
    lc_load6(q, g.npad, t.s, q6);
    lc_grad_lap(q6, [&](int c, int sgn, T (&v)[6]) { lc_load6(q, g.npad, lc_nb(t, c, sgn), v); }, dQ, lap);
    lc_molecular_field(q6, lap, cf, tr2, qq, H);
    lc_stress(q6, dQ, H, qq, tr2, cf, [&](int a, int b, T v) { sigma[(3 * a + b) * g.npad + t.s] = v; });
#pragma unroll
    for (int k = 0; k < 5; ++k) h[k * g.npad + t.s] = H[k];
}

template <class T>
__global__ void __launch_bounds__(kLcThreads) k_lc_collide(LcGeom g, LcModel<T> m, const T* __restrict__ sigma,
                                                           const T* __restrict__ f, T* __restrict__ fd,
                                                           T* __restrict__ u) {
    LcSite t;
    if (!lc_site_of(g, t)) return;
    T Fa[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const int sp = lc_nb(t, b, 1), sm = lc_nb(t, b, -1);
#pragma unroll
        for (int a = 0; a < 3; ++a) Fa[a] += T(0.5) * (sigma[(3 * a + b) * g.npad + sp] - sigma[(3 * a + b) * g.npad + sm]);
    }
    T fv[Q], uv[3];
#pragma unroll
    for (int i = 0; i < Q; ++i) fv[i] = f[i * g.npad + t.s];
    lc_collide_site(fv, Fa, m, uv);
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a * g.npad + t.s] = uv[a];
    // push: the destination's offset from s is the sum of its axis steps
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int d = t.s + (cx(i) > 0 ? t.nbr[0] - t.s : (cx(i) < 0 ? t.nbr[1] - t.s : 0)) +
                      (cy(i) > 0 ? t.nbr[2] - t.s : (cy(i) < 0 ? t.nbr[3] - t.s : 0)) +
                      (cz(i) > 0 ? t.nbr[4] - t.s : (cz(i) < 0 ? t.nbr[5] - t.s : 0));
        fd[i * g.npad + d] = fv[i];
    }
}

// RECOMPUTE_H: form H from Q here (the fused step stores no H) instead of
// reading the h written by k_lc_field; the same arithmetic either way.
template <class T, bool RECOMPUTE_H>
__global__ void __launch_bounds__(kLcThreads) k_lc_update(LcGeom g, LcModel<T> m, const T* __restrict__ q,
                                                          const T* __restrict__ u, const T* __restrict__ h,
                                                          T* __restrict__ qn) {
    LcSite t;
    if (!lc_site_of(g, t)) return;
    T W[3][3], q6[6], H[6], us[3], qv[5];
#pragma unroll
    for (int a = 0; a < 3; ++a) us[a] = u[a * g.npad + t.s];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const int sp = lc_nb(t, b, 1), sm = lc_nb(t, b, -1);
#pragma unroll
        for (int a = 0; a < 3; ++a) W[a][b] = T(0.5) * (u[a * g.npad + sp] - u[a * g.npad + sm]);
    }
    lc_load6(q, g.npad, t.s, q6);
    T qnb[3][2][6];  // Q at the six neighbours, for H and the upwind differences
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        lc_load6(q, g.npad, lc_nb(t, c, 1), qnb[c][0]);
        lc_load6(q, g.npad, lc_nb(t, c, -1), qnb[c][1]);
    }
    if constexpr (RECOMPUTE_H) {
        T dQ[3][6], lap[6], qq[6], tr2;
        lc_grad_lap(q6, [&](int c, int sgn, T (&v)[6]) {
#pragma unroll
            for (int k = 0; k < 6; ++k) v[k] = qnb[c][sgn > 0 ? 0 : 1][k];
        }, dQ, lap);
        lc_molecular_field(q6, lap, lc_coef<T>(m), tr2, qq, H);
    } else {
#pragma unroll
        for (int k = 0; k < 5; ++k) H[k] = h[k * g.npad + t.s];
        H[5] = T(0);  // unused by the update
    }
    lc_update_site(q6, H, us, W, m, [&](int k, int c, int sgn) { return qnb[c][sgn > 0 ? 0 : 1][k]; }, qv);
#pragma unroll
    for (int k = 0; k < 5; ++k) qn[k * g.npad + t.s] = qv[k];
}

// ---------------------------------------------------------------------------
// Fused field + collision step. Each CTA owns a kLcTX x kLcTY column of sites
// and marches up a chunk of z-planes. The stress chain Q -> (H, sigma) ->
// F = div sigma needs sigma within one site and so Q within two sites of every
// collided site. Shared memory holds:
//   Q ring:     4 planes x 5 components over the tile + 2-site halo;
//   sigma:      what F reads of the planes sigma has been formed for:
//               sigma_a0 over the tile + x halo and sigma_a1 over the tile +
//               y halo (planes k, k+1), sigma_a2 over the tile (k-1..k+1);
//   f tile:     the 19 distributions of the plane being collided (STAGE_F).
// Iteration k: copies of f(k) and of Q(k+3) are issued (cp.async, no
// registers held), sigma(k+1) is formed from Q(k..k+2) (which landed during
// the previous iteration), then F, u, the collision and push of plane k read
// f(k) from shared memory and store f and u. Per site the launch reads Q once
// from HBM (halo re-reads hit L2) and f once, and writes f and u; H and sigma
// never leave the SM. The arithmetic of every site is the per-site kernels'
// (lc_grad_lap, lc_molecular_field, lc_stress, lc_collide_site), in the same
// order, so FP64 gives their bits.
constexpr int kLcTX = 32, kLcTY = 8, kLcFusedThreads = kLcTX * kLcTY;
constexpr int kLcQW = kLcTX + 4, kLcQH = kLcTY + 4;  // Q ring plane (tile + 2-halo)
constexpr int kLcQSlots = 4;
// sigma sites: the tile, then its x halo (2 columns x TY), then its y halo
constexpr int kLcSigmaSites = kLcTX * kLcTY + 2 * kLcTY + 2 * kLcTX;

// Shared-memory layout, in elements of T.
struct LcFusedLayout {
    static constexpr int q = 0;                                        // [4][5][QH][QW]
    static constexpr int sx = q + kLcQSlots * 5 * kLcQH * kLcQW;       // [2][3][TY][TX+2]
    static constexpr int sy = sx + 2 * 3 * kLcTY * (kLcTX + 2);        // [2][3][TY+2][TX]
    static constexpr int sz = sy + 2 * 3 * (kLcTY + 2) * kLcTX;        // [3][3][TY][TX]
    static constexpr int f = sz + 3 * 3 * kLcTY * kLcTX;               // [19][TY][TX]
    static constexpr int end_nof = f;
    static constexpr int end = f + Q * kLcTY * kLcTX;
};
template <class T, bool STAGE_F>
constexpr size_t lc_fused_smem() {
    return (size_t)(STAGE_F ? LcFusedLayout::end : LcFusedLayout::end_nof) * sizeof(T);
}
// Resident CTAs per SM that the shared memory allows (FP32: 77 KB with the f
// tile, two CTAs; 58 KB without, three; FP64: one).
template <class T, bool STAGE_F>
constexpr int lc_fused_ctas() {
    return sizeof(T) == 8 ? 1 : (STAGE_F ? 2 : 3);
}
// Stage f through shared memory in FP32 (measured against register loads).
constexpr bool kLcStageF = true;
// FP32: form sigma two x-adjacent sites at a time in packed arithmetic.
constexpr bool kLcPairSigma = true;

__device__ __forceinline__ int lc_wrap(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// First plane of z-chunk b when nz planes are split into nchunks chunks
// whose lengths differ by at most one.
__host__ __device__ inline int lc_chunk_begin(int b, int nz, int nchunks) {
    return (int)(((long long)b * nz) / nchunks);
}

// cp.async of 8 or 16 bytes (both addresses aligned to the size), and the
// group waits; hardware waits, the copies always land.
template <int BYTES>
__device__ __forceinline__ void lc_cp_async(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void lc_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void lc_cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// I: type of the element offsets i * npad + s (32-bit where 19 npad fits).
template <class T, class I, bool STAGE_F>
__global__ void __launch_bounds__(kLcFusedThreads, (lc_fused_ctas<T, STAGE_F>()))
    k_lc_fused(LcGeom g, LcModel<T> m, int nchunks, const T* __restrict__ q, const T* __restrict__ f,
               T* __restrict__ fd, T* __restrict__ u) {
    using L = LcFusedLayout;
    extern __shared__ __align__(16) unsigned char lc_smem[];
    T* sm = reinterpret_cast<T*>(lc_smem);
    auto QR = [&](int slot, int k, int py, int px) -> T& { return sm[L::q + ((slot * 5 + k) * kLcQH + py) * kLcQW + px]; };
    auto SX = [&](int slot, int a, int r, int c) -> T& { return sm[L::sx + ((slot * 3 + a) * kLcTY + r) * (kLcTX + 2) + c]; };
    auto SY = [&](int slot, int a, int r, int c) -> T& { return sm[L::sy + ((slot * 3 + a) * (kLcTY + 2) + r) * kLcTX + c]; };
    auto SZ = [&](int slot, int a, int r, int c) -> T& { return sm[L::sz + ((slot * 3 + a) * kLcTY + r) * kLcTX + c]; };
    auto FT = [&](int i, int r, int c) -> T& { return sm[L::f + (i * kLcTY + r) * kLcTX + c]; };

    const int tid = threadIdx.x;
    const int tx = tid % kLcTX, ty = tid / kLcTX;
    const int x0 = blockIdx.x * kLcTX, y0 = blockIdx.y * kLcTY;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int z0 = lc_chunk_begin(blockIdx.z, nz, nchunks), z1 = lc_chunk_begin(blockIdx.z + 1, nz, nchunks);
    const int plane = nx * ny;
    const I npad = (I)g.npad;

    // Copies of Q of plane zp over the tile + 2-halo into ring slot `slot`,
    // two x-adjacent sites per copy (the halo starts at an even x and nx is
    // even, so a pair never straddles the periodic wrap).
    auto q_plane_async = [&](int zp, int slot) {
        constexpr int QW2 = kLcQW / 2;
        const int zoff = lc_wrap(zp, nz) * plane;
        for (int idx = tid; idx < QW2 * kLcQH; idx += kLcFusedThreads) {
            const int px = 2 * (idx % QW2), py = idx / QW2;
            const int s = zoff + lc_wrap(y0 + py - 2, ny) * nx + lc_wrap(x0 + px - 2, nx);
#pragma unroll
            for (int k = 0; k < 5; ++k) lc_cp_async<2 * sizeof(T)>(&QR(slot, k, py, px), q + k * npad + s);
        }
    };
    // Copies of the tile's f of plane zp (16-byte pieces of its rows).
    auto f_plane_async = [&](int zp) {
        constexpr int kPer = 16 / sizeof(T), kRow = kLcTX / kPer;
        for (int idx = tid; idx < Q * kLcTY * kRow; idx += kLcFusedThreads) {
            const int c = (idx % kRow) * kPer, r = (idx / kRow) % kLcTY, i = idx / (kRow * kLcTY);
            lc_cp_async<16>(&FT(i, r, c), f + i * npad + (zp * plane + (y0 + r) * nx + x0 + c));
        }
    };
    auto six_at = [&](int slot, int py, int px, T (&v)[6]) {
#pragma unroll
        for (int k = 0; k < 5; ++k) v[k] = QR(slot, k, py, px);
        v[5] = -v[0] - v[3];
    };
    // The sigma components that F reads, of the site at (hx, hy) of the
    // tile + 1-halo frame: sigma_a0 on the tile rows, sigma_a1 on the tile
    // columns, sigma_a2 on the tile; into slot xy of SX/SY and zs of SZ.
    auto put_sigma = [&](int hx, int hy, int xy, int zs, int a, int b, T v) {
        const bool in_x = hx >= 1 && hx <= kLcTX, in_y = hy >= 1 && hy <= kLcTY;
        if (b == 0 && in_y) SX(xy, a, hy - 1, hx) = v;
        if (b == 1 && in_x) SY(xy, a, hy, hx - 1) = v;
        if (b == 2 && in_x && in_y) SZ(zs, a, hy - 1, hx - 1) = v;
    };
    // sigma of the plane whose Q is in slot `mid` (below: lo, above: hi).
    // Scalar: one site per thread over the tile, then its x halo and y halo.
    // Pairs (FP32): the (TX+2) x (TY+2) frame as x-adjacent pairs of sites,
    // one pair per thread in packed arithmetic (the corners come along and are
    // not stored).
    auto sigma_plane = [&](int lo, int mid, int hi, int xy, int zs) {
        if constexpr (kLcPairSigma && sizeof(T) == 4) {
            const LcCoef<LcF2> cf = lc_coef<LcF2>(m);
            constexpr int kPairsX = (kLcTX + 2) / 2;
            for (int idx = tid; idx < kPairsX * (kLcTY + 2); idx += kLcFusedThreads) {
                const int hx = 2 * (idx % kPairsX), hy = idx / kPairsX;
                const int px = hx + 1, py = hy + 1;
                auto six2 = [&](int slot, int yy, int xx, LcF2 (&v)[6]) {
#pragma unroll
                    for (int k = 0; k < 5; ++k) v[k] = LcF2(make_float2(QR(slot, k, yy, xx), QR(slot, k, yy, xx + 1)));
                    v[5] = lc_zz(v[0], v[3]);
                };
                LcF2 q6[6], dQ[3][6], lap[6], H[6], qq[6], tr2;
                six2(mid, py, px, q6);
                lc_grad_lap(q6, [&](int c, int sgn, LcF2 (&v)[6]) {
                    six2(c == 2 ? (sgn > 0 ? hi : lo) : mid, py + sgn * (c == 1), px + sgn * (c == 0), v);
                }, dQ, lap);
                lc_molecular_field(q6, lap, cf, tr2, qq, H);
                lc_stress(q6, dQ, H, qq, tr2, cf, [&](int a, int b, LcF2 v) {
                    put_sigma(hx, hy, xy, zs, a, b, v.v.x);
                    put_sigma(hx + 1, hy, xy, zs, a, b, v.v.y);
                });
            }
        } else {
            const LcCoef<T> cf = lc_coef<T>(m);
            for (int idx = tid; idx < kLcSigmaSites; idx += kLcFusedThreads) {
                int hx, hy;  // position in the tile + 1-halo frame
                if (idx < kLcTX * kLcTY) {
                    hx = 1 + idx % kLcTX;
                    hy = 1 + idx / kLcTX;
                } else if (idx < kLcTX * kLcTY + 2 * kLcTY) {
                    const int j = idx - kLcTX * kLcTY;
                    hx = (j & 1) * (kLcTX + 1);
                    hy = 1 + (j >> 1);
                } else {
                    const int j = idx - kLcTX * kLcTY - 2 * kLcTY;
                    hx = 1 + j % kLcTX;
                    hy = (j / kLcTX) * (kLcTY + 1);
                }
                const int px = hx + 1, py = hy + 1;
                T q6[6], dQ[3][6], lap[6], H[6], qq[6], tr2;
                six_at(mid, py, px, q6);
                lc_grad_lap(q6, [&](int c, int sgn, T (&v)[6]) {
                    six_at(c == 2 ? (sgn > 0 ? hi : lo) : mid, py + sgn * (c == 1), px + sgn * (c == 0), v);
                }, dQ, lap);
                lc_molecular_field(q6, lap, cf, tr2, qq, H);
                lc_stress(q6, dQ, H, qq, tr2, cf, [&](int a, int b, T v) { put_sigma(hx, hy, xy, zs, a, b, v); });
            }
        }
    };
    auto qs = [&](int zp) { return (zp - z0 + 2) % kLcQSlots; };  // Q slot of plane zp (zp >= z0-2)
    auto xs = [&](int zp) { return (zp - z0 + 1) % 2; };          // SX/SY slot (zp >= z0-1)
    auto ss = [&](int zp) { return (zp - z0 + 1) % 3; };          // SZ slot (zp >= z0-1)

    // Prologue: Q(z0-2..z0+1), sigma(z0-1), sigma(z0); then Q(z0+2) in flight.
    for (int zp = z0 - 2; zp <= z0 + 1; ++zp) q_plane_async(zp, qs(zp));
    lc_cp_commit();
    lc_cp_wait<0>();
    __syncthreads();
    sigma_plane(qs(z0 - 2), qs(z0 - 1), qs(z0), xs(z0 - 1), ss(z0 - 1));
    sigma_plane(qs(z0 - 1), qs(z0), qs(z0 + 1), xs(z0), ss(z0));
    __syncthreads();  // Q(z0+2) takes the slot of Q(z0-2), which sigma(z0-1) read
    q_plane_async(z0 + 2, qs(z0 + 2));
    lc_cp_commit();

    const int x = x0 + tx, y = y0 + ty;
    const int oxp = x + 1 == nx ? 1 - nx : 1, oxm = x == 0 ? nx - 1 : -1;
    const int oyp = y + 1 == ny ? (1 - ny) * nx : nx, oym = y == 0 ? (ny - 1) * nx : -nx;

    for (int k = z0; k < z1; ++k) {
        // the last collision is done with the f tile and the sigma slots of
        // plane k-1, the last sigma pass with Q(k-1)
        __syncthreads();
        if constexpr (STAGE_F) f_plane_async(k);
        lc_cp_commit();
        q_plane_async(k + 3, qs(k + 3));
        lc_cp_commit();
        lc_cp_wait<2>();  // Q(k+2) (issued one iteration ago) has landed
        __syncthreads();
        sigma_plane(qs(k), qs(k + 1), qs(k + 2), xs(k + 1), ss(k + 1));
        lc_cp_wait<1>();  // f(k) has landed
        __syncthreads();

        const int s = k * plane + y * nx + x;  // z1 <= nz
        T Fa[3] = {T(0), T(0), T(0)};
        const int sxy = xs(k), szp = ss(k + 1), szm = ss(k - 1);
#pragma unroll
        for (int a = 0; a < 3; ++a) Fa[a] += T(0.5) * (SX(sxy, a, ty, tx + 2) - SX(sxy, a, ty, tx));
#pragma unroll
        for (int a = 0; a < 3; ++a) Fa[a] += T(0.5) * (SY(sxy, a, ty + 2, tx) - SY(sxy, a, ty, tx));
#pragma unroll
        for (int a = 0; a < 3; ++a) Fa[a] += T(0.5) * (SZ(szp, a, ty, tx) - SZ(szm, a, ty, tx));
        T fv[Q], uv[3];
#pragma unroll
        for (int i = 0; i < Q; ++i) fv[i] = STAGE_F ? FT(i, ty, tx) : __ldcs(f + i * npad + s);
        lc_collide_site(fv, Fa, m, uv);
#pragma unroll
        for (int a = 0; a < 3; ++a) u[a * npad + s] = uv[a];
        const int ozp = k + 1 == nz ? (1 - nz) * plane : plane, ozm = k == 0 ? (nz - 1) * plane : -plane;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int d = s + (cx(i) > 0 ? oxp : (cx(i) < 0 ? oxm : 0)) + (cy(i) > 0 ? oyp : (cy(i) < 0 ? oym : 0)) +
                          (cz(i) > 0 ? ozp : (cz(i) < 0 ? ozm : 0));
            __stcs(fd + i * npad + d, fv[i]);
        }
    }
    lc_cp_wait<0>();  // the last Q prefetch (not read) lands before the CTA exits
}

// z-chunks per tile column: chunk b spans [lc_chunk_begin(b),
// lc_chunk_begin(b + 1)). m in 1..nz minimises waves x (longest chunk + 2),
// each CTA paying about two planes of prologue; the smaller m on a tie.
inline int lc_choose_chunks(int nx, int ny, int nz, int num_sms, int per_sm) {
    const long long cols = (long long)(nx / kLcTX) * (ny / kLcTY);
    const long long slots = (long long)per_sm * num_sms;
    int best = 0;
    long long best_cost = 0;
    for (int m = 1; m <= nz; ++m) {
        const long long cost = ((cols * m + slots - 1) / slots) * ((nz + m - 1) / m + 2);
        if (best == 0 || cost < best_cost) {
            best = m;
            best_cost = cost;
        }
    }
    return best;
}

// Initial f = feq(rho, u) and Q from FP64 inputs (layout [k][n] -> [k][npad]).
template <class T>
__global__ void __launch_bounds__(kLcThreads) k_lc_init(LcGeom g, double rho0, const double* __restrict__ qin,
                                                        const double* __restrict__ rho, const double* __restrict__ uin,
                                                        T* __restrict__ f, T* __restrict__ q) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.n) return;
    const T r = rho ? (T)rho[s] : (T)rho0;
    const T ux = uin ? (T)uin[s] : T(0), uy = uin ? (T)uin[g.n + s] : T(0), uz = uin ? (T)uin[2 * g.n + s] : T(0);
    const T uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T cu = T(cx(i)) * ux + T(cy(i)) * uy + T(cz(i)) * uz;
        f[i * g.npad + s] = wgt<T>(i) * r * (T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu);
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) q[k * g.npad + s] = (T)qin[k * g.n + s];
}

// Outputs as FP64 [k][n]: Q (5), rho, u (3) of the current state (u from the
// stress of the current Q), H (5), f (19); each may be null.
template <class T>
__global__ void __launch_bounds__(kLcThreads) k_lc_out(LcGeom g, const T* __restrict__ q, const T* __restrict__ f,
                                                       const T* __restrict__ sigma, const T* __restrict__ h,
                                                       double* __restrict__ qo, double* __restrict__ rho,
                                                       double* __restrict__ uo, double* __restrict__ ho,
                                                       double* __restrict__ fo) {
    LcSite t;
    if (!lc_site_of(g, t)) return;
    const long long s = t.s;
    if (qo)
        for (int k = 0; k < 5; ++k) qo[k * g.n + s] = (double)q[k * g.npad + s];
    if (ho)
        for (int k = 0; k < 5; ++k) ho[k * g.n + s] = (double)h[k * g.npad + s];
    if (fo)
        for (int i = 0; i < Q; ++i) fo[i * g.n + s] = (double)f[i * g.npad + s];
    if (rho || uo) {
        T Fa[3] = {T(0), T(0), T(0)};
        for (int b = 0; b < 3; ++b) {
            const int sp = lc_nb(t, b, 1), sm = lc_nb(t, b, -1);
            for (int a = 0; a < 3; ++a)
                Fa[a] += T(0.5) * (sigma[(3 * a + b) * g.npad + sp] - sigma[(3 * a + b) * g.npad + sm]);
        }
        T fv[Q], r, uv[3];
#pragma unroll
        for (int i = 0; i < Q; ++i) fv[i] = f[i * g.npad + s];
        lc_moments_u(fv, Fa, r, uv);
        if (rho) rho[s] = (double)r;
        if (uo)
            for (int a = 0; a < 3; ++a) uo[a * g.n + s] = (double)uv[a];
    }
}

inline unsigned lc_blocks(long long n) { return (unsigned)((n + kLcThreads - 1) / kLcThreads); }

template <class T>
struct LcBufs {
    T *f[2], *q[2], *h, *sigma, *u;
};
template <class T>
LcBufs<T> lc_bufs(lc_ctx* c) {
    LcBufs<T> b;
    for (int k = 0; k < 2; ++k) {
        b.f[k] = (T*)c->f[k];
        b.q[k] = (T*)c->q[k];
    }
    b.h = (T*)c->h;
    b.sigma = (T*)c->sigma;
    b.u = (T*)c->u;
    return b;
}
inline LcGeom lc_geom(const lc_ctx* c) { return LcGeom{c->nx, c->ny, c->nz, c->n, c->npad}; }

template <class T>
cudaError_t lc_init_t(lc_ctx* c, const double* q, const double* rho, const double* u) {
    const LcBufs<T> b = lc_bufs<T>(c);
    k_lc_init<T><<<lc_blocks(c->n), kLcThreads, 0, c->stream>>>(lc_geom(c), c->prm.rho0, q, rho, u, b.f[0], b.q[0]);
    return cudaGetLastError();
}

template <class T, class I>
cudaError_t launch_lc_fused(lc_ctx* c, const LcGeom& g, const LcModel<T>& m, const LcBufs<T>& b) {
    constexpr bool kStage = kLcStageF;
    constexpr int smem = (int)lc_fused_smem<T, kStage>();
    const cudaError_t e = ld::set_max_dynamic_smem_once<k_lc_fused<T, I, kStage>>(smem);
    if (e != cudaSuccess) return e;
    const int nchunks = lc_choose_chunks(g.nx, g.ny, g.nz, c->num_sms, lc_fused_ctas<T, kStage>());
    const dim3 grid(g.nx / kLcTX, g.ny / kLcTY, nchunks);
    k_lc_fused<T, I, kStage><<<grid, kLcFusedThreads, smem, c->stream>>>(g, m, nchunks, b.q[c->cur], b.f[c->cur],
                                                                         b.f[1 - c->cur], b.u);
    return cudaGetLastError();
}

template <class T>
cudaError_t lc_step_t(lc_ctx* c) {
    const LcBufs<T> b = lc_bufs<T>(c);
    const LcGeom g = lc_geom(c);
    const LcModel<T> m = lc_model_of<T>(c->prm);
    const unsigned nb = lc_blocks(c->n);
    const int cur = c->cur;
    if (c->kernel == LD_KERNEL_FUSED) {
        const cudaError_t e = (long long)Q * c->npad <= 0x7fffffffLL ? launch_lc_fused<T, int>(c, g, m, b)
                                                                     : launch_lc_fused<T, long long>(c, g, m, b);
        if (e != cudaSuccess) return e;
        k_lc_update<T, true><<<nb, kLcThreads, 0, c->stream>>>(g, m, b.q[cur], b.u, nullptr, b.q[1 - cur]);
        return cudaGetLastError();
    }
    k_lc_field<T><<<nb, kLcThreads, 0, c->stream>>>(g, m, b.q[cur], b.h, b.sigma);
    k_lc_collide<T><<<nb, kLcThreads, 0, c->stream>>>(g, m, b.sigma, b.f[cur], b.f[1 - cur], b.u);
    k_lc_update<T, false><<<nb, kLcThreads, 0, c->stream>>>(g, m, b.q[cur], b.u, b.h, b.q[1 - cur]);
    return cudaGetLastError();
}

template <class T>
cudaError_t lc_out_t(lc_ctx* c, double* q, double* rho, double* u, double* h, double* f) {
    const LcBufs<T> b = lc_bufs<T>(c);
    const LcGeom g = lc_geom(c);
    const unsigned nb = lc_blocks(c->n);
    if (rho || u || h) k_lc_field<T><<<nb, kLcThreads, 0, c->stream>>>(g, lc_model_of<T>(c->prm), b.q[c->cur], b.h, b.sigma);
    k_lc_out<T><<<nb, kLcThreads, 0, c->stream>>>(g, b.q[c->cur], b.f[c->cur], b.sigma, b.h, q, rho, u, h, f);
    return cudaGetLastError();
}

}  // namespace
}  // namespace lc
