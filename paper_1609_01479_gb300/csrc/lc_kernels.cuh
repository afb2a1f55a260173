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
// Three launches per step, one thread per site in site order:
//   k_lc_field    Q (+ its six neighbours) -> H (5 values), sigma (9)
//   k_lc_collide  sigma (+ neighbours), f -> F, u (3 values stored), f collided
//                 and pushed into the other buffer
//   k_lc_update   Q, H, u (+ neighbours) -> Q of the next step (other buffer)
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

template <class T>
struct LcModel {
    T A0, gamma, kappa, Gamma, xi, omega, pre;
};
template <class T>
LcModel<T> lc_model_of(const lc_params& p) {
    return LcModel<T>{(T)p.A0, (T)p.gamma, (T)p.kappa, (T)p.Gamma, (T)p.xi, (T)(1.0 / p.tau_f),
                      (T)(1.0 - 0.5 / p.tau_f)};
}

struct LcGeom {
    int nx, ny, nz;
    long long n, npad;
};

__device__ __forceinline__ long long lc_site(const LcGeom& g, int x, int y, int z) {
    x = x < 0 ? x + g.nx : (x >= g.nx ? x - g.nx : x);
    y = y < 0 ? y + g.ny : (y >= g.ny ? y - g.ny : y);
    z = z < 0 ? z + g.nz : (z >= g.nz ? z - g.nz : z);
    return (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * z);
}
__device__ __forceinline__ bool lc_coords(const LcGeom& g, long long s, int& x, int& y, int& z) {
    if (s >= g.n) return false;
    x = (int)(s % g.nx);
    const long long t = s / g.nx;
    y = (int)(t % g.ny);
    z = (int)(t / g.ny);
    return true;
}

// The full tensor of site s from its five stored components.
template <class T>
__device__ __forceinline__ void lc_full(const T* q, long long npad, long long s, T (&M)[3][3]) {
    const T xx = q[s], xy = q[npad + s], xz = q[2 * npad + s], yy = q[3 * npad + s], yz = q[4 * npad + s];
    M[0][0] = xx;
    M[0][1] = xy;
    M[0][2] = xz;
    M[1][0] = xy;
    M[1][1] = yy;
    M[1][2] = yz;
    M[2][0] = xz;
    M[2][1] = yz;
    M[2][2] = -xx - yy;
}

__device__ __forceinline__ int comp_a(int k) { return k < 3 ? 0 : 1; }
__device__ __forceinline__ int comp_b(int k) { return k < 3 ? k : k - 2; }

// Central-difference gradient and 7-point Laplacian of Q at a site. nb(c,
// sgn, M) fills M with the full tensor of the neighbour at sgn * e_c.
template <class T, class Nb>
__device__ __forceinline__ void lc_grad_lap(const T (&Qc)[3][3], Nb nb, T (&dQ)[3][3][3], T (&lapQ)[3][3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) lapQ[a][b] = T(-6) * Qc[a][b];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        T Qp[3][3], Qm[3][3];
        nb(c, 1, Qp);
        nb(c, -1, Qm);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                dQ[c][a][b] = T(0.5) * (Qp[a][b] - Qm[a][b]);
                lapQ[a][b] += Qp[a][b] + Qm[a][b];
            }
    }
}

// Molecular field H = -dF/dQ (traceless part) of the Landau-de Gennes free
// energy with one elastic constant; tr2 = Q:Q is returned for the stress.
template <class T>
__device__ __forceinline__ void lc_molecular_field(const T (&Qc)[3][3], const T (&lapQ)[3][3], const LcModel<T>& m,
                                                   T& tr2, T (&H)[3][3]) {
    tr2 = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) tr2 += Qc[a][b] * Qc[a][b];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            T qq = T(0);
#pragma unroll
            for (int c = 0; c < 3; ++c) qq += Qc[a][c] * Qc[c][b];
            const T delta = a == b ? T(1) : T(0);
            H[a][b] = -m.A0 * (T(1) - m.gamma / T(3)) * Qc[a][b] + m.A0 * m.gamma * (qq - delta * tr2 / T(3)) -
                      m.A0 * m.gamma * tr2 * Qc[a][b] + m.kappa * lapQ[a][b];
        }
}

// Chemical stress sigma_ab of a site: the free energy density on the
// diagonal, the elastic (gradient) term, and the flow-aligning and
// antisymmetric terms of H.
template <class T>
__device__ __forceinline__ void lc_stress(const T (&Qc)[3][3], const T (&dQ)[3][3][3], const T (&H)[3][3], T tr2,
                                          const LcModel<T>& m, T (&sg)[3][3]) {
    T tr3 = T(0), grad2 = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) tr3 += Qc[a][b] * Qc[b][c] * Qc[c][a];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) grad2 += dQ[c][a][b] * dQ[c][a][b];
    const T fe = T(0.5) * m.A0 * (T(1) - m.gamma / T(3)) * tr2 - m.A0 * m.gamma / T(3) * tr3 +
                 T(0.25) * m.A0 * m.gamma * tr2 * tr2 + T(0.5) * m.kappa * grad2;
    T qh = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) qh += Qc[a][b] * H[a][b];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const T dab = a == b ? T(1) : T(0);
            T s = fe * dab;
            T grad = T(0);
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int d = 0; d < 3; ++d) grad += dQ[a][c][d] * dQ[b][c][d];
            s -= m.kappa * grad;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const T dcb = c == b ? T(1) : T(0), dac = a == c ? T(1) : T(0);
                s -= m.xi * H[a][c] * (Qc[c][b] + dcb / T(3));
                s -= m.xi * (Qc[a][c] + dac / T(3)) * H[c][b];
                s += Qc[a][c] * H[c][b] - H[a][c] * Qc[c][b];
            }
            s += T(2) * m.xi * (Qc[a][b] + dab / T(3)) * qh;
            sg[a][b] = s;
        }
}

// Velocity u = (j + F/2)/rho and the BGK + Guo collision of one site's f
// (in place); u is returned in uv.
template <class T>
__device__ __forceinline__ void lc_collide_site(T (&fv)[Q], const T (&Fa)[3], const LcModel<T>& m, T (&uv)[3]) {
    T rho = T(0), j[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        rho += fv[i];
        j[0] += T(cx(i)) * fv[i];
        j[1] += T(cy(i)) * fv[i];
        j[2] += T(cz(i)) * fv[i];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) uv[a] = (j[a] + T(0.5) * Fa[a]) / rho;
    const T uu = uv[0] * uv[0] + uv[1] * uv[1] + uv[2] * uv[2];
    const T uF = uv[0] * Fa[0] + uv[1] * Fa[1] + uv[2] * Fa[2];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T cu = T(cx(i)) * uv[0] + T(cy(i)) * uv[1] + T(cz(i)) * uv[2];
        const T cF = T(cx(i)) * Fa[0] + T(cy(i)) * Fa[1] + T(cz(i)) * Fa[2];
        const T feq = wgt<T>(i) * rho * (T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu);
        const T src = m.pre * wgt<T>(i) * (T(3) * (cF - uF) + T(9) * cu * cF);
        fv[i] = fv[i] - m.omega * (fv[i] - feq) + src;
    }
}

// The Q update of one site: Q + Gamma H + S(W, Q) - u.grad(Q), the
// advection first-order upwind. qk(k) is component k of Q at the site,
// qnb(k, c, sgn) at its neighbour sgn * e_c; W from the central difference
// of u.
template <class T, class Qk, class QNb>
__device__ __forceinline__ void lc_update_site(const T (&Qc)[3][3], const T (&H)[3][3], const T (&us)[3],
                                               const T (&W)[3][3], const LcModel<T>& m, Qk qk, QNb qnb, T (&qn)[5]) {
    T D[3][3], Om[3][3], Qp[3][3];
    T trQW = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            D[a][b] = T(0.5) * (W[a][b] + W[b][a]);
            Om[a][b] = T(0.5) * (W[a][b] - W[b][a]);
            Qp[a][b] = Qc[a][b] + (a == b ? T(1) / T(3) : T(0));
            trQW += Qc[a][b] * W[b][a];
        }
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int a = comp_a(k), b = comp_b(k);
        T S = T(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) S += (m.xi * D[a][c] + Om[a][c]) * Qp[c][b] + Qp[a][c] * (m.xi * D[c][b] - Om[c][b]);
        S = S - T(2) * m.xi * Qp[a][b] * trQW;
        const T qc = qk(k);
        T adv = T(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const bool fwd = us[c] >= T(0);
            const T diff = fwd ? qc - qnb(k, c, -1) : qnb(k, c, 1) - qc;
            adv += us[c] * diff;
        }
        qn[k] = qc + m.Gamma * H[a][b] + S - adv;
    }
}

template <class T>
__global__ void __launch_bounds__(kLcThreads) k_lc_field(LcGeom g, LcModel<T> m, const T* __restrict__ q,
                                                         T* __restrict__ h, T* __restrict__ sigma) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int x, y, z;
    if (!lc_coords(g, s, x, y, z)) return;
    T Qc[3][3], dQ[3][3][3], lapQ[3][3], H[3][3], sg[3][3], tr2;
    lc_full(q, g.npad, s, Qc);
    lc_grad_lap(Qc, [&](int c, int sgn, T (&M)[3][3]) {
        lc_full(q, g.npad, lc_site(g, x + sgn * (c == 0), y + sgn * (c == 1), z + sgn * (c == 2)), M);
    }, dQ, lapQ);
    lc_molecular_field(Qc, lapQ, m, tr2, H);
    lc_stress(Qc, dQ, H, tr2, m, sg);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) sigma[(3 * a + b) * g.npad + s] = sg[a][b];
#pragma unroll
    for (int k = 0; k < 5; ++k) h[k * g.npad + s] = H[comp_a(k)][comp_b(k)];
}

template <class T>
__global__ void __launch_bounds__(kLcThreads) k_lc_collide(LcGeom g, LcModel<T> m, const T* __restrict__ sigma,
                                                           const T* __restrict__ f, T* __restrict__ fd,
                                                           T* __restrict__ u) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int x, y, z;
    if (!lc_coords(g, s, x, y, z)) return;
    T Fa[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const long long sp = lc_site(g, x + (b == 0), y + (b == 1), z + (b == 2));
        const long long sm = lc_site(g, x - (b == 0), y - (b == 1), z - (b == 2));
#pragma unroll
        for (int a = 0; a < 3; ++a) Fa[a] += T(0.5) * (sigma[(3 * a + b) * g.npad + sp] - sigma[(3 * a + b) * g.npad + sm]);
    }
    T fv[Q], uv[3];
#pragma unroll
    for (int i = 0; i < Q; ++i) fv[i] = f[i * g.npad + s];
    lc_collide_site(fv, Fa, m, uv);
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a * g.npad + s] = uv[a];
#pragma unroll
    for (int i = 0; i < Q; ++i) fd[i * g.npad + lc_site(g, x + cx(i), y + cy(i), z + cz(i))] = fv[i];
}

// RECOMPUTE_H: form H from Q here (the fused step stores no H) instead of
// reading the h written by k_lc_field; the same arithmetic either way.
template <class T, bool RECOMPUTE_H>
__global__ void __launch_bounds__(kLcThreads) k_lc_update(LcGeom g, LcModel<T> m, const T* __restrict__ q,
                                                          const T* __restrict__ u, const T* __restrict__ h,
                                                          T* __restrict__ qn) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int x, y, z;
    if (!lc_coords(g, s, x, y, z)) return;
    T W[3][3], Qc[3][3], H[3][3], us[3], qv[5];
#pragma unroll
    for (int a = 0; a < 3; ++a) us[a] = u[a * g.npad + s];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const long long sp = lc_site(g, x + (b == 0), y + (b == 1), z + (b == 2));
        const long long sm = lc_site(g, x - (b == 0), y - (b == 1), z - (b == 2));
#pragma unroll
        for (int a = 0; a < 3; ++a) W[a][b] = T(0.5) * (u[a * g.npad + sp] - u[a * g.npad + sm]);
    }
    lc_full(q, g.npad, s, Qc);
    auto nb_site = [&](int c, int sgn) {
        return lc_site(g, x + sgn * (c == 0), y + sgn * (c == 1), z + sgn * (c == 2));
    };
    if constexpr (RECOMPUTE_H) {
        T dQ[3][3][3], lapQ[3][3], tr2;
        lc_grad_lap(Qc, [&](int c, int sgn, T (&M)[3][3]) { lc_full(q, g.npad, nb_site(c, sgn), M); }, dQ, lapQ);
        lc_molecular_field(Qc, lapQ, m, tr2, H);
    } else {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const T v = h[k * g.npad + s];
            H[comp_a(k)][comp_b(k)] = v;
            H[comp_b(k)][comp_a(k)] = v;
        }
    }
    lc_update_site(
        Qc, H, us, W, m, [&](int k) { return q[k * g.npad + s]; },
        [&](int k, int c, int sgn) { return q[k * g.npad + nb_site(c, sgn)]; }, qv);
#pragma unroll
    for (int k = 0; k < 5; ++k) qn[k * g.npad + s] = qv[k];
}

// ---------------------------------------------------------------------------
// Fused field + collision step. Each CTA owns a kLcTX x kLcTY column of sites
// and marches up a chunk of zc z-planes. The stress chain Q -> (H, sigma) ->
// F = div sigma needs sigma within one site and so Q within two sites of every
// collided site: the CTA keeps two rolling rings in shared memory,
//   Q ring:     3 planes x 5 components over the tile + 2-site halo,
//   sigma ring: 3 planes x 9 components over the tile + 1-site halo (corners
//               unused and not computed).
// Iteration k loads Q of plane k+2, forms H and sigma of plane k+1, then
// reads f of plane k, forms F, u, collides and pushes f, and stores u (which
// the Q update, k_lc_update, reads with its neighbours). Per site the launch
// reads Q once from HBM (halo re-reads hit L2) and f once, and writes f and u;
// H and sigma never leave shared memory. The arithmetic of every site is the
// per-site kernels' (lc_grad_lap, lc_molecular_field, lc_stress,
// lc_collide_site), in the same order.
constexpr int kLcTX = 32, kLcTY = 8, kLcFusedThreads = kLcTX * kLcTY;
constexpr int kLcQW = kLcTX + 4, kLcQH = kLcTY + 4;  // Q ring plane
constexpr int kLcSW = kLcTX + 2, kLcSH = kLcTY + 2;  // sigma ring plane

// Resident CTAs per SM: the shared-memory rings (62.6 KB in FP32, 125 KB in
// FP64) allow three FP32 CTAs, one FP64 CTA.
template <class T>
constexpr int lc_fused_ctas() {
    return sizeof(T) == 4 ? 3 : 1;
}
template <class T>
constexpr size_t lc_fused_smem() {
    return (size_t)(3 * 5 * kLcQH * kLcQW + 3 * 9 * kLcSH * kLcSW) * sizeof(T);
}

template <class T>
struct LcPair;
template <>
struct LcPair<float> {
    using type = float2;
};
template <>
struct LcPair<double> {
    using type = double2;
};

__device__ __forceinline__ int lc_wrap(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// I: type of the element offsets i * npad + s (32-bit where 19 npad fits).
template <class T, class I>
__global__ void __launch_bounds__(kLcFusedThreads, lc_fused_ctas<T>())
    k_lc_fused(LcGeom g, LcModel<T> m, int zc, const T* __restrict__ q, const T* __restrict__ f,
               T* __restrict__ fd, T* __restrict__ u) {
    using T2 = typename LcPair<T>::type;
    extern __shared__ __align__(16) unsigned char lc_smem[];
    T* qring = reinterpret_cast<T*>(lc_smem);   // [3][5][kLcQH][kLcQW]
    T* sring = qring + 3 * 5 * kLcQH * kLcQW;    // [3][9][kLcSH][kLcSW]
    auto QR = [&](int slot, int k, int py, int px) -> T& { return qring[((slot * 5 + k) * kLcQH + py) * kLcQW + px]; };
    auto SR = [&](int slot, int k, int hy, int hx) -> T& { return sring[((slot * 9 + k) * kLcSH + hy) * kLcSW + hx]; };

    const int tid = threadIdx.x;
    const int tx = tid % kLcTX, ty = tid / kLcTX;
    const int x0 = blockIdx.x * kLcTX, y0 = blockIdx.y * kLcTY, z0 = blockIdx.z * zc;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int plane = nx * ny;
    const I npad = (I)g.npad;

    // Q of plane zp over the tile + 2-halo into ring slot `slot`: two
    // x-adjacent sites per paired load (the halo starts at an even x and nx is
    // even, so a pair never straddles the periodic wrap).
    auto q_plane = [&](int zp, int slot) {
        constexpr int QW2 = kLcQW / 2;
        const int zoff = lc_wrap(zp, nz) * plane;
        for (int idx = tid; idx < QW2 * kLcQH; idx += kLcFusedThreads) {
            const int px = 2 * (idx % QW2), py = idx / QW2;
            const int s = zoff + lc_wrap(y0 + py - 2, ny) * nx + lc_wrap(x0 + px - 2, nx);
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const T2 v = __ldg(reinterpret_cast<const T2*>(q + k * npad + s));
                QR(slot, k, py, px) = v.x;
                QR(slot, k, py, px + 1) = v.y;
            }
        }
    };
    auto full_at = [&](int slot, int py, int px, T (&M)[3][3]) {
        const T xx = QR(slot, 0, py, px), xy = QR(slot, 1, py, px), xz = QR(slot, 2, py, px);
        const T yy = QR(slot, 3, py, px), yz = QR(slot, 4, py, px);
        M[0][0] = xx;
        M[0][1] = xy;
        M[0][2] = xz;
        M[1][0] = xy;
        M[1][1] = yy;
        M[1][2] = yz;
        M[2][0] = xz;
        M[2][1] = yz;
        M[2][2] = -xx - yy;
    };
    // sigma of the plane whose Q is in slot `mid` (below: lo, above: hi) over
    // the tile + 1-halo, into sigma slot `slot`.
    auto sigma_plane = [&](int lo, int mid, int hi, int slot) {
        for (int idx = tid; idx < kLcSW * kLcSH; idx += kLcFusedThreads) {
            const int hx = idx % kLcSW, hy = idx / kLcSW;
            if ((hx == 0 || hx == kLcSW - 1) && (hy == 0 || hy == kLcSH - 1)) continue;
            const int px = hx + 1, py = hy + 1;
            T Qc[3][3], dQ[3][3][3], lapQ[3][3], H[3][3], sg[3][3], tr2;
            full_at(mid, py, px, Qc);
            lc_grad_lap(Qc, [&](int c, int sgn, T (&M)[3][3]) {
                full_at(c == 2 ? (sgn > 0 ? hi : lo) : mid, py + sgn * (c == 1), px + sgn * (c == 0), M);
            }, dQ, lapQ);
            lc_molecular_field(Qc, lapQ, m, tr2, H);
            lc_stress(Qc, dQ, H, tr2, m, sg);
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) SR(slot, 3 * a + b, hy, hx) = sg[a][b];
        }
    };
    auto qs = [&](int zp) { return (zp - z0 + 2) % 3; };  // Q slot of plane zp (zp >= z0-2)
    auto ss = [&](int zp) { return (zp - z0 + 1) % 3; };  // sigma slot of plane zp (zp >= z0-1)

    // Prologue: Q(z0-2..z0+1), sigma(z0-1), sigma(z0).
    q_plane(z0 - 2, qs(z0 - 2));
    q_plane(z0 - 1, qs(z0 - 1));
    q_plane(z0, qs(z0));
    __syncthreads();
    sigma_plane(qs(z0 - 2), qs(z0 - 1), qs(z0), ss(z0 - 1));
    __syncthreads();  // Q(z0+1) takes the slot of Q(z0-2)
    q_plane(z0 + 1, qs(z0 + 1));
    __syncthreads();
    sigma_plane(qs(z0 - 1), qs(z0), qs(z0 + 1), ss(z0));

    const int x = x0 + tx, y = y0 + ty;
    const int oxp = x + 1 == nx ? 1 - nx : 1, oxm = x == 0 ? nx - 1 : -1;
    const int oyp = y + 1 == ny ? (1 - ny) * nx : nx, oym = y == 0 ? (ny - 1) * nx : -nx;

    for (int k = z0; k < z0 + zc; ++k) {
        __syncthreads();  // the last collision is done with sigma(k-2), the last sigma pass with Q(k-1)
        q_plane(k + 2, qs(k + 2));
        __syncthreads();
        sigma_plane(qs(k), qs(k + 1), qs(k + 2), ss(k + 1));
        __syncthreads();

        const int s = k * plane + y * nx + x;  // zc divides nz: k < nz
        T Fa[3] = {T(0), T(0), T(0)};
        const int sc = ss(k), sp = ss(k + 1), sm = ss(k - 1);
#pragma unroll
        for (int a = 0; a < 3; ++a) Fa[a] += T(0.5) * (SR(sc, 3 * a, ty + 1, tx + 2) - SR(sc, 3 * a, ty + 1, tx));
#pragma unroll
        for (int a = 0; a < 3; ++a) Fa[a] += T(0.5) * (SR(sc, 3 * a + 1, ty + 2, tx + 1) - SR(sc, 3 * a + 1, ty, tx + 1));
#pragma unroll
        for (int a = 0; a < 3; ++a) Fa[a] += T(0.5) * (SR(sp, 3 * a + 2, ty + 1, tx + 1) - SR(sm, 3 * a + 2, ty + 1, tx + 1));
        T fv[Q], uv[3];
#pragma unroll
        for (int i = 0; i < Q; ++i) fv[i] = __ldcs(f + i * npad + s);
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
}

// Planes per CTA: the divisor of nz among 64..1 that minimises waves x
// (planes + 2), each CTA paying about two planes of prologue.
inline int lc_choose_zc(int nx, int ny, int nz, int num_sms, int per_sm) {
    const long long cols = (long long)(nx / kLcTX) * (ny / kLcTY);
    const long long slots = (long long)per_sm * num_sms;
    int best = 0;
    long long best_cost = 0;
    for (int zc = 64; zc >= 1; zc /= 2) {
        if (nz % zc) continue;
        const long long cost = ((cols * (nz / zc) + slots - 1) / slots) * (zc + 2);
        if (best == 0 || cost < best_cost) {
            best = zc;
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
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int x, y, z;
    if (!lc_coords(g, s, x, y, z)) return;
    if (qo)
        for (int k = 0; k < 5; ++k) qo[k * g.n + s] = (double)q[k * g.npad + s];
    if (ho)
        for (int k = 0; k < 5; ++k) ho[k * g.n + s] = (double)h[k * g.npad + s];
    if (fo)
        for (int i = 0; i < Q; ++i) fo[i * g.n + s] = (double)f[i * g.npad + s];
    if (rho || uo) {
        T Fa[3] = {T(0), T(0), T(0)};
        for (int b = 0; b < 3; ++b) {
            const long long sp = lc_site(g, x + (b == 0), y + (b == 1), z + (b == 2));
            const long long sm = lc_site(g, x - (b == 0), y - (b == 1), z - (b == 2));
            for (int a = 0; a < 3; ++a)
                Fa[a] += T(0.5) * (sigma[(3 * a + b) * g.npad + sp] - sigma[(3 * a + b) * g.npad + sm]);
        }
        T r = T(0), j[3] = {T(0), T(0), T(0)};
        for (int i = 0; i < Q; ++i) {
            const T fi = f[i * g.npad + s];
            r += fi;
            j[0] += T(cx(i)) * fi;
            j[1] += T(cy(i)) * fi;
            j[2] += T(cz(i)) * fi;
        }
        if (rho) rho[s] = (double)r;
        if (uo)
            for (int a = 0; a < 3; ++a) uo[a * g.n + s] = (double)((j[a] + T(0.5) * Fa[a]) / r);
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
    constexpr int smem = (int)lc_fused_smem<T>();
    const cudaError_t e = ld::set_max_dynamic_smem_once<k_lc_fused<T, I>>(smem);
    if (e != cudaSuccess) return e;
    const int zc = lc_choose_zc(g.nx, g.ny, g.nz, c->num_sms, lc_fused_ctas<T>());
    const dim3 grid(g.nx / kLcTX, g.ny / kLcTY, g.nz / zc);
    k_lc_fused<T, I><<<grid, kLcFusedThreads, smem, c->stream>>>(g, m, zc, b.q[c->cur], b.f[c->cur], b.f[1 - c->cur],
                                                                 b.u);
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
