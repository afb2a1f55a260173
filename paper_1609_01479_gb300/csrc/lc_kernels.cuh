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

template <class T>
__global__ void __launch_bounds__(kLcThreads) k_lc_field(LcGeom g, LcModel<T> m, const T* __restrict__ q,
                                                         T* __restrict__ h, T* __restrict__ sigma) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int x, y, z;
    if (!lc_coords(g, s, x, y, z)) return;
    T Qc[3][3], dQ[3][3][3], lapQ[3][3];
    lc_full(q, g.npad, s, Qc);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) lapQ[a][b] = T(-6) * Qc[a][b];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        T Qp[3][3], Qm[3][3];
        lc_full(q, g.npad, lc_site(g, x + (c == 0), y + (c == 1), z + (c == 2)), Qp);
        lc_full(q, g.npad, lc_site(g, x - (c == 0), y - (c == 1), z - (c == 2)), Qm);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                dQ[c][a][b] = T(0.5) * (Qp[a][b] - Qm[a][b]);
                lapQ[a][b] += Qp[a][b] + Qm[a][b];
            }
    }
    // molecular field
    T tr2 = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) tr2 += Qc[a][b] * Qc[a][b];
    T H[3][3];
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
    // free energy density
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
    // stress
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
            T sg = fe * dab;
            T grad = T(0);
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int d = 0; d < 3; ++d) grad += dQ[a][c][d] * dQ[b][c][d];
            sg -= m.kappa * grad;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const T dcb = c == b ? T(1) : T(0), dac = a == c ? T(1) : T(0);
                sg -= m.xi * H[a][c] * (Qc[c][b] + dcb / T(3));
                sg -= m.xi * (Qc[a][c] + dac / T(3)) * H[c][b];
                sg += Qc[a][c] * H[c][b] - H[a][c] * Qc[c][b];
            }
            sg += T(2) * m.xi * (Qc[a][b] + dab / T(3)) * qh;
            sigma[(3 * a + b) * g.npad + s] = sg;
        }
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
    T fv[Q];
    T rho = T(0), j[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        fv[i] = f[i * g.npad + s];
        rho += fv[i];
        j[0] += T(cx(i)) * fv[i];
        j[1] += T(cy(i)) * fv[i];
        j[2] += T(cz(i)) * fv[i];
    }
    T uv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        uv[a] = (j[a] + T(0.5) * Fa[a]) / rho;
        u[a * g.npad + s] = uv[a];
    }
    const T uu = uv[0] * uv[0] + uv[1] * uv[1] + uv[2] * uv[2];
    const T uF = uv[0] * Fa[0] + uv[1] * Fa[1] + uv[2] * Fa[2];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T cu = T(cx(i)) * uv[0] + T(cy(i)) * uv[1] + T(cz(i)) * uv[2];
        const T cF = T(cx(i)) * Fa[0] + T(cy(i)) * Fa[1] + T(cz(i)) * Fa[2];
        const T feq = wgt<T>(i) * rho * (T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu);
        const T src = m.pre * wgt<T>(i) * (T(3) * (cF - uF) + T(9) * cu * cF);
        fd[i * g.npad + lc_site(g, x + cx(i), y + cy(i), z + cz(i))] = fv[i] - m.omega * (fv[i] - feq) + src;
    }
}

template <class T>
__global__ void __launch_bounds__(kLcThreads) k_lc_update(LcGeom g, LcModel<T> m, const T* __restrict__ q,
                                                          const T* __restrict__ u, const T* __restrict__ h,
                                                          T* __restrict__ qn) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int x, y, z;
    if (!lc_coords(g, s, x, y, z)) return;
    T W[3][3], Qc[3][3];
    T us[3];
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
    // co-rotation S(W, Q)
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
        const T qc = q[k * g.npad + s];
        T adv = T(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const bool fwd = us[c] >= T(0);
            const long long up = fwd ? lc_site(g, x - (c == 0), y - (c == 1), z - (c == 2))
                                     : lc_site(g, x + (c == 0), y + (c == 1), z + (c == 2));
            const T diff = fwd ? qc - q[k * g.npad + up] : q[k * g.npad + up] - qc;
            adv += us[c] * diff;
        }
        qn[k * g.npad + s] = qc + m.Gamma * h[k * g.npad + s] + S - adv;
    }
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

template <class T>
cudaError_t lc_step_t(lc_ctx* c) {
    const LcBufs<T> b = lc_bufs<T>(c);
    const LcGeom g = lc_geom(c);
    const LcModel<T> m = lc_model_of<T>(c->prm);
    const unsigned nb = lc_blocks(c->n);
    const int cur = c->cur;
    k_lc_field<T><<<nb, kLcThreads, 0, c->stream>>>(g, m, b.q[cur], b.h, b.sigma);
    k_lc_collide<T><<<nb, kLcThreads, 0, c->stream>>>(g, m, b.sigma, b.f[cur], b.f[1 - cur], b.u);
    k_lc_update<T><<<nb, kLcThreads, 0, c->stream>>>(g, m, b.q[cur], b.u, b.h, b.q[1 - cur]);
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
