// Adjoint (reverse mode) of one timestep, of the initialiser, and the
// parameter gradients d/dkappa and d/dtau_f; templates instantiated per
// storage precision. The adjoint state (fbar, gbar) is held in the arithmetic
// type: FP64 for FP64 contexts, FP32 otherwise.
//
// Forward step at site x (state f, g at time t; see ld_common.cuh):
//   rho = sum f, j = sum f c, phi = sum g
//   mu = A phi + B phi^3 - kappa lap(phi),   gm_a = (mu(x+e_a) - mu(x-e_a))/2
//   F = -phi gm,   u = (j + F/2)/rho
//   f*_i = (1-w_f) f_i + w_f feq_i(rho,u) + (1 - w_f/2) S_i(u,F),  w_f = 1/tau_f
//   g*_i = (1-w_g) g_i + w_g geq_i(phi,u,mu)
//   f_i(x + c_i, t+1) = f*_i(x),  g likewise.
// Reverse, given the adjoint of the state at t+1:
//   1. reverse propagation: f*bar_i(x) = fbar_i(x + c_i, t+1) (a pull), g alike;
//   2. at each site, the adjoint of both collisions and of u and F gives
//      rhobar, jbar, Fbar, the local parts of phibar and mubar, and gmbar;
//      fbar_i(x,t) = (1-w_f) f*bar_i + rhobar + c_i.jbar (purely local, since F
//      depends on phi only);
//   3. mubar(y) += sum_a (gmbar_a(y-e_a) - gmbar_a(y+e_a))/2   (transposed gradient);
//   4. phibar(y) += (A + 3B phi^2) mubar - kappa lap(mubar)    (lap is symmetric);
//      gbar_i(y,t) = (1-w_g) g*bar_i(y) + phibar(y).
// The adjoint g is kept factored as gbar_i = G_i + P with a per-site scalar
// P: step 2 writes G_i = (1-w_g) g*bar_i at the site it already owns, step 4
// writes only P = phibar, and the next step's pull adds P of the source
// site. This saves a full read and write pass over the 19 gbar values.
// Parameter sums (FP64, fixed order): kappabar += sum mubar (-lap phi);
// taubar_f = -(1/tau_f^2) sum_i,x f*bar_i (feq_i - f_i - S_i/2).
#pragma once
#include "ld_common.cuh"
#include "ld_generic.cuh"
#include "ld_internal.h"

namespace ld {
namespace {

constexpr int kAdjThreads = 256;

// Fixed-order block sum of one double per thread into out[0] (thread 0 writes).
__device__ __forceinline__ void block_sum_one(double v, double* out) {
    __shared__ double red[kAdjThreads / 32];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int w = 0; w < kAdjThreads / 32; ++w) a += red[w];
        *out = a;
    }
}

// Two resident 256-thread CTAs per SM for the local adjoint kernel: at three
// (80 registers) it spills and runs 16% slower.
template <int P>
constexpr int adj_ctas_per_sm() {
    return 2;
}

// Step 1 + 2: local adjoint at every site.
template <int P, bool ISO>
__global__ void __launch_bounds__(kAdjThreads, adj_ctas_per_sm<P>())
    k_adj_local(Geom g, Model<typename Prec<P>::real_t> m, const typename Prec<P>::store_t* __restrict__ tf,
                const typename Prec<P>::real_t* __restrict__ phi, const typename Prec<P>::real_t* __restrict__ mu,
                const float* __restrict__ ref, const typename Prec<P>::real_t* __restrict__ fb1,
                const typename Prec<P>::real_t* __restrict__ gb1, const typename Prec<P>::real_t* __restrict__ pb1,
                typename Prec<P>::real_t* __restrict__ fb0, typename Prec<P>::real_t* __restrict__ gb0,
                typename Prec<P>::real_t* __restrict__ gmb, typename Prec<P>::real_t* __restrict__ mub,
                typename Prec<P>::real_t* __restrict__ phib, double* __restrict__ part) {
    using R = typename Prec<P>::real_t;
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double omega_bar = 0.0;
    if (s < g.n) {
        typename Prec<P>::real_t omega_site = 0;
        int x, y, z;
        site_coords(g, s, x, y, z);
        const int xp = wrap_inc(x, g.nx), xm = wrap_dec(x, g.nx);
        const int yp = wrap_inc(y, g.ny), ym = wrap_dec(y, g.ny);
        const int zp = wrap_inc(z, g.nz), zm = wrap_dec(z, g.nz);
        // forward quantities
        const R ph = phi[s];
        R gmx, gmy, gmz;
        if constexpr (ISO) {
            auto nb = [&](int i) {
                return mu[site_of(g, step_coord(x, cx(i), g.nx), step_coord(y, cy(i), g.ny), step_coord(z, cz(i), g.nz))];
            };
            grad19(nb, gmx, gmy, gmz);
        } else {
            gmx = R(0.5) * (mu[site_of(g, xp, y, z)] - mu[site_of(g, xm, y, z)]);
            gmy = R(0.5) * (mu[site_of(g, x, yp, z)] - mu[site_of(g, x, ym, z)]);
            gmz = R(0.5) * (mu[site_of(g, x, y, zp)] - mu[site_of(g, x, y, zm)]);
        }
        const R Fx = -ph * gmx, Fy = -ph * gmy, Fz = -ph * gmz;
        // reverse propagation: the values pushed from x along c_i. They do
        // not depend on the forward moments, so they are loaded together with
        // the tape values and both sets of loads are in flight at once.
        R fbs[Q], gbs[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const long long o = site_of(g, step_coord(x, cx(i), g.nx), step_coord(y, cy(i), g.ny),
                                        step_coord(z, cz(i), g.nz));
            fbs[i] = fb1[i * g.npad + o];
            gbs[i] = gb1[i * g.npad + o] + pb1[o];
        }
        R f[Q];
        R rho = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            f[i] = Prec<P>::decode(tf[i * g.npad + s], ref[i]);
            rho += f[i];
            add_c(i, f[i], jx, jy, jz);
        }
        R ux, uy, uz;
        guo_velocity(rho, jx, jy, jz, Fx, Fy, Fz, ux, uy, uz);
        const R uu = ux * ux + uy * uy + uz * uz;
        const R uF = ux * Fx + uy * Fy + uz * Fz;

        // accumulators of the local adjoint
        R rhob = R(0);
        R ucx = R(0), ucy = R(0), ucz = R(0);  // sum of c_i x (scalar) terms of ubar
        R u_u = R(0), u_F = R(0);             // ubar += u_u u + u_F F
        R Fcx = R(0), Fcy = R(0), Fcz = R(0);  // sum of c_i x (scalar) terms of Fbar
        R F_u = R(0);                          // Fbar += F_u u
        R phib_l = R(0), mub_l = R(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            gb0[i * g.npad + s] = (R(1) - m.omega_g) * gbs[i];
            const R w = wgt<R>(i);
            const R cu = cdot(i, ux, uy, uz);
            const R cF = cdot(i, Fx, Fy, Fz);
            const R base = R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu;
            const R feq = w * rho * base;
            const R src = w * (R(3) * (cF - uF) + R(9) * cu * cF);
            // f collision: f* = (1-w_f) f + w_f feq + pre S
            omega_site += fbs[i] * (feq - f[i] - R(0.5) * src);
            const R feqb = m.omega_f * fbs[i];
            const R Sb = m.force_pre * fbs[i];
            rhob += feqb * w * base;
            const R tfe = feqb * w * rho;
            // g collision: g* = (1-w_g) g + w_g geq
            const R tg = m.omega_g * gbs[i] * w;
            phib_l += tg * (R(1) + R(3) * cu - R(1.5) * R(c2(i) - 1) + R(4.5) * cu * cu - R(1.5) * uu);
            mub_l += tg * R(4.5) * m.Gamma * R(c2(i) - 1);
            // d feq/du = w rho ((3 + 9cu) c - 3u); d S/du = w (9 cF c - 3F);
            // d geq/du = w phi ((3 + 9cu) c - 3u); d S/dF = w ((3 + 9cu) c - 3u)
            add_c(i, tfe * (R(3) + R(9) * cu) + Sb * w * R(9) * cF + tg * ph * (R(3) + R(9) * cu), ucx, ucy, ucz);
            u_u -= R(3) * (tfe + tg * ph);
            u_F -= R(3) * Sb * w;
            add_c(i, Sb * w * (R(3) + R(9) * cu), Fcx, Fcy, Fcz);
            F_u -= R(3) * Sb * w;
        }
        const R ubx = ucx + u_u * ux + u_F * Fx;
        const R uby = ucy + u_u * uy + u_F * Fy;
        const R ubz = ucz + u_u * uz + u_F * Fz;
        R Fbx = Fcx + F_u * ux, Fby = Fcy + F_u * uy, Fbz = Fcz + F_u * uz;
        // u = (j + F/2) / rho
        const R jbx = ubx / rho, jby = uby / rho, jbz = ubz / rho;
        Fbx += R(0.5) * jbx;
        Fby += R(0.5) * jby;
        Fbz += R(0.5) * jbz;
        rhob -= (ubx * ux + uby * uy + ubz * uz) / rho;
        // F = -phi gm
        phib_l -= Fbx * gmx + Fby * gmy + Fbz * gmz;
        gmb[s] = -ph * Fbx;
        gmb[g.npad + s] = -ph * Fby;
        gmb[2 * g.npad + s] = -ph * Fbz;
        mub[s] = mub_l;
        phib[s] = phib_l;
        omega_bar = (double)omega_site;
        // fbar at t: direct term + rho and j
#pragma unroll
        for (int i = 0; i < Q; ++i)
            fb0[i * g.npad + s] = (R(1) - m.omega_f) * fbs[i] + rhob + cdot(i, jbx, jby, jbz);
    }
    block_sum_one(omega_bar, part + 2 * (long long)blockIdx.x);
}

// Step 3: mubar += transpose of the gradient applied to gmbar; kappa
// partials mubar (-lap phi). 7-point: the transposed central difference;
// 19-point: mubar(y) += sum_i 3 w_i c_i . gmbar(y - c_i).
template <class R, bool ISO>
__global__ void __launch_bounds__(kAdjThreads)
    k_adj_mu(Geom g, const R* __restrict__ phi, const R* __restrict__ gmb, R* __restrict__ mub,
             double* __restrict__ part) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double kappa_bar = 0.0;
    if (s < g.n) {
        int x, y, z;
        site_coords(g, s, x, y, z);
        R t, lap;
        if constexpr (ISO) {
            t = mub[s];
            lap = R(0);
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const long long back = site_of(g, step_coord(x, -cx(i), g.nx), step_coord(y, -cy(i), g.ny),
                                               step_coord(z, -cz(i), g.nz));
                const long long fwd = site_of(g, step_coord(x, cx(i), g.nx), step_coord(y, cy(i), g.ny),
                                              step_coord(z, cz(i), g.nz));
                const R dot = cdot(i, gmb[back], gmb[g.npad + back], gmb[2 * g.npad + back]);
                t += grad19_coef<R>(i) * dot;
                lap += lap19_coef<R>(i) * (phi[fwd] - phi[s]);
            }
        } else {
            const long long sxm = site_of(g, wrap_dec(x, g.nx), y, z), sxp = site_of(g, wrap_inc(x, g.nx), y, z);
            const long long sym = site_of(g, x, wrap_dec(y, g.ny), z), syp = site_of(g, x, wrap_inc(y, g.ny), z);
            const long long szm = site_of(g, x, y, wrap_dec(z, g.nz)), szp = site_of(g, x, y, wrap_inc(z, g.nz));
            t = mub[s] + R(0.5) * (gmb[sxm] - gmb[sxp]) + R(0.5) * (gmb[g.npad + sym] - gmb[g.npad + syp]) +
                R(0.5) * (gmb[2 * g.npad + szm] - gmb[2 * g.npad + szp]);
            lap = phi[sxp] + phi[sxm] + phi[syp] + phi[sym] + phi[szp] + phi[szm] - R(6) * phi[s];
        }
        mub[s] = t;
        kappa_bar = -(double)t * (double)lap;
    }
    block_sum_one(kappa_bar, part + 2 * (long long)blockIdx.x + 1);
}

// Laplacian (7-point or 19-point, symmetric: its own transpose) of a field
// at site s = (x, y, z), in the type of the field.
template <bool ISO, class T>
__device__ __forceinline__ T lap_at(const Geom& g, const T* h, long long s, int x, int y, int z) {
    if constexpr (ISO) {
        T lap = T(0);
#pragma unroll
        for (int i = 1; i < Q; ++i)
            lap += lap19_coef<T>(i) *
                   (h[site_of(g, step_coord(x, cx(i), g.nx), step_coord(y, cy(i), g.ny), step_coord(z, cz(i), g.nz))] -
                    h[s]);
        return lap;
    }
    return h[site_of(g, wrap_inc(x, g.nx), y, z)] + h[site_of(g, wrap_dec(x, g.nx), y, z)] +
           h[site_of(g, x, wrap_inc(y, g.ny), z)] + h[site_of(g, x, wrap_dec(y, g.ny), z)] +
           h[site_of(g, x, y, wrap_inc(z, g.nz))] + h[site_of(g, x, y, wrap_dec(z, g.nz))] - T(6) * h[s];
}

// Step 4: phibar, the per-site part P of gbar at t.
template <class R, bool ISO>
__global__ void __launch_bounds__(kAdjThreads)
    k_adj_p(Geom g, Model<R> m, const R* __restrict__ phi, const R* __restrict__ mub, const R* __restrict__ phib,
            R* __restrict__ pb0) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.n) return;
    int x, y, z;
    site_coords(g, s, x, y, z);
    const R ph = phi[s];
    const R lapm = lap_at<ISO>(g, mub, s, x, y, z);
    pb0[s] = phib[s] + (m.A + R(3) * m.B * ph * ph) * mub[s] - m.kappa * lapm;
}

// grad[0] += sum_b part[2b+1] (kappa); grad[1] += taub_scale * sum_b part[2b]
// (tau_f); one block, fixed order.
__global__ void __launch_bounds__(kAdjThreads)
    k_adj_finalize(const double* __restrict__ part, long long nblk, double taub_scale, double* __restrict__ grad) {
    __shared__ double red[2][kAdjThreads / 32];
    double a = 0.0, b = 0.0;
    for (long long k = threadIdx.x; k < nblk; k += kAdjThreads) {
        a += part[2 * k + 1];
        b += part[2 * k];
    }
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        b += __shfl_down_sync(0xffffffffu, b, off);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][warp] = a;
        red[1][warp] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ka = 0.0, tb = 0.0;
        for (int w = 0; w < kAdjThreads / 32; ++w) {
            ka += red[0][w];
            tb += red[1][w];
        }
        grad[0] += ka;
        grad[1] += taub_scale * tb;
    }
}

// Seed: fbar = 0, gbar_i = phibar (the adjoint of phi_T = sum_i g_i), i.e.
// G = 0 and P = phibar.
template <class R>
__global__ void __launch_bounds__(kAdjThreads)
    k_adj_seed(Geom g, const double* __restrict__ phibar, R* __restrict__ fb, R* __restrict__ gb, R* __restrict__ pb) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.n) return;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        fb[i * g.npad + s] = R(0);
        gb[i * g.npad + s] = R(0);
    }
    pb[s] = (R)phibar[s];
}

// Initialiser adjoint, part 1: mubar(x) = sum_i gbar_i d geq_i / d mu, in
// the arithmetic type.
template <class R>
__global__ void __launch_bounds__(kAdjThreads)
    k_adj_init_mu(Geom g, R Gamma, const R* __restrict__ gb, const R* __restrict__ pb, R* __restrict__ mub) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.n) return;
    R acc = R(0);
    const R p = pb[s];
#pragma unroll
    for (int i = 0; i < Q; ++i) acc += (gb[i * g.npad + s] + p) * (wgt<R>(i) * R(4.5) * R(c2(i) - 1));
    mub[s] = Gamma * acc;
}

// Initialiser adjoint, part 2: dL/dphi0 and the kappa partials
// (g = geq(phi0, u0, mu(phi0)); f does not depend on phi0, kappa or tau_f).
// Per-site sums in the arithmetic type; outputs and partials in FP64.
template <class R, bool ISO>
__global__ void __launch_bounds__(kAdjThreads)
    k_adj_init_phi(Geom g, Model<R> m, const double* __restrict__ phi0, const double* __restrict__ u0,
                   const R* __restrict__ gb, const R* __restrict__ pb, const R* __restrict__ mub,
                   double* __restrict__ grad_phi0, double* __restrict__ part) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double kappa_bar = 0.0;
    if (s < g.n) {
        int x, y, z;
        site_coords(g, s, x, y, z);
        R ux = R(0), uy = R(0), uz = R(0);
        if (u0) {
            ux = (R)u0[s];
            uy = (R)u0[g.n + s];
            uz = (R)u0[2 * g.n + s];
        }
        const R uu = ux * ux + uy * uy + uz * uz;
        const R p = pb[s];
        R acc = R(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const R cu = cdot(i, ux, uy, uz);
            acc += (gb[i * g.npad + s] + p) * wgt<R>(i) *
                   (R(1) + R(3) * cu - R(1.5) * R(c2(i) - 1) + R(4.5) * cu * cu - R(1.5) * uu);
        }
        const R ph = (R)phi0[s];
        const R mb = mub[s];
        const R lapm = lap_at<ISO>(g, mub, s, x, y, z);
        grad_phi0[s] = (double)(acc + (m.A + R(3) * m.B * ph * ph) * mb - m.kappa * lapm);
        const double lap = lap_at<ISO>(g, phi0, s, x, y, z);
        kappa_bar = -(double)mb * lap;
    }
    if (threadIdx.x == 0) part[2 * (long long)blockIdx.x] = 0.0;  // no tau_f term in the initialiser
    block_sum_one(kappa_bar, part + 2 * (long long)blockIdx.x + 1);
}

// Adjoint state I/O as double[19][n]. For the g part `pb` is the per-site
// term: read adds it; write stores the values in G and clears it.
template <class R>
__global__ void __launch_bounds__(kAdjThreads)
    k_adj_io(Geom g, int to_double, R* __restrict__ a, R* __restrict__ pb, double* __restrict__ d) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.n) return;
    const R add = (pb && to_double) ? pb[s] : R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (to_double)
            d[i * g.n + s] = (double)(a[i * g.npad + s] + add);
        else
            a[i * g.npad + s] = (R)d[i * g.n + s];
    }
    if (pb && !to_double) pb[s] = R(0);
}

// ---------------------------------------------------------------------------
template <int P>
struct AdjPtrs {
    using R = typename Prec<P>::real_t;
    R *fb1, *gb1, *pb1, *fb0, *gb0, *pb0, *gmb, *mub, *phib;
};

template <int P>
AdjPtrs<P> adj_ptrs(ld_ctx* c, int in_buf) {
    using R = typename Prec<P>::real_t;
    AdjPtrs<P> p;
    const size_t comp = (size_t)Q * c->geom.npad;
    R* a = (R*)c->adj[in_buf];
    R* b = (R*)c->adj[1 - in_buf];
    p.fb1 = a;
    p.gb1 = a + comp;
    p.pb1 = (R*)c->adj_p[in_buf];
    p.fb0 = b;
    p.gb0 = b + comp;
    p.pb0 = (R*)c->adj_p[1 - in_buf];
    p.gmb = (R*)c->adj_gmb;
    p.mub = (R*)c->adj_mub;
    p.phib = (R*)c->adj_phib;
    return p;
}

template <int P, bool ISO>
cudaError_t adj_step_iso(ld_ctx* c, const void* state_t, const void* fields_t, double* grad) {
    using S = typename Prec<P>::store_t;
    using R = typename Prec<P>::real_t;
    const Geom g = to_dev(c->geom);
    if (!fields_t) {
        cudaError_t e = phi_mu_p<P>(c, state_t);
        if (e != cudaSuccess) return e;
    }
    const R* phi = fields_t ? (const R*)fields_t : (const R*)c->phi;
    const R* mu = fields_t ? (const R*)fields_t + g.npad : (const R*)c->mu;
    const AdjPtrs<P> p = adj_ptrs<P>(c, c->adj_cur);
    const Model<R> m = model_of<R>(c->prm);
    const unsigned nb = blocks_for(g.n);
    k_adj_local<P, ISO><<<nb, kAdjThreads, 0, c->stream>>>(g, m, (const S*)f_part(c, state_t), phi, mu, c->ref, p.fb1,
                                                      p.gb1, p.pb1, p.fb0, p.gb0, p.gmb, p.mub, p.phib, c->adj_part);
    k_adj_mu<R, ISO><<<nb, kAdjThreads, 0, c->stream>>>(g, phi, p.gmb, p.mub, c->adj_part);
    k_adj_p<R, ISO><<<nb, kAdjThreads, 0, c->stream>>>(g, m, phi, p.mub, p.phib, p.pb0);
    if (grad)
        k_adj_finalize<<<1, kAdjThreads, 0, c->stream>>>(c->adj_part, nb, -1.0 / (c->prm.tau_f * c->prm.tau_f),
                                                         grad);
    return cudaGetLastError();
}

template <int P>
cudaError_t adj_step_p(ld_ctx* c, const void* state_t, const void* fields_t, double* grad) {
    return c->prm.stencil == LD_STENCIL_19 ? adj_step_iso<P, true>(c, state_t, fields_t, grad)
                                           : adj_step_iso<P, false>(c, state_t, fields_t, grad);
}

template <int P>
cudaError_t adj_seed_p(ld_ctx* c, const double* phibar) {
    using R = typename Prec<P>::real_t;
    const Geom g = to_dev(c->geom);
    const AdjPtrs<P> p = adj_ptrs<P>(c, c->adj_cur);
    k_adj_seed<R><<<blocks_for(g.n), kAdjThreads, 0, c->stream>>>(g, phibar, p.fb1, p.gb1, p.pb1);
    return cudaGetLastError();
}

template <int P, bool ISO>
cudaError_t adj_init_iso(ld_ctx* c, const double* phi0, const double* u0, double* grad_phi0, double* grad) {
    using R = typename Prec<P>::real_t;
    const Geom g = to_dev(c->geom);
    const AdjPtrs<P> p = adj_ptrs<P>(c, c->adj_cur);
    const unsigned nb = blocks_for(g.n);
    k_adj_init_mu<R><<<nb, kAdjThreads, 0, c->stream>>>(g, (R)c->prm.Gamma, p.gb1, p.pb1, p.mub);
    k_adj_init_phi<R, ISO><<<nb, kAdjThreads, 0, c->stream>>>(g, model_of<R>(c->prm), phi0, u0, p.gb1, p.pb1, p.mub,
                                                         grad_phi0, c->adj_part);
    if (grad) k_adj_finalize<<<1, kAdjThreads, 0, c->stream>>>(c->adj_part, nb, 0.0, grad);
    return cudaGetLastError();
}

template <int P>
cudaError_t adj_init_p(ld_ctx* c, const double* phi0, const double* u0, double* grad_phi0, double* grad) {
    return c->prm.stencil == LD_STENCIL_19 ? adj_init_iso<P, true>(c, phi0, u0, grad_phi0, grad)
                                           : adj_init_iso<P, false>(c, phi0, u0, grad_phi0, grad);
}

template <int P>
cudaError_t adj_io_p(ld_ctx* c, int to_double, double* fbar, double* gbar) {
    using R = typename Prec<P>::real_t;
    const Geom g = to_dev(c->geom);
    const AdjPtrs<P> p = adj_ptrs<P>(c, c->adj_cur);
    if (fbar) k_adj_io<R><<<blocks_for(g.n), kAdjThreads, 0, c->stream>>>(g, to_double, p.fb1, nullptr, fbar);
    if (gbar) k_adj_io<R><<<blocks_for(g.n), kAdjThreads, 0, c->stream>>>(g, to_double, p.gb1, p.pb1, gbar);
    return cudaGetLastError();
}

}  // namespace
}  // namespace ld
