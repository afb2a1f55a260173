// Generic kernels: any lattice size >= 4 in every dimension, one thread per
// site. The step runs as three launches in row order -- phi (zeroth moment
// of g), mu (7- or 19-point Laplacian), and collide+propagate, with a fourth
// for the chemical stress when the force is -div P -- and the same file holds the
// initialiser, the macroscopic output, the FP64 conservation sums, the
// codec I/O and propagation alone. Templates only: instantiated per storage
// precision by ld_prec_f64.cu and ld_prec_lp.cu.
#pragma once
#include "ld_common.cuh"
#include "ld_internal.h"

namespace ld {
namespace {

constexpr int kThreads = 256;

inline Geom to_dev(const GeomH& h) { return Geom{h.nx, h.ny, h.nz, h.n, h.npad}; }

inline unsigned blocks_for(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

__device__ __forceinline__ void site_coords(const Geom& g, long long s, int& x, int& y, int& z) {
    x = (int)(s % g.nx);
    long long t = s / g.nx;
    y = (int)(t % g.ny);
    z = (int)(t / g.ny);
}

__device__ __forceinline__ long long site_of(const Geom& g, int x, int y, int z) {
    return (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * z);
}

// Coordinate after a displacement of -1, 0 or +1 (periodic).
__device__ __forceinline__ int step_coord(int a, int d, int n) {
    return d > 0 ? wrap_inc(a, n) : (d < 0 ? wrap_dec(a, n) : a);
}

// ---------------------------------------------------------------------------
// The step as three launches in site order, one thread per site, each block
// a segment of kRowThreads sites of one x-row (a block never straddles two
// rows, so the coordinates need one division per thread).
// Consecutive blocks cover consecutive addresses of every stream, the order
// that lets HBM run at its copy rate. Element offsets i npad + s are of type
// I: 32-bit where 19 npad fits.
struct RowGeom {
    int nx, ny, nz, nchunks;  // nchunks = blocks per row
};

inline RowGeom row_geom(const GeomH& h) {
    return RowGeom{h.nx, h.ny, h.nz, (h.nx + kRowThreads - 1) / kRowThreads};
}

inline unsigned row_blocks(const GeomH& h) { return (unsigned)row_segments(h); }

// Site of this thread in row segment b (false past the end of its row).
__device__ __forceinline__ bool row_site(const RowGeom& rg, int b, int& x, int& y, int& z, int& s) {
    const int r = b / rg.nchunks;
    x = (b - r * rg.nchunks) * kRowThreads + threadIdx.x;
    y = r % rg.ny;
    z = r / rg.ny;
    s = r * rg.nx + x;
    return x < rg.nx;
}

// Stage 1: phi = sum_i g_i (the stored state is the post-propagation one).
template <int P, class I>
__global__ void __launch_bounds__(kRowThreads) k_phi(RowGeom rg, I npad, const typename Prec<P>::store_t* __restrict__ gs,
                                                     const float* __restrict__ ref,
                                                     typename Prec<P>::real_t* __restrict__ phi, int* __restrict__ status) {
    using R = typename Prec<P>::real_t;
    int x, y, z, s;
    if (!row_site(rg, blockIdx.x, x, y, z, s)) return;
    if (!site_ok(s, (long long)rg.nx * rg.ny * rg.nz, status)) return;
    R acc = R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) acc += Prec<P>::decode(gs[i * npad + s], ref[Q + i]);
    phi[s] = acc;
}

// Stage 2: mu = A phi + B phi^3 - kappa lap(phi), with the 7-point or the
// 19-point Laplacian.
template <class R>
__global__ void __launch_bounds__(kRowThreads) k_mu(RowGeom rg, Model<R> m, const R* __restrict__ phi,
                                                    R* __restrict__ mu) {
    int x, y, z, s;
    if (!row_site(rg, blockIdx.x, x, y, z, s)) return;
    const int nx = rg.nx, plane = rg.nx * rg.ny;
    const int xp = x + 1 == nx ? 1 - nx : 1, xm = x == 0 ? nx - 1 : -1;
    const int yp = y + 1 == rg.ny ? (1 - rg.ny) * nx : nx, ym = y == 0 ? (rg.ny - 1) * nx : -nx;
    const int zp = z + 1 == rg.nz ? (1 - rg.nz) * plane : plane, zm = z == 0 ? (rg.nz - 1) * plane : -plane;
    if (m.iso) {
        auto nb = [&](int i) {
            return phi[s + (cx(i) > 0 ? xp : (cx(i) < 0 ? xm : 0)) + (cy(i) > 0 ? yp : (cy(i) < 0 ? ym : 0)) +
                       (cz(i) > 0 ? zp : (cz(i) < 0 ? zm : 0))];
        };
        mu[s] = chem_potential_lap(phi[s], lap19(phi[s], nb), m);
        return;
    }
    const R nb = phi[s + xp] + phi[s + xm] + phi[s + yp] + phi[s + ym] + phi[s + zp] + phi[s + zm];
    mu[s] = chem_potential(phi[s], nb, m);
}

// Neighbour offsets of a row-ordered site (periodic).
struct RowNbr {
    int xp, xm, yp, ym, zp, zm;
    __device__ __forceinline__ int of(int i) const {
        return (cx(i) > 0 ? xp : (cx(i) < 0 ? xm : 0)) + (cy(i) > 0 ? yp : (cy(i) < 0 ? ym : 0)) +
               (cz(i) > 0 ? zp : (cz(i) < 0 ? zm : 0));
    }
};
__device__ __forceinline__ RowNbr row_nbr(const RowGeom& rg, int x, int y, int z) {
    const int nx = rg.nx, plane = rg.nx * rg.ny;
    return RowNbr{x + 1 == nx ? 1 - nx : 1,
                  x == 0 ? nx - 1 : -1,
                  y + 1 == rg.ny ? (1 - rg.ny) * nx : nx,
                  y == 0 ? (rg.ny - 1) * nx : -nx,
                  z + 1 == rg.nz ? (1 - rg.nz) * plane : plane,
                  z == 0 ? (rg.nz - 1) * plane : -plane};
}

// Gradient of a field at s with the selected stencils (7-point: central
// difference; 19-point: grad19), in the type of the field.
template <class T>
__device__ __forceinline__ void grad_at(int iso, const T* h, int s, const RowNbr& o, T& gx, T& gy, T& gz) {
    if (iso) {
        auto nb = [&](int i) { return h[s + o.of(i)]; };
        grad19(nb, gx, gy, gz);
    } else {
        gx = T(0.5) * (h[s + o.xp] - h[s + o.xm]);
        gy = T(0.5) * (h[s + o.yp] - h[s + o.ym]);
        gz = T(0.5) * (h[s + o.zp] - h[s + o.zm]);
    }
}

// Stage 2b (LD_FORCE_STRESS): chemical stress P[6][npad] (xx, yy, zz, xy,
// xz, yz) from grad phi and lap(phi) with the selected stencils:
//   iso = A/2 phi^2 + 3B/4 phi^4 - kappa phi lap - kappa/2 |grad phi|^2,
//   P_aa = iso + kappa (d_a phi)^2, P_ab = kappa d_a phi d_b phi,
// each expression in that operation order.
template <class R, class I>
__global__ void __launch_bounds__(kRowThreads) k_stress(RowGeom rg, I npad, Model<R> m, const R* __restrict__ phi,
                                                        R* __restrict__ P) {
    int x, y, z, s;
    if (!row_site(rg, blockIdx.x, x, y, z, s)) return;
    const RowNbr o = row_nbr(rg, x, y, z);
    const R ph = phi[s];
    R gx, gy, gz, lap;
    grad_at(m.iso, phi, s, o, gx, gy, gz);
    if (m.iso) {
        auto nb = [&](int i) { return phi[s + o.of(i)]; };
        lap = lap19(ph, nb);
    } else {
        lap = phi[s + o.xp] + phi[s + o.xm] + phi[s + o.yp] + phi[s + o.ym] + phi[s + o.zp] + phi[s + o.zm] - R(6) * ph;
    }
    const R pb = R(0.5) * m.A * ph * ph + R(0.75) * m.B * ph * ph * ph * ph;
    const R iso = pb - m.kappa * ph * lap - R(0.5) * m.kappa * (gx * gx + gy * gy + gz * gz);
    P[s] = iso + m.kappa * gx * gx;
    P[npad + s] = iso + m.kappa * gy * gy;
    P[2 * npad + s] = iso + m.kappa * gz * gz;
    P[3 * npad + s] = m.kappa * gx * gy;
    P[4 * npad + s] = m.kappa * gx * gz;
    P[5 * npad + s] = m.kappa * gy * gz;
}

// F = -div P at s: F_a = -((D_x P_ax + D_y P_ay) + D_z P_az), D the selected
// gradient, components of P indexed xx 0, yy 1, zz 2, xy 3, xz 4, yz 5.
template <class T, class I>
__device__ __forceinline__ void stress_force_at(int iso, const T* P, I npad, int s, const RowNbr& o, T& Fx, T& Fy,
                                                T& Fz) {
    T d[6][3];
#pragma unroll
    for (int c = 0; c < 6; ++c) grad_at(iso, P + c * npad, s, o, d[c][0], d[c][1], d[c][2]);
    Fx = -((d[0][0] + d[3][1]) + d[4][2]);
    Fy = -((d[3][0] + d[1][1]) + d[5][2]);
    Fz = -((d[4][0] + d[5][1]) + d[2][2]);
}

// Resident blocks per SM the collision kernel is compiled for: 6 x 128
// threads (80 registers) with FP32 arithmetic, 3 with FP64.
template <int P>
constexpr int rows_blocks_per_sm() {
    return sizeof(typename Prec<P>::real_t) == 4 ? 6 : 3;
}

// Stage 3: force, velocity, collisions of f and g, and propagation (push: the
// post-collision value of direction i goes to x + c_i) with streaming stores;
// SR: the 16-bit stores rounded stochastically from the stream `sr`.
template <int P, class I, bool SR>
__global__ void __launch_bounds__(kRowThreads, rows_blocks_per_sm<P>())
    k_collide(RowGeom rg, I npad, Model<typename Prec<P>::real_t> m, SrStream sr, const typename Prec<P>::store_t* __restrict__ fs,
              const typename Prec<P>::store_t* __restrict__ gs, typename Prec<P>::store_t* __restrict__ fd,
              typename Prec<P>::store_t* __restrict__ gd, const typename Prec<P>::real_t* __restrict__ phi,
              const typename Prec<P>::real_t* __restrict__ mu, const float* __restrict__ ref,
              const typename Prec<P>::real_t* __restrict__ stress, int* __restrict__ status) {
    using R = typename Prec<P>::real_t;
    using S = typename Prec<P>::store_t;
    __shared__ float refs[2 * Q];  // codec references, read once per block
    if (threadIdx.x < 2 * Q) refs[threadIdx.x] = ref[threadIdx.x];
    __syncthreads();
    int x, y, z, s;
    if (!row_site(rg, blockIdx.x, x, y, z, s)) return;
    const long long n = (long long)rg.nx * rg.ny * rg.nz;
    if (!site_ok(s, n, status)) return;
    // FP32 and FP64 issue all 38 loads first; the 16-bit forms issue g after
    // the f stores (each 16-bit value held early would take a register).
    constexpr bool kEarlyG = sizeof(S) >= 4;
    S fr[Q], gr[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        fr[i] = __ldcs(fs + i * npad + s);
        if (kEarlyG) gr[i] = __ldcs(gs + i * npad + s);
    }
    const int nx = rg.nx, plane = rg.nx * rg.ny;
    const int oxp = x + 1 == nx ? 1 - nx : 1, oxm = x == 0 ? nx - 1 : -1;
    const int oyp = y + 1 == rg.ny ? (1 - rg.ny) * nx : nx, oym = y == 0 ? (rg.ny - 1) * nx : -nx;
    const int ozp = z + 1 == rg.nz ? (1 - rg.nz) * plane : plane, ozm = z == 0 ? (rg.nz - 1) * plane : -plane;

    const R ph = phi[s], muc = mu[s];
    const RowNbr o{oxp, oxm, oyp, oym, ozp, ozm};
    R Fx, Fy, Fz;
    if (stress) {  // F = -div P
        stress_force_at(m.iso, stress, npad, s, o, Fx, Fy, Fz);
    } else {  // F = -phi grad(mu)
        R gmx, gmy, gmz;
        grad_at(m.iso, mu, s, o, gmx, gmy, gmz);
        Fx = -ph * gmx, Fy = -ph * gmy, Fz = -ph * gmz;
    }

    R f[Q];
    R rho = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        f[i] = Prec<P>::decode(fr[i], refs[i]);
        rho += f[i];
        add_c(i, f[i], jx, jy, jz);
    }
    R ux, uy, uz;
    guo_velocity(rho, jx, jy, jz, Fx, Fy, Fz, ux, uy, uz);
    if (m.trt)
        collide_f_trt(f, rho, ux, uy, uz, Fx, Fy, Fz, m);
    else
        collide_f(f, rho, ux, uy, uz, Fx, Fy, Fz, m);
    const unsigned long long sr_st = SR ? sr.base + (unsigned long long)s * kSrGamma : 0ull;
    unsigned long long sr_w = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int d = s + (cx(i) > 0 ? oxp : (cx(i) < 0 ? oxm : 0)) + (cy(i) > 0 ? oyp : (cy(i) < 0 ? oym : 0)) +
                      (cz(i) > 0 ? ozp : (cz(i) < 0 ? ozm : 0));
        S v;
        if constexpr (SR)
            v = Prec<P>::encode_sr(f[i], refs[i], sr_key(sr, sr_st, 0, i, sr_w));
        else
            v = Prec<P>::encode(f[i], refs[i]);
        if (site_ok(d, n, status)) __stcs(fd + i * npad + d, v);
    }
    R gg[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) gg[i] = Prec<P>::decode(kEarlyG ? gr[i] : __ldcs(gs + i * npad + s), refs[Q + i]);
    collide_g(gg, ph, muc, ux, uy, uz, m);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int d = s + (cx(i) > 0 ? oxp : (cx(i) < 0 ? oxm : 0)) + (cy(i) > 0 ? oyp : (cy(i) < 0 ? oym : 0)) +
                      (cz(i) > 0 ? ozp : (cz(i) < 0 ? ozm : 0));
        S v;
        if constexpr (SR)
            v = Prec<P>::encode_sr(gg[i], refs[Q + i], sr_key(sr, sr_st, 1, i, sr_w));
        else
            v = Prec<P>::encode(gg[i], refs[Q + i]);
        if (site_ok(d, n, status)) __stcs(gd + i * npad + d, v);
    }
}

// ---------------------------------------------------------------------------
// Initial state: f = feq(rho, u), g = geq(phi, u, mu(phi)), computed in the
// arithmetic type of the precision from the FP64 inputs, then encoded.
template <int P>
__global__ void __launch_bounds__(kThreads)
    k_init(Geom g, Model<typename Prec<P>::real_t> m, double rho0, const double* __restrict__ phi,
           const double* __restrict__ rho_in, const double* __restrict__ u_in, const float* __restrict__ ref,
           typename Prec<P>::store_t* __restrict__ fd, typename Prec<P>::store_t* __restrict__ gd) {
    using R = typename Prec<P>::real_t;
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.n) return;
    int x, y, z;
    site_coords(g, s, x, y, z);
    const R p = (R)phi[s];
    R lap;
    if (m.iso) {
        lap = R(0);
#pragma unroll
        for (int i = 1; i < Q; ++i)
            lap += lap19_coef<R>(i) *
                   ((R)phi[site_of(g, step_coord(x, cx(i), g.nx), step_coord(y, cy(i), g.ny), step_coord(z, cz(i), g.nz))] -
                    p);
    } else {
        lap = (R)phi[site_of(g, wrap_inc(x, g.nx), y, z)] + (R)phi[site_of(g, wrap_dec(x, g.nx), y, z)]
            + (R)phi[site_of(g, x, wrap_inc(y, g.ny), z)] + (R)phi[site_of(g, x, wrap_dec(y, g.ny), z)]
            + (R)phi[site_of(g, x, y, wrap_inc(z, g.nz))] + (R)phi[site_of(g, x, y, wrap_dec(z, g.nz))] - R(6) * p;
    }
    const R mu = m.A * p + m.B * p * p * p - m.kappa * lap;
    const R rho = (R)(rho_in ? rho_in[s] : rho0);
    R ux = R(0), uy = R(0), uz = R(0);
    if (u_in) {
        ux = (R)u_in[s];
        uy = (R)u_in[g.n + s];
        uz = (R)u_in[2 * g.n + s];
    }
    const R uu = ux * ux + uy * uy + uz * uz;
    const R dev = m.Gamma * mu - p / R(3);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const R cu = cdot(i, ux, uy, uz);
        const R feq = wgt<R>(i) * rho * (R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu);
        const R geq = wgt<R>(i) * (p + R(3) * p * cu + R(4.5) * dev * R(c2(i) - 1) + R(4.5) * p * cu * cu
                                   - R(1.5) * p * uu);
        fd[i * g.npad + s] = Prec<P>::encode_d((double)feq, ref[i]);
        gd[i * g.npad + s] = Prec<P>::encode_d((double)geq, ref[Q + i]);
    }
}

// Deviation references from the total of phi (in totals[0]): f_i: w_i rho0;
// g_i: geq_i(phibar, 0, A phibar + B phibar^3).
// Deviation references of the 16-bit forms: f_i w_i rho0; g_i geq_i(pb, 0, mu(pb))
// with pb the mean of the initial phi: totals[0] / n (mean_given = false) or
// `mean` itself (a part of a larger lattice that takes the whole one's mean).
__global__ void k_refs(const double* __restrict__ totals, long long n, double mean, int mean_given, Model<double> m,
                       double rho0, float* __restrict__ ref) {
    const int i = threadIdx.x;
    if (i >= Q) return;
    const double pb = mean_given ? mean : totals[0] / (double)n;
    const double mub = m.A * pb + m.B * pb * pb * pb;
    ref[i] = (float)(wgt<double>(i) * rho0);
    ref[Q + i] = (float)(wgt<double>(i) * (pb + 4.5 * (m.Gamma * mub - pb / 3.0) * (c2(i) - 1)));
}

__global__ void k_default_refs(double rho0, float* __restrict__ ref) {
    const int i = threadIdx.x;
    if (i >= Q) return;
    ref[i] = (float)(wgt<double>(i) * rho0);
    ref[Q + i] = 0.0f;
}

// ---------------------------------------------------------------------------
// Deterministic FP64 reductions: fixed grid, fixed per-thread order, fixed
// shuffle tree; then one ordered pass over the block partials.
template <int K>
__device__ __forceinline__ void block_sum_store(double (&v)[K], double* __restrict__ out_block) {
    __shared__ double red[kRedThreads / 32][K];
#pragma unroll
    for (int k = 0; k < K; ++k)
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) red[warp][k] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double a = lane < kRedThreads / 32 ? red[lane][k] : 0.0;
            for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
            if (lane == 0) out_block[k] = a;
        }
    }
}

__global__ void __launch_bounds__(kRedThreads) k_sum_field(long long n, const double* __restrict__ x,
                                                           double* __restrict__ partials) {
    double v[1] = {0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += stride) v[0] += x[s];
    block_sum_store<1>(v, partials + (long long)blockIdx.x * kRedFields);
}

template <int P>
__global__ void __launch_bounds__(kRedThreads)
    k_totals(Geom g, const typename Prec<P>::store_t* __restrict__ fs,
             const typename Prec<P>::store_t* __restrict__ gs, const float* __restrict__ ref,
             double* __restrict__ partials) {
    // Each site's moments are summed in the arithmetic type of the precision
    // (as the step itself forms them); sites accumulate in FP64.
    using R = typename Prec<P>::real_t;
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.n; s += stride) {
        R rho = R(0), phi = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const R fi = Prec<P>::decode(fs[i * g.npad + s], ref[i]);
            rho += fi;
            add_c(i, fi, jx, jy, jz);
            phi += Prec<P>::decode(gs[i * g.npad + s], ref[Q + i]);
        }
        v[0] += (double)rho;
        v[1] += (double)phi;
        v[2] += (double)jx;
        v[3] += (double)jy;
        v[4] += (double)jz;
    }
    block_sum_store<5>(v, partials + (long long)blockIdx.x * kRedFields);
}

// Final ordered pass: out[k] = sum over blocks of partials[b][k].
__global__ void __launch_bounds__(kRedBlocks) k_finalize(const double* __restrict__ partials, int nfields,
                                                         double* __restrict__ out) {
    __shared__ double red[kRedBlocks / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < nfields; ++k) {
        double a = partials[(long long)threadIdx.x * kRedFields + k];
        for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
        if (lane == 0) red[warp] = a;
        __syncthreads();
        if (warp == 0) {
            double b = red[lane];
            for (int off = 16; off > 0; off >>= 1) b += __shfl_down_sync(0xffffffffu, b, off);
            if (lane == 0) out[k] = b;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Macroscopic output (double): rho, u = (j + F/2)/rho, phi, grad phi.
template <int P>
__global__ void __launch_bounds__(kThreads)
    k_macros(Geom g, const typename Prec<P>::store_t* __restrict__ fs,
             const typename Prec<P>::store_t* __restrict__ gs, const typename Prec<P>::real_t* __restrict__ phis,
             const typename Prec<P>::real_t* __restrict__ mu, const float* __restrict__ ref,
             double* __restrict__ rho_out, double* __restrict__ u_out, double* __restrict__ phi_out,
             double* __restrict__ gphi_out, int iso, const typename Prec<P>::real_t* __restrict__ stress) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.n) return;
    int x, y, z;
    site_coords(g, s, x, y, z);
    const int xp = wrap_inc(x, g.nx), xm = wrap_dec(x, g.nx);
    const int yp = wrap_inc(y, g.ny), ym = wrap_dec(y, g.ny);
    const int zp = wrap_inc(z, g.nz), zm = wrap_dec(z, g.nz);
    double rho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0, ph = 0.0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const double fi = Prec<P>::decode_d(fs[i * g.npad + s], ref[i]);
        rho += fi;
        jx += cx(i) * fi;
        jy += cy(i) * fi;
        jz += cz(i) * fi;
        ph += Prec<P>::decode_d(gs[i * g.npad + s], ref[Q + i]);
    }
    if (rho_out) rho_out[s] = rho;
    if (phi_out) phi_out[s] = ph;
    // gradient of a field (the selected stencil), in FP64
    auto grad = [&](const typename Prec<P>::real_t* h, double& gx, double& gy, double& gz) {
        if (iso) {
            auto nb = [&](int i) {
                return (double)h[site_of(g, step_coord(x, cx(i), g.nx), step_coord(y, cy(i), g.ny),
                                         step_coord(z, cz(i), g.nz))];
            };
            grad19(nb, gx, gy, gz);
        } else {
            gx = 0.5 * ((double)h[site_of(g, xp, y, z)] - (double)h[site_of(g, xm, y, z)]);
            gy = 0.5 * ((double)h[site_of(g, x, yp, z)] - (double)h[site_of(g, x, ym, z)]);
            gz = 0.5 * ((double)h[site_of(g, x, y, zp)] - (double)h[site_of(g, x, y, zm)]);
        }
    };
    if (u_out) {
        double Fx, Fy, Fz;
        if (stress) {  // F = -div P
            double d[6][3];
            for (int c = 0; c < 6; ++c) grad(stress + c * g.npad, d[c][0], d[c][1], d[c][2]);
            Fx = -((d[0][0] + d[3][1]) + d[4][2]);
            Fy = -((d[3][0] + d[1][1]) + d[5][2]);
            Fz = -((d[4][0] + d[5][1]) + d[2][2]);
        } else {  // F = -phi grad(mu)
            double gx, gy, gz;
            grad(mu, gx, gy, gz);
            Fx = -ph * gx, Fy = -ph * gy, Fz = -ph * gz;
        }
        u_out[s] = (jx + 0.5 * Fx) / rho;
        u_out[g.n + s] = (jy + 0.5 * Fy) / rho;
        u_out[2 * g.n + s] = (jz + 0.5 * Fz) / rho;
    }
    if (gphi_out) grad(phis, gphi_out[s], gphi_out[g.n + s], gphi_out[2 * g.n + s]);
}

// Distributions out (decoded, stride n) and in (encoded).
template <int P>
__global__ void __launch_bounds__(kThreads) k_decode(Geom g, const typename Prec<P>::store_t* __restrict__ src,
                                                     const float* __restrict__ ref, double* __restrict__ out) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.n) return;
#pragma unroll
    for (int i = 0; i < Q; ++i) out[i * g.n + s] = Prec<P>::decode_d(src[i * g.npad + s], ref[i]);
}

template <int P>
__global__ void __launch_bounds__(kThreads) k_encode(Geom g, const double* __restrict__ in,
                                                     const float* __restrict__ ref,
                                                     typename Prec<P>::store_t* __restrict__ dst) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.n) return;
#pragma unroll
    for (int i = 0; i < Q; ++i) dst[i * g.npad + s] = Prec<P>::encode_d(in[i * g.n + s], ref[i]);
}

// Propagation alone on raw storage words (T has the storage width).
template <class T>
__global__ void __launch_bounds__(kThreads) k_propagate(Geom g, int reverse, const T* __restrict__ src,
                                                        T* __restrict__ dst) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.n) return;
    int x, y, z;
    site_coords(g, s, x, y, z);
#pragma unroll
    for (int i = 0; i < 2 * Q; ++i) {  // f components then g components
        const int q = i % Q;
        const long long o = site_of(g, step_coord(x, cx(q), g.nx), step_coord(y, cy(q), g.ny),
                                    step_coord(z, cz(q), g.nz));
        if (reverse)
            dst[i * g.npad + s] = src[i * g.npad + o];
        else
            dst[i * g.npad + o] = src[i * g.npad + s];
    }
}

// ---------------------------------------------------------------------------
template <int P>
cudaError_t init_p(ld_ctx* c, const double* phi, const double* rho, const double* u, const double* ref_mean) {
    using S = typename Prec<P>::store_t;
    const Geom g = to_dev(c->geom);
    const Model<double> m = model_of<double>(c->prm);
    if (Prec<P>::kDev) {
        if (!ref_mean) {
            k_sum_field<<<kRedBlocks, kRedThreads, 0, c->stream>>>(g.n, phi, c->partials);
            k_finalize<<<1, kRedBlocks, 0, c->stream>>>(c->partials, 1, c->totals);
        }
        k_refs<<<1, 32, 0, c->stream>>>(c->totals, g.n, ref_mean ? *ref_mean : 0.0, ref_mean ? 1 : 0, m, c->prm.rho0,
                                        c->ref);
    } else {
        k_default_refs<<<1, 32, 0, c->stream>>>(c->prm.rho0, c->ref);
    }
    k_init<P><<<blocks_for(g.n), kThreads, 0, c->stream>>>(g, model_of<typename Prec<P>::real_t>(c->prm),
                                                           c->prm.rho0, phi, rho, u, c->ref,
                                                           (S*)f_of(c, c->cur), (S*)g_of(c, c->cur));
    return cudaGetLastError();
}

// phi and mu of a state into `fields` ([phi npad][mu npad]), or into the
// context's scratch when fields is null.
template <int P, class I>
cudaError_t phi_mu_rows(ld_ctx* c, const void* state, void* fields) {
    using S = typename Prec<P>::store_t;
    using R = typename Prec<P>::real_t;
    const RowGeom rg = row_geom(c->geom);
    const unsigned nb = row_blocks(c->geom);
    R* phi = fields ? (R*)fields : (R*)c->phi;
    R* mu = fields ? (R*)fields + c->geom.npad : (R*)c->mu;
    k_phi<P, I><<<nb, kRowThreads, 0, c->stream>>>(rg, (I)c->geom.npad, (const S*)g_part(c, state), c->ref, phi,
                                                   c->status);
    k_mu<R><<<nb, kRowThreads, 0, c->stream>>>(rg, model_of<R>(c->prm), phi, mu);
    return cudaGetLastError();
}

inline bool offsets_fit_int(const ld_ctx* c) { return (long long)Q * c->geom.npad <= 0x7fffffffLL; }

template <int P>
cudaError_t phi_mu_p(ld_ctx* c, const void* state, void* fields = nullptr) {
    return offsets_fit_int(c) ? phi_mu_rows<P, int>(c, state, fields) : phi_mu_rows<P, long long>(c, state, fields);
}

template <int P, class I, bool SR>
cudaError_t collide_rows(ld_ctx* c, const void* src, void* dst, void* fields) {
    using S = typename Prec<P>::store_t;
    using R = typename Prec<P>::real_t;
    cudaError_t e = phi_mu_rows<P, I>(c, src, fields);
    if (e != cudaSuccess) return e;
    const R* phi = fields ? (const R*)fields : (const R*)c->phi;
    const R* mu = fields ? (const R*)fields + c->geom.npad : (const R*)c->mu;
    if (c->stress)
        k_stress<R, I><<<row_blocks(c->geom), kRowThreads, 0, c->stream>>>(row_geom(c->geom), (I)c->geom.npad,
                                                                           model_of<R>(c->prm), phi, (R*)c->stress);
    k_collide<P, I, SR><<<row_blocks(c->geom), kRowThreads, 0, c->stream>>>(
        row_geom(c->geom), (I)c->geom.npad, model_of<R>(c->prm), sr_stream(c->prm.seed, c->sr_step, c->geom.n),
        (const S*)f_part(c, src), (const S*)g_part(c, src),
        (S*)f_part(c, dst), (S*)g_part(c, dst), phi, mu, c->ref, (const R*)c->stress, c->status);
    return cudaGetLastError();
}

template <int P, bool SR>
cudaError_t collide_r(ld_ctx* c, const void* src, void* dst, void* fields) {
    return offsets_fit_int(c) ? collide_rows<P, int, SR>(c, src, dst, fields)
                              : collide_rows<P, long long, SR>(c, src, dst, fields);
}

template <int P>
cudaError_t collide_p(ld_ctx* c, const void* src, void* dst, void* fields) {
    if constexpr (Prec<P>::kDev) {
        if (c->prm.rounding == LD_ROUND_STOCHASTIC) return collide_r<P, true>(c, src, dst, fields);
    }
    return collide_r<P, false>(c, src, dst, fields);
}

template <int P>
cudaError_t macros_p(ld_ctx* c, double* rho, double* u, double* phi, double* gphi) {
    using S = typename Prec<P>::store_t;
    using R = typename Prec<P>::real_t;
    const Geom g = to_dev(c->geom);
    cudaError_t e = phi_mu_p<P>(c, c->dist[c->cur]);
    if (e != cudaSuccess) return e;
    if (c->stress) {
        if (offsets_fit_int(c))
            k_stress<R, int><<<row_blocks(c->geom), kRowThreads, 0, c->stream>>>(
                row_geom(c->geom), (int)g.npad, model_of<R>(c->prm), (const R*)c->phi, (R*)c->stress);
        else
            k_stress<R, long long><<<row_blocks(c->geom), kRowThreads, 0, c->stream>>>(
                row_geom(c->geom), (long long)g.npad, model_of<R>(c->prm), (const R*)c->phi, (R*)c->stress);
    }
    k_macros<P><<<blocks_for(g.n), kThreads, 0, c->stream>>>(g, (const S*)f_of(c, c->cur), (const S*)g_of(c, c->cur),
                                                             (const R*)c->phi, (const R*)c->mu, c->ref, rho, u,
                                                             phi, gphi, c->prm.stencil == LD_STENCIL_19,
                                                             (const R*)c->stress);
    return cudaGetLastError();
}

template <int P>
cudaError_t totals_p(ld_ctx* c, double* out) {
    using S = typename Prec<P>::store_t;
    const Geom g = to_dev(c->geom);
    k_totals<P><<<kRedBlocks, kRedThreads, 0, c->stream>>>(g, (const S*)f_of(c, c->cur), (const S*)g_of(c, c->cur),
                                                           c->ref, c->partials);
    k_finalize<<<1, kRedBlocks, 0, c->stream>>>(c->partials, 5, out);
    return cudaGetLastError();
}

template <int P>
cudaError_t decode_p(ld_ctx* c, double* f, double* gout) {
    using S = typename Prec<P>::store_t;
    const Geom g = to_dev(c->geom);
    if (f) k_decode<P><<<blocks_for(g.n), kThreads, 0, c->stream>>>(g, (const S*)f_of(c, c->cur), c->ref, f);
    if (gout)
        k_decode<P><<<blocks_for(g.n), kThreads, 0, c->stream>>>(g, (const S*)g_of(c, c->cur), c->ref + Q, gout);
    return cudaGetLastError();
}

template <int P>
cudaError_t encode_p(ld_ctx* c, const double* f, const double* gin) {
    using S = typename Prec<P>::store_t;
    const Geom g = to_dev(c->geom);
    if (f) k_encode<P><<<blocks_for(g.n), kThreads, 0, c->stream>>>(g, f, c->ref, (S*)f_of(c, c->cur));
    if (gin) k_encode<P><<<blocks_for(g.n), kThreads, 0, c->stream>>>(g, gin, c->ref + Q, (S*)g_of(c, c->cur));
    return cudaGetLastError();
}


// Precision-independent launches.
cudaError_t default_refs(ld_ctx* c) {
    k_default_refs<<<1, 32, 0, c->stream>>>(c->prm.rho0, c->ref);
    return cudaGetLastError();
}

cudaError_t propagate_raw(ld_ctx* c, int reverse) {
    const Geom g = to_dev(c->geom);
    const void* src = c->dist[c->cur];
    void* dst = c->dist[1 - c->cur];
    const unsigned nb = blocks_for(g.n);
    switch (c->store_bytes) {
        case 8:
            k_propagate<unsigned long long><<<nb, kThreads, 0, c->stream>>>(g, reverse, (const unsigned long long*)src,
                                                                            (unsigned long long*)dst);
            break;
        case 4:
            k_propagate<unsigned int><<<nb, kThreads, 0, c->stream>>>(g, reverse, (const unsigned int*)src,
                                                                      (unsigned int*)dst);
            break;
        case 2:
            k_propagate<unsigned short><<<nb, kThreads, 0, c->stream>>>(g, reverse, (const unsigned short*)src,
                                                                        (unsigned short*)dst);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace
}  // namespace ld
