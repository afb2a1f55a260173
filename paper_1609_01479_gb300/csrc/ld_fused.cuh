// Fused single-pass step: one launch per timestep that reads each stored
// distribution once from HBM and writes each once.
//
// Each CTA owns a TX x TY column of sites and marches up a chunk of ZC
// z-planes. The order-parameter chain phi -> mu -> grad(mu) needs phi within
// radius 2 and mu within radius 1 of every collided site, so the CTA keeps
// two rolling rings in shared memory:
//   phi ring: 3 planes of (TX+4) x (TY+4)  (tile + 2-site halo)
//   mu ring:  3 planes of (TX+2) x (TY+2)  (tile + 1-site halo)
// Iteration k computes phi(k+2) from the stored g of that plane (the state is
// the post-propagation one, so phi is the local sum of 19 values), then
// mu(k+1), then collides plane k and propagates it (push to x + c_i). The g
// of plane k is read again for the collision two planes after phi(k) read
// it; that second read and the halo reads of neighbouring tiles are served by
// L2 (the phi pass loads g under an evict-last policy, the collision re-reads
// it as evict-first). Propagation writes into the other buffer of the
// ping-pong pair.
// The 16-bit storage forms keep the tile's g values of the last three planes
// in a shared-memory ring (29 KB) as the phi pass loads them, so the
// collision two planes later reads g from shared memory rather than again
// from L2 or HBM (under a full machine those lines have often left L2 by
// then). FP32 and FP64 read g again: their ring (58 KB, 117 KB) would cost
// CTAs per SM, which measured slower.
// Template only: instantiated per storage precision by ld_prec_f64.cu and
// ld_prec_lp.cu.
#pragma once
#include "ld_common.cuh"
#include "ld_internal.h"
#include "ld_async.cuh"

namespace ld {
namespace {

constexpr int kTX = 32;

// FP32: where the collision's loads of the plane are issued. Before the phi
// pass (kF32TopLoad) or after it (kF32MidLoad): 0 neither, 1 the g re-read (an
// L2 hit), 2 f (from HBM); the rest at the collision. Measured on one box at
// 256^3 / 384^3 (fraction of HBM): g after the phi pass 0.718 / 0.734, g
// before it 0.717 / 0.715, f after it (g before) 0.697 / 0.697, f before and
// g after 0.658 / 0.665, f after and g at the collision 0.677 / 0.684, f
// before 0.697 / 0.666.
constexpr int kF32TopLoad = 0, kF32MidLoad = 1;

// Resident CTAs per SM the kernel is compiled for: three 256-thread CTAs
// (80 registers a thread) with FP32 arithmetic, two with FP64.
template <int P>
constexpr int fused_ctas_per_sm() {
    return sizeof(typename Prec<P>::real_t) == 4 ? 3 : 2;
}

// Periodic image of a coordinate at most one period outside [0, n).
__device__ __forceinline__ int wrap_once(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// First plane of z-chunk b when nz planes are split into nchunks chunks
// whose lengths differ by at most one.
__host__ __device__ inline int chunk_begin(int b, int nz, int nchunks) {
    return (int)(((long long)b * nz) / nchunks);
}

// A 16-bit storage word from its bit pattern.
template <class T>
__device__ __forceinline__ T bits16(unsigned b) {
    const unsigned short u = (unsigned short)b;
    T v;
    memcpy(&v, &u, 2);
    return v;
}

// I: type of the element offsets i * npad + s. A 32-bit offset keeps the
// 19 per-direction offsets, which the compiler holds for the whole kernel,
// in one register each; 64-bit only where 19 npad does not fit in it.
// ISO: the 19-point isotropic stencils (mu's Laplacian over the phi ring,
// grad mu over the mu ring, corners included) instead of the 7-point ones.
// SR: stochastic rounding of the 16-bit stores, from the stream `sr`.
template <int P, int TY, class I, bool ISO, bool SR>
__global__ void __launch_bounds__(kTX * TY, fused_ctas_per_sm<P>())
    k_step_fused(Geom g, Model<typename Prec<P>::real_t> m, int nchunks,
                 const typename Prec<P>::store_t* __restrict__ fs, const typename Prec<P>::store_t* __restrict__ gs,
                 typename Prec<P>::store_t* __restrict__ fd, typename Prec<P>::store_t* __restrict__ gd,
                 const float* __restrict__ ref_g, typename Prec<P>::real_t* __restrict__ phi_out,
                 typename Prec<P>::real_t* __restrict__ mu_out, SrStream sr, int* __restrict__ status) {
    using R = typename Prec<P>::real_t;
    using S = typename Prec<P>::store_t;
    constexpr int PW = kTX + 4, PH = TY + 4;  // phi ring plane
    constexpr int MW = kTX + 2, MH = TY + 2;  // mu ring plane
    constexpr int NT = kTX * TY;
    constexpr bool kKeepG = sizeof(S) == 2;
    // Where the collision's loads are issued (FP64 has no registers to spare
    // for either): before the phi pass (top) or after it (mid).
    constexpr bool k32 = sizeof(S) == 4;
    constexpr bool kTopG = k32 && kF32TopLoad == 1, kTopF = k32 && kF32TopLoad == 2;
    constexpr bool kMidG = k32 && kF32MidLoad == 1, kMidF = kKeepG || (k32 && kF32MidLoad == 2);
    constexpr bool kEarlyG = kTopG || kMidG, kEarlyF = kTopF || kMidF;
    __shared__ R phis[3][PH][PW];
    __shared__ R mus[3][MH][MW];
    __shared__ float refs[2 * Q];
    __shared__ DevRefs dref;  // deviation-space constants (16-bit forms)
    extern __shared__ __align__(16) unsigned char keep_smem[];
    S* gring = reinterpret_cast<S*>(keep_smem);  // [3][Q][TY][kTX], slot = phi slot of the plane

    const int tid = threadIdx.x;
    const int tx = tid % kTX, ty = tid / kTX;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * TY;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int z0 = chunk_begin(blockIdx.z, nz, nchunks), z1 = chunk_begin(blockIdx.z + 1, nz, nchunks);
    const int plane = nx * ny;
    const I npad = (I)g.npad;
    if (tid < 2 * Q) refs[tid] = ref_g[tid];
    if constexpr (kKeepG) {
        if (tid == 0) dref = dev_refs_of(ref_g, m);
    }
    // g is read by the phi pass and, two planes later, by the collision:
    // keep those lines in L2 until then, and release them at the second read.
    const uint64_t keep_l2 = make_l2_evict_last_policy(), drop_l2 = make_l2_evict_first_policy();
    __syncthreads();

    // phi of plane zp over the tile + 2-halo, into ring slot `slot`. With
    // 32- and 16-bit storage each thread sums two x-adjacent sites from
    // paired loads: 216 pairs, one round for 256 threads, half the load and
    // address instructions. The halo's x range starts at an even x and nx is
    // even, so a pair never straddles the periodic wrap; each site's sum over
    // i keeps its order, so phi is the same as from single loads.
    auto phi_plane = [&](int zp, int slot) {
        const int zoff = wrap_once(zp, nz) * plane;
        if constexpr (sizeof(S) <= 4) {
            constexpr int PW2 = PW / 2;
            for (int idx = tid; idx < PW2 * PH; idx += NT) {
                const int hx = 2 * (idx % PW2), hy = idx / PW2;
                const int gx = wrap_once(x0 + hx - 2, nx), gy = wrap_once(y0 + hy - 2, ny);
                const int s = zoff + gy * nx + gx;  // even
                const bool sok = site_ok(s, g.n, status) && site_ok(s + 1, g.n, status);
                const bool interior = kKeepG && hx >= 2 && hx < kTX + 2 && hy >= 2 && hy < TY + 2;
                S* keep = gring + ((size_t)slot * Q * TY + (hy - 2)) * kTX + (hx - 2);
                R a0 = R(0), a1 = R(0);
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    if constexpr (sizeof(S) == 4) {
                        const float2 v = sok ? ld_l2_hint_pair(gs + i * npad + s, keep_l2) : make_float2(0.f, 0.f);
                        a0 += v.x;
                        a1 += v.y;
                    } else {  // psi: the sum of the deviations
                        const unsigned v = sok ? ld_l2_hint_pair(gs + i * npad + s, keep_l2) : 0u;
                        if constexpr (P == LD_FP16DEV) {
                            a0 = add_f16(a0, (unsigned short)(v & 0xffffu));
                            a1 = add_f16(a1, (unsigned short)(v >> 16));
                        } else {
                            a0 = add_bf16(a0, (unsigned short)(v & 0xffffu));
                            a1 = add_bf16(a1, (unsigned short)(v >> 16));
                        }
                        if (interior) *reinterpret_cast<unsigned*>(keep + i * (TY * kTX)) = v;
                    }
                }
                phis[slot][hy][hx] = a0;
                phis[slot][hy][hx + 1] = a1;
            }
        } else {
            for (int idx = tid; idx < PW * PH; idx += NT) {
                const int hx = idx % PW, hy = idx / PW;
                const int gx = wrap_once(x0 + hx - 2, nx), gy = wrap_once(y0 + hy - 2, ny);
                const int s = zoff + gy * nx + gx;
                const bool sok = site_ok(s, g.n, status);
                const bool interior = kKeepG && hx >= 2 && hx < kTX + 2 && hy >= 2 && hy < TY + 2;
                S* keep = gring + ((size_t)slot * Q * TY + (hy - 2)) * kTX + (hx - 2);
                R acc = R(0);
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const S v = sok ? ld_l2_hint(gs + i * npad + s, keep_l2) : S(0);
                    acc += Prec<P>::decode(v, refs[Q + i]);
                    if (interior) keep[i * (TY * kTX)] = v;
                }
                phis[slot][hy][hx] = acc;
            }
        }
    };
    // mu over the tile + 1-halo from three phi slots (below, middle, above).
    // The ring holds phi, or psi = phi - Phi in the 16-bit forms: the
    // Laplacian is the same, the cubic term takes phi.
    auto mu_plane = [&](int slot, int lo, int mid, int hi) {
        for (int idx = tid; idx < MW * MH; idx += NT) {
            const int mx = idx % MW, my = idx / MW;
            const int hx = mx + 1, hy = my + 1;
            const R c = phis[mid][hy][hx];
            R lap;
            if constexpr (ISO) {
                auto nb = [&](int i) { return phis[cz(i) > 0 ? hi : (cz(i) < 0 ? lo : mid)][hy + cy(i)][hx + cx(i)]; };
                lap = lap19(c, nb);
            } else {
                const R nb = phis[mid][hy][hx + 1] + phis[mid][hy][hx - 1] + phis[mid][hy + 1][hx]
                           + phis[mid][hy - 1][hx] + phis[hi][hy][hx] + phis[lo][hy][hx];
                lap = sub_rn(nb, mul_rn(R(6), c));
            }
            if constexpr (kKeepG)
                mus[slot][my][mx] = chem_potential_lap(dref.Phi + c, lap, m);
            else
                mus[slot][my][mx] = chem_potential_lap(c, lap, m);
        }
    };
    auto ps = [&](int zp) { return (zp - z0 + 2) % 3; };  // phi slot of plane zp (zp >= z0-2)
    auto ms = [&](int zp) { return (zp - z0 + 1) % 3; };  // mu slot of plane zp (zp >= z0-1)

    // Prologue: phi(z0-2..z0+1), mu(z0-1), mu(z0).
    phi_plane(z0 - 2, ps(z0 - 2));
    phi_plane(z0 - 1, ps(z0 - 1));
    phi_plane(z0, ps(z0));
    __syncthreads();
    mu_plane(ms(z0 - 1), ps(z0 - 2), ps(z0 - 1), ps(z0));
    __syncthreads();                // phi(z0+1) reuses the slot mu(z0-1) just read
    phi_plane(z0 + 1, ps(z0 + 1));
    __syncthreads();
    mu_plane(ms(z0), ps(z0 - 1), ps(z0), ps(z0 + 1));

    const int x = x0 + tx, y = y0 + ty;
    const int oxp = x + 1 == nx ? 1 - nx : 1, oxm = x == 0 ? nx - 1 : -1;
    const int oyp = y + 1 == ny ? (1 - ny) * nx : nx, oym = y == 0 ? (ny - 1) * nx : -nx;

    for (int k = z0; k < z1; ++k) {
        const int z = k;  // z1 <= nz
        const int s = z * plane + y * nx + x;
        const bool cok = site_ok(s, g.n, status);
        // Loads for this plane's collision issued ahead of the mu pass, after
        // the phi pass's own loads, so that their latency overlaps that work:
        // in FP32 the g re-read (an L2 hit), in the 16-bit forms (g kept in
        // shared memory) f. Other placements measured slower (kF32TopLoad).
        S gpre[Q], fpre[Q];
        auto load_g = [&]() {
#pragma unroll
            for (int i = 0; i < Q; ++i) gpre[i] = cok ? ld_l2_hint_now(gs + i * npad + s, drop_l2) : S(0);
        };
        auto load_f = [&]() {
#pragma unroll
            for (int i = 0; i < Q; ++i) fpre[i] = cok ? ld_l2_hint_now(fs + i * npad + s, drop_l2) : S(0);
        };
        if constexpr (kTopG) load_g();
        if constexpr (kTopF) load_f();
        __syncthreads();  // previous collision done with phi(k-1) and mu(k-2) slots
        phi_plane(k + 2, ps(k + 2));
        if constexpr (kMidF) load_f();
        if constexpr (kMidG) load_g();
        __syncthreads();
        mu_plane(ms(k + 1), ps(k), ps(k + 1), ps(k + 2));
        __syncthreads();

        const int ozp = z + 1 == nz ? (1 - nz) * plane : plane, ozm = z == 0 ? (nz - 1) * plane : -plane;
        const R ring_c = phis[ps(k)][ty + 2][tx + 2];  // phi, or psi in the 16-bit forms
        R ph;
        if constexpr (kKeepG)
            ph = dref.Phi + ring_c;
        else
            ph = ring_c;
        const int mc = ms(k);
        const R muc = mus[mc][ty + 1][tx + 1];
        R gmx, gmy, gmz;
        if constexpr (ISO) {
            const int mp = ms(k + 1), mm = ms(k - 1);
            auto nb = [&](int i) { return mus[cz(i) > 0 ? mp : (cz(i) < 0 ? mm : mc)][ty + 1 + cy(i)][tx + 1 + cx(i)]; };
            grad19(nb, gmx, gmy, gmz);
        } else {
            gmx = R(0.5) * (mus[mc][ty + 1][tx + 2] - mus[mc][ty + 1][tx]);
            gmy = R(0.5) * (mus[mc][ty + 2][tx + 1] - mus[mc][ty][tx + 1]);
            gmz = R(0.5) * (mus[ms(k + 1)][ty + 1][tx + 1] - mus[ms(k - 1)][ty + 1][tx + 1]);
        }
        const R Fx = -ph * gmx, Fy = -ph * gmy, Fz = -ph * gmz;
        if (phi_out && cok) {  // fields of the source state, for the adjoint
            phi_out[s] = ph;
            mu_out[s] = muc;
        }
        const unsigned long long sr_st = SR ? sr.base + (unsigned long long)s * kSrGamma : 0ull;
        unsigned long long sr_w = 0;
        auto dest = [&](int i) {
            return s + (cx(i) > 0 ? oxp : (cx(i) < 0 ? oxm : 0)) + (cy(i) > 0 ? oyp : (cy(i) < 0 ? oym : 0)) +
                   (cz(i) > 0 ? ozp : (cz(i) < 0 ? ozm : 0));
        };

        R f[Q];
        R ux, uy, uz;
        if constexpr (kKeepG) {  // deviation space
            R delta = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                f[i] = to_float(fpre[i]);
                delta += f[i];
                add_c(i, f[i], jx, jy, jz);
            }
            const R rho = dref.R + delta;
            guo_velocity(rho, jx, jy, jz, Fx, Fy, Fz, ux, uy, uz);
            collide_f_dev(f, delta, rho, ux, uy, uz, Fx, Fy, Fz, m, dref);
        } else {
            R rho = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                f[i] = Prec<P>::decode(kEarlyF ? fpre[i] : (cok ? fs[i * npad + s] : S(0)), refs[i]);
                rho += f[i];
                add_c(i, f[i], jx, jy, jz);
            }
            guo_velocity(rho, jx, jy, jz, Fx, Fy, Fz, ux, uy, uz);
            collide_f(f, rho, ux, uy, uz, Fx, Fy, Fz, m);
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const R ref = kKeepG ? R(0) : refs[i];  // deviations are stored as they are
            const int d = dest(i);
            S v;
            if constexpr (SR)
                v = Prec<P>::encode_sr(f[i], ref, sr_key(sr, sr_st, 0, i, sr_w));
            else
                v = Prec<P>::encode(f[i], ref);
            if (site_ok(d, g.n, status)) __stcs(fd + i * npad + d, v);
        }

        R gg[Q];
        if constexpr (kKeepG) {
#pragma unroll
            for (int i = 0; i < Q; ++i) gg[i] = to_float(gring[((size_t)ps(k) * Q + i) * (TY * kTX) + ty * kTX + tx]);
            collide_g_dev(gg, ring_c, ph, muc - dref.muP, ux, uy, uz, m, dref);
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const S v = kEarlyG ? gpre[i] : (cok ? ld_l2_hint(gs + i * npad + s, drop_l2) : S(0));
                gg[i] = Prec<P>::decode(v, refs[Q + i]);
            }
            collide_g(gg, ph, muc, ux, uy, uz, m);
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const R ref = kKeepG ? R(0) : refs[Q + i];
            const int d = dest(i);
            S v;
            if constexpr (SR)
                v = Prec<P>::encode_sr(gg[i], ref, sr_key(sr, sr_st, 1, i, sr_w));
            else
                v = Prec<P>::encode(gg[i], ref);
            if (site_ok(d, g.n, status)) __stcs(gd + i * npad + d, v);
        }
    }
}

constexpr int kTY = 8;

// z-chunks per tile column. Each CTA marches one chunk of the nz planes,
// chunk b spanning [chunk_begin(b), chunk_begin(b + 1)). The chunk length zc
// is the divisor of nz among 64, 32, ..., 4 that minimises
//   (zc + 4) x (columns x m / (per_sm x SMs) + 0.6),   m = nz / zc:
// each CTA pays a prologue of about four planes (four extra phi planes, two
// mu planes and the pipeline start), the m chunks of every column are spread
// over the resident CTA slots, and the tail of the launch costs about 0.6 of
// one chunk (CTAs are scheduled as slots free up, so less than a whole
// wave). The weights reproduce the measured order of the lengths (fraction of
// measured HBM): 256^3 FP32 32 (0.728) > 16 (0.718) > 8 (0.706) > 64 (0.666);
// 256^3 16-bit pairs 16 (0.545) ~ 32 (0.542) > 64 (0.519) ~ 8 (0.514); 384^3
// FP32 64 ahead of 32 and 16 (16.4 k against 15.5-15.8 k MLUPS). Chunks of
// any length (nz split into m near-equal parts) measured no faster for FP32
// and 10 % slower for the 16-bit pairs at 384^3.
int choose_chunks(int nx, int ny, int nz, int rows, int num_sms = 152, int per_sm = 2) {
    const long long cols = (long long)(nx / kTX) * (ny / rows);
    const long long slots = (long long)per_sm * num_sms;
    int best = 0;
    long long best_cost = 0;
    for (int zc = 64; zc >= 4; zc /= 2) {
        if (nz % zc) continue;
        const long long m = nz / zc;
        const long long cost = (zc + 4) * (10 * cols * m + 6 * slots);  // x 10 slots
        if (best == 0 || cost < best_cost) {
            best = (int)m;
            best_cost = cost;
        }
    }
    return best;
}

template <int P, class I, bool ISO, bool SR>
cudaError_t launch_fused(ld_ctx* c, const void* src, void* dst, void* fields) {
    using S = typename Prec<P>::store_t;
    using R = typename Prec<P>::real_t;
    constexpr size_t kRingBytes = sizeof(S) == 2 ? 3 * (size_t)Q * kTY * kTX * sizeof(S) : 0;
    cudaError_t e = set_max_dynamic_smem_once<k_step_fused<P, kTY, I, ISO, SR>>((int)kRingBytes);
    if (e != cudaSuccess) return e;
    const Geom g{c->geom.nx, c->geom.ny, c->geom.nz, c->geom.n, c->geom.npad};
    const int nchunks = choose_chunks(g.nx, g.ny, g.nz, kTY, c->num_sms, fused_ctas_per_sm<P>());
    const dim3 grid(g.nx / kTX, g.ny / kTY, nchunks);
    k_step_fused<P, kTY, I, ISO, SR><<<grid, kTX * kTY, kRingBytes, c->stream>>>(
        g, model_of<R>(c->prm), nchunks, (const S*)f_part(c, src), (const S*)g_part(c, src), (S*)f_part(c, dst),
        (S*)g_part(c, dst), c->ref, fields ? (R*)fields : nullptr, fields ? (R*)fields + c->geom.npad : nullptr,
        sr_stream(c->prm.seed, c->sr_step, c->geom.n), c->status);
    return cudaGetLastError();
}

template <int P, bool SR>
cudaError_t step_fused_r(ld_ctx* c, const void* src, void* dst, void* fields) {
    const bool small = (long long)Q * c->geom.npad <= 0x7fffffffLL;
    if (c->prm.stencil == LD_STENCIL_19)
        return small ? launch_fused<P, int, true, SR>(c, src, dst, fields)
                     : launch_fused<P, long long, true, SR>(c, src, dst, fields);
    return small ? launch_fused<P, int, false, SR>(c, src, dst, fields)
                 : launch_fused<P, long long, false, SR>(c, src, dst, fields);
}

// Stochastic rounding exists for the 16-bit forms only (it is refused at
// ld_create for the others).
template <int P>
cudaError_t step_fused_p(ld_ctx* c, const void* src, void* dst, void* fields) {
    if constexpr (Prec<P>::kDev) {
        if (c->prm.rounding == LD_ROUND_STOCHASTIC) return step_fused_r<P, true>(c, src, dst, fields);
    }
    return step_fused_r<P, false>(c, src, dst, fields);
}

}  // namespace

inline bool fused_supported_impl(int nx, int ny, int nz) {
    return nx % kTX == 0 && ny % kTY == 0 && nz >= 4 && nz % 4 == 0;
}

}  // namespace ld
