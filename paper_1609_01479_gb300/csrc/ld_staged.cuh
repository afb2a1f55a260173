// Fused single-pass step with the f tile staged asynchronously (FP32 and
// the 16-bit storage forms).
//
// Same decomposition, passes and arithmetic as k_step_fused (ld_fused.cuh):
// a CTA of 256 threads owns a 32 x 8 column of sites, marches up a chunk of
// z-planes, computes phi(k+2) over the tile + 2-halo from global loads into
// a rolling ring, mu(k+1), then collides plane k and pushes it. What differs
// is how the collision gets its f: every thread issues 16-byte cp.async
// copies of the tile's f of plane k at the top of iteration k (19 x 8 rows x
// 32 values into shared memory; each thread owns fixed 16-byte slots, so a
// plane costs one address add per component), and waits for its own copies
// (cp.async.wait_group, a hardware wait that ends when they land) before
// the barrier that precedes the collision. Their latency overlaps the phi
// and mu passes without holding registers. FP32 re-reads g with early
// register loads and the 16-bit forms keep the tile's g in a ring, as in
// k_step_fused; the 16-bit forms compute in deviation space.
// Measured against k_step_fused it is slower (FP32 0.69 against 0.74 of the
// measured HBM roofline at 384^3): the staged tile takes shared memory from
// L1, where the collision's second read of g partly hits.
//
// The kernel has one spin-wait, bounded: with `probe_wait` != 0 (a test
// setting, ld_test_bounded_wait) every thread also waits, once, on an
// mbarrier that nothing arrives on and that tracks no copy; that wait gives
// up after max_polls polls, sets kStatusWaitTimeout in the status word
// (ld_check reports it) and the step completes normally.
// Template only: instantiated for FP32, FP16-dev and BF16-dev by ld_prec_lp.cu.
#pragma once
#include "ld_async.cuh"
#include "ld_common.cuh"
#include "ld_fused.cuh"
#include "ld_internal.h"

namespace ld {
namespace {

template <int P>
struct StagedLayout {
    using S = typename Prec<P>::store_t;
    using R = typename Prec<P>::real_t;
    static constexpr int TX = 32, TY = 8, NT = TX * TY;
    static constexpr int CH = 16 / (int)sizeof(S);  // values per 16-byte chunk
    static constexpr int FCH = TX / CH;             // chunks per f tile row
    static constexpr bool kDev = sizeof(S) == 2;    // deviation-space arithmetic and g ring (16-bit forms)
    static constexpr size_t OFF_F = 0;
    static constexpr size_t OFF_RING = OFF_F + (size_t)Q * TY * TX * sizeof(S);
    static constexpr size_t OFF_BAR = OFF_RING + (kDev ? 3 * (size_t)Q * TY * TX * sizeof(S) : 0);
    static constexpr size_t BYTES = OFF_BAR + sizeof(unsigned long long);
    // static shared memory: phi and mu rings, codec references, deviation constants
    static constexpr size_t STATIC_BYTES = 3 * (size_t)(TY + 4) * (TX + 4) * sizeof(R) +
                                           3 * (size_t)(TY + 2) * (TX + 2) * sizeof(R) + 2 * Q * 4 + 64;
    static_assert(sizeof(S) == 4 || sizeof(S) == 2, "FP32 and 16-bit storage");
    static_assert(OFF_RING % 16 == 0 && OFF_BAR % 8 == 0, "aligned regions");
    // three CTAs per SM, each with 1 KB reserved by the hardware, in 228 KB
    static_assert(3 * (BYTES + STATIC_BYTES + 1024) <= 228 * 1024, "three CTAs per SM");
};

template <int P, class I, bool ISO, bool SR>
__global__ void __launch_bounds__(StagedLayout<P>::NT, 3)
    k_step_staged(Geom g, Model<typename Prec<P>::real_t> m, int nchunks, const typename Prec<P>::store_t* __restrict__ fs,
                  const typename Prec<P>::store_t* __restrict__ gs, typename Prec<P>::store_t* __restrict__ fd,
                  typename Prec<P>::store_t* __restrict__ gd, const float* __restrict__ ref_g,
                  typename Prec<P>::real_t* __restrict__ phi_out, typename Prec<P>::real_t* __restrict__ mu_out,
                  SrStream sr, int* __restrict__ status, int max_polls, int probe_wait) {
    using L = StagedLayout<P>;
    using R = typename L::R;
    using S = typename L::S;
    constexpr int TX = L::TX, TY = L::TY, NT = L::NT, CH = L::CH;
    constexpr int PW = TX + 4, PH = TY + 4;  // phi ring plane
    constexpr int MW = TX + 2, MH = TY + 2;  // mu ring plane
    constexpr bool kDev = L::kDev;
    __shared__ R phis[3][PH][PW];
    __shared__ R mus[3][MH][MW];
    __shared__ float refs[2 * Q];
    __shared__ DevRefs dref;  // deviation-space constants (16-bit forms)
    extern __shared__ __align__(128) unsigned char smem[];
    S* ftile = reinterpret_cast<S*>(smem + L::OFF_F);    // [Q][TY][TX]
    S* gring = reinterpret_cast<S*>(smem + L::OFF_RING);  // [3][Q][TY][TX] (16-bit forms)
    unsigned long long* bar_probe_p = reinterpret_cast<unsigned long long*>(smem + L::OFF_BAR);

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = chunk_begin(blockIdx.z, g.nz, nchunks), z1 = chunk_begin(blockIdx.z + 1, g.nz, nchunks);
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int plane = nx * ny;
    const I npad = (I)g.npad;
    if (tid < 2 * Q) refs[tid] = ref_g[tid];
    if constexpr (kDev) {
        if (tid == 0) dref = dev_refs_of(ref_g, m);
    }
    if (tid == 0 && probe_wait) {
        mbar_init(smem_addr(bar_probe_p), 1);
        fence_mbar_init();
    }
    const uint64_t keep_l2 = make_l2_evict_last_policy(), drop_l2 = make_l2_evict_first_policy();
    __syncthreads();
    if (probe_wait) mbar_wait_bounded_n(smem_addr(bar_probe_p), 0, status, max_polls);  // nothing arrives: runs out

    // f tile copies: thread t owns the (row, 16-byte column) slot t % FSLOT of
    // a plane and the components t / FSLOT, + FG, + 2 FG, ...
    constexpr int FSLOT = TY * L::FCH, FG = NT / FSLOT;
    static_assert(FG >= 1, "one copy slot per thread at most");
    const int fgrp = tid / FSLOT;
    int f_src = 0;
    uint32_t f_dst = 0;
    if (fgrp < FG) {
        const int slot = tid % FSLOT, r = slot / L::FCH, j = slot % L::FCH;
        f_src = (y0 + r) * nx + x0 + j * CH;
        f_dst = smem_addr(ftile + (fgrp * TY + r) * TX + j * CH);
    }
    auto issue_f = [&](int zp) {
        if (fgrp < FG && site_ok((long long)zp * plane + f_src + CH - 1, g.n, status)) {
            const S* src = fs + (I)fgrp * npad + ((I)zp * plane + f_src);
            uint32_t dst = f_dst;
            for (int i = fgrp; i < Q; i += FG) {
                cp_async16(dst, src, drop_l2);
                src += (I)FG * npad;
                dst += FG * TY * TX * (int)sizeof(S);
            }
        }
    };

    // phi of plane zp over the tile + 2-halo into ring slot `slot` (16-bit
    // forms: psi = phi - Phi), from global memory with evict-last loads (the
    // collision reads g again two planes later); two x-adjacent sites per
    // thread from paired loads (216 pairs, one round). Each site's sum over i
    // keeps its order: phi is the same as in k_step_fused.
    auto phi_plane = [&](int zp, int slot) {
        constexpr int PW2 = PW / 2;
        const int zoff = wrap_once(zp, nz) * plane;
        for (int idx = tid; idx < PW2 * PH; idx += NT) {
            const int hx = 2 * (idx % PW2), hy = idx / PW2;
            const int sg = zoff + wrap_once(y0 + hy - 2, ny) * nx + wrap_once(x0 + hx - 2, nx);  // even
            const bool sok = site_ok(sg, g.n, status) && site_ok(sg + 1, g.n, status);
            const bool interior = kDev && hx >= 2 && hx < TX + 2 && hy >= 2 && hy < TY + 2;
            S* keep = gring + ((size_t)slot * Q * TY + (hy - 2)) * TX + (hx - 2);
            R a0 = R(0), a1 = R(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if constexpr (sizeof(S) == 4) {
                    const float2 v = sok ? ld_l2_hint_pair(gs + (I)i * npad + sg, keep_l2) : make_float2(0.f, 0.f);
                    a0 += v.x;
                    a1 += v.y;
                } else {
                    const unsigned v = sok ? ld_l2_hint_pair(gs + (I)i * npad + sg, keep_l2) : 0u;
                    if constexpr (P == LD_FP16DEV) {
                        a0 = add_f16(a0, (unsigned short)(v & 0xffffu));
                        a1 = add_f16(a1, (unsigned short)(v >> 16));
                    } else {
                        a0 = add_bf16(a0, (unsigned short)(v & 0xffffu));
                        a1 = add_bf16(a1, (unsigned short)(v >> 16));
                    }
                    if (interior) *reinterpret_cast<unsigned*>(keep + i * (TY * TX)) = v;
                }
            }
            phis[slot][hy][hx] = a0;
            phis[slot][hy][hx + 1] = a1;
        }
    };
    auto mu_plane = [&](int slot, int lo, int mid, int hi) {
        for (int idx = tid; idx < MW * MH; idx += NT) {
            const int mx = idx % MW, my = idx / MW;
            const int hx = mx + 1, hy = my + 1;
            // the ring holds phi (FP32) or psi = phi - Phi (16-bit forms): the
            // Laplacian is the same, the cubic term takes phi
            const R c = phis[mid][hy][hx];
            const R ph = kDev ? dref.Phi + c : c;
            R lap;
            if constexpr (ISO) {
                auto nb = [&](int i) { return phis[cz(i) > 0 ? hi : (cz(i) < 0 ? lo : mid)][hy + cy(i)][hx + cx(i)]; };
                lap = lap19(c, nb);
            } else {
                const R nb = phis[mid][hy][hx + 1] + phis[mid][hy][hx - 1] + phis[mid][hy + 1][hx]
                           + phis[mid][hy - 1][hx] + phis[hi][hy][hx] + phis[lo][hy][hx];
                lap = sub_rn(nb, mul_rn(R(6), c));
            }
            mus[slot][my][mx] = chem_potential_lap(ph, lap, m);
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
    __syncthreads();  // phi(z0+1) reuses the slot mu(z0-1) just read
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
        // FP32: the collision's g re-read (an L2 hit) issued before the
        // passes, so that its latency overlaps them.
        S gpre[Q];
        if constexpr (!kDev) {
#pragma unroll
            for (int i = 0; i < Q; ++i) gpre[i] = cok ? ld_l2_hint_now(gs + (I)i * npad + s, drop_l2) : S(0);
        }
        __syncthreads();  // collision k-1 done with the f tile and the ring slots of phi(k-1), mu(k-2)
        issue_f(k);
        cp_async_commit();
        phi_plane(k + 2, ps(k + 2));
        __syncthreads();
        mu_plane(ms(k + 1), ps(k), ps(k + 1), ps(k + 2));
        cp_async_wait_group0();  // this thread's f copies have landed
        __syncthreads();         // mu(k+1) and every thread's f copies visible

        const int ozp = z + 1 == nz ? (1 - nz) * plane : plane, ozm = z == 0 ? (nz - 1) * plane : -plane;
        const R ring_c = phis[ps(k)][ty + 2][tx + 2];  // phi, or psi in the 16-bit forms
        const R ph = kDev ? dref.Phi + ring_c : ring_c;
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
        if constexpr (kDev) {  // deviation space
            R delta = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                f[i] = to_float(ftile[(i * TY + ty) * TX + tx]);
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
                f[i] = Prec<P>::decode(ftile[(i * TY + ty) * TX + tx], refs[i]);
                rho += f[i];
                add_c(i, f[i], jx, jy, jz);
            }
            guo_velocity(rho, jx, jy, jz, Fx, Fy, Fz, ux, uy, uz);
            collide_f(f, rho, ux, uy, uz, Fx, Fy, Fz, m);
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const R ref = kDev ? R(0) : refs[i];  // deviations are stored as they are
            const int d = dest(i);
            S v;
            if constexpr (SR)
                v = Prec<P>::encode_sr(f[i], ref, sr_key(sr, sr_st, 0, i, sr_w));
            else
                v = Prec<P>::encode(f[i], ref);
            if (site_ok(d, g.n, status)) __stcs(fd + (I)i * npad + d, v);
        }

        R gg[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const S v = kDev ? gring[((size_t)ps(k) * Q + i) * (TY * TX) + ty * TX + tx] : gpre[i];
            gg[i] = kDev ? to_float(v) : Prec<P>::decode(v, refs[Q + i]);
        }
        if constexpr (kDev)
            collide_g_dev(gg, ring_c, ph, muc - dref.muP, ux, uy, uz, m, dref);
        else
            collide_g(gg, ph, muc, ux, uy, uz, m);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const R ref = kDev ? R(0) : refs[Q + i];
            const int d = dest(i);
            S v;
            if constexpr (SR)
                v = Prec<P>::encode_sr(gg[i], ref, sr_key(sr, sr_st, 1, i, sr_w));
            else
                v = Prec<P>::encode(gg[i], ref);
            if (site_ok(d, g.n, status)) __stcs(gd + (I)i * npad + d, v);
        }
    }
}

template <int P>
bool staged_supported_p(int nx, int ny, int nz) {
    using L = StagedLayout<P>;
    return nx % L::TX == 0 && ny % L::TY == 0 && nz >= 4 && nz % 4 == 0;
}

template <int P, class I, bool ISO, bool SR>
cudaError_t launch_staged(ld_ctx* c, const void* src, void* dst, void* fields) {
    using L = StagedLayout<P>;
    using S = typename L::S;
    using R = typename L::R;
    cudaError_t e = set_max_dynamic_smem_once<k_step_staged<P, I, ISO, SR>>((int)L::BYTES);
    if (e != cudaSuccess) return e;
    const Geom g{c->geom.nx, c->geom.ny, c->geom.nz, c->geom.n, c->geom.npad};
    const int nchunks = choose_chunks(g.nx, g.ny, g.nz, L::TY, c->num_sms, 3);
    const dim3 grid(g.nx / L::TX, g.ny / L::TY, nchunks);
    k_step_staged<P, I, ISO, SR><<<grid, L::NT, L::BYTES, c->stream>>>(
        g, model_of<R>(c->prm), nchunks, (const S*)f_part(c, src), (const S*)g_part(c, src), (S*)f_part(c, dst),
        (S*)g_part(c, dst), c->ref, fields ? (R*)fields : nullptr, fields ? (R*)fields + c->geom.npad : nullptr,
        sr_stream(c->prm.seed, c->sr_step, c->geom.n), c->status, c->wait_polls, c->wait_probe);
    return cudaGetLastError();
}

template <int P, bool SR>
cudaError_t step_staged_r(ld_ctx* c, const void* src, void* dst, void* fields) {
    const bool small = (long long)Q * c->geom.npad <= 0x7fffffffLL;
    if (c->prm.stencil == LD_STENCIL_19)
        return small ? launch_staged<P, int, true, SR>(c, src, dst, fields)
                     : launch_staged<P, long long, true, SR>(c, src, dst, fields);
    return small ? launch_staged<P, int, false, SR>(c, src, dst, fields)
                 : launch_staged<P, long long, false, SR>(c, src, dst, fields);
}

template <int P>
cudaError_t step_staged_p(ld_ctx* c, const void* src, void* dst, void* fields) {
    if constexpr (Prec<P>::kDev) {
        if (c->prm.rounding == LD_ROUND_STOCHASTIC) return step_staged_r<P, true>(c, src, dst, fields);
    }
    return step_staged_r<P, false>(c, src, dst, fields);
}

}  // namespace
}  // namespace ld
