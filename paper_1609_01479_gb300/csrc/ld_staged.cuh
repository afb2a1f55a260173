// Fused single-pass step with asynchronously staged planes (FP32 and the
// 16-bit storage forms).
//
// Same decomposition and arithmetic as k_step_fused (ld_fused.cuh): a CTA of
// 256 threads owns a 32 x 8 column of sites, marches up a chunk of z-planes
// and keeps rolling phi and mu rings in shared memory. What differs is how
// the distributions reach the threads. 16-byte cp.async copies, issued by
// every thread and tracked on an mbarrier (cp.async.mbarrier.arrive.noinc),
// stage one plane ahead of use:
//   * the g box of plane k+3: 19 components x 12 rows (tile + 2-row halo in
//     y) x (32 + 2 CH) values (tile + one 16-byte chunk of halo each side in
//     x), issued once phi(k+2) is done with the box, so its latency overlaps
//     mu(k+1) and the collision of plane k. Chunks wrap periodically on
//     their own: nx is a multiple of 32, so a chunk never straddles the seam;
//   * the f tile of plane k: 19 x 8 rows x 32 values, issued at the top of
//     iteration k, so its latency overlaps the phi and mu passes.
// The phi pass then sums g from shared memory. The collision's g is read
// again with plain loads in FP32 (an L2 hit: the box copy brought those
// lines in two planes earlier under an evict-last policy); the 16-bit forms
// keep the tile's g of the last three planes in a shared-memory ring, filled
// by the phi pass.
// The 16-bit forms compute in deviation space (collide_f_dev and
// collide_g_dev in ld_common.cuh): the phi ring holds psi = sum_i h_i (phi =
// Phi + psi), each stored value enters its sum with one mixed-precision add,
// and the collisions read and write deviations without adding or removing
// the references.
//
// Every wait is bounded (max_polls try_wait polls). A wait that gives up sets
// kStatusWaitTimeout in the status word; the thread then stops waiting, lets
// its own copies land (cp.async.wait_all) and finishes its loop on whatever
// the staged buffers hold, so every thread still meets the same barriers and
// the kernel returns; the step's result is then invalid, which ld_check
// reports. `probe_wait` != 0 (a test setting, ld_test_bounded_wait) makes
// every thread also wait, once, on a third barrier that nothing arrives on:
// that wait runs out after max_polls polls with no copy tracked by it, sets
// the status bit, and the step itself completes normally.
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
    static constexpr int CH = 16 / (int)sizeof(S);   // values per 16-byte chunk
    static constexpr int BW = TX + 2 * CH, BH = TY + 4;  // g box row width, rows
    static constexpr int BCH = BW / CH;              // chunks per box row
    static constexpr int FCH = TX / CH;              // chunks per f tile row
    static constexpr int BOX_CHUNKS = Q * BH * BCH;
    static constexpr int F_CHUNKS = Q * TY * FCH;
    static constexpr bool kKeepG = sizeof(S) == 2;   // g ring of the last three planes (16-bit forms)
    static constexpr size_t OFF_BOX = 0;
    static constexpr size_t OFF_F = OFF_BOX + (size_t)Q * BH * BW * sizeof(S);
    static constexpr size_t OFF_RING = OFF_F + (size_t)Q * TY * TX * sizeof(S);
    static constexpr size_t OFF_BAR = OFF_RING + (kKeepG ? 3 * (size_t)Q * TY * TX * sizeof(S) : 0);
    static constexpr size_t BYTES = OFF_BAR + 3 * sizeof(unsigned long long);
    // static shared memory: phi and mu rings, codec references
    static constexpr size_t STATIC_BYTES =
        3 * (size_t)(TY + 4) * (TX + 4) * sizeof(R) + 3 * (size_t)(TY + 2) * (TX + 2) * sizeof(R) + 2 * Q * 4;
    static_assert(sizeof(S) == 4 || sizeof(S) == 2, "FP32 and 16-bit storage");
    static_assert(OFF_F % 16 == 0 && OFF_RING % 16 == 0 && OFF_BAR % 8 == 0, "aligned regions");
    // three CTAs per SM, each with 1 KB reserved by the hardware, in 228 KB
    static_assert(3 * (BYTES + STATIC_BYTES + 1024) <= 228 * 1024, "three CTAs per SM");
};

template <int P, class I, bool ISO, bool SR>
__global__ void __launch_bounds__(StagedLayout<P>::NT, 3)
    k_step_staged(Geom g, Model<typename Prec<P>::real_t> m, int zc, const typename Prec<P>::store_t* __restrict__ fs,
                  const typename Prec<P>::store_t* __restrict__ gs, typename Prec<P>::store_t* __restrict__ fd,
                  typename Prec<P>::store_t* __restrict__ gd, const float* __restrict__ ref_g,
                  typename Prec<P>::real_t* __restrict__ phi_out, typename Prec<P>::real_t* __restrict__ mu_out,
                  SrStream sr, int* __restrict__ status, int max_polls, int probe_wait) {
    using L = StagedLayout<P>;
    using R = typename L::R;
    using S = typename L::S;
    constexpr int TX = L::TX, TY = L::TY, NT = L::NT, CH = L::CH, BW = L::BW, BH = L::BH;
    constexpr int PW = TX + 4, PH = TY + 4;  // phi ring plane
    constexpr int MW = TX + 2, MH = TY + 2;  // mu ring plane
    constexpr bool kKeepG = L::kKeepG;
    constexpr bool kEarlyG = !kKeepG;
    __shared__ R phis[3][PH][PW];
    __shared__ R mus[3][MH][MW];
    __shared__ float refs[2 * Q];
    __shared__ DevRefs dref;  // deviation-space constants (16-bit forms)
    extern __shared__ __align__(128) unsigned char smem[];
    S* box = reinterpret_cast<S*>(smem + L::OFF_BOX);    // [Q][BH][BW], x from x0 - CH, y from y0 - 2
    S* ftile = reinterpret_cast<S*>(smem + L::OFF_F);    // [Q][TY][TX]
    S* gring = reinterpret_cast<S*>(smem + L::OFF_RING);  // [3][Q][TY][TX] (16-bit forms)
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem + L::OFF_BAR);  // box, f tile, probe
    const uint32_t bar_box = smem_addr(&bars[0]), bar_f = smem_addr(&bars[1]), bar_probe = smem_addr(&bars[2]);

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * zc;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int plane = nx * ny;
    const I npad = (I)g.npad;
    if (tid < 2 * Q) refs[tid] = ref_g[tid];
    if constexpr (kKeepG) {
        if (tid == 0) dref = dev_refs_of(ref_g, m);
    }
    if (tid == 0) {
        mbar_init(bar_box, NT);
        mbar_init(bar_f, NT);
        mbar_init(bar_probe, 1);
        fence_mbar_init();
    }
    const uint64_t keep_l2 = make_l2_evict_last_policy(), drop_l2 = make_l2_evict_first_policy();
    __syncthreads();

    unsigned phase_box = 0, phase_f = 0;
    bool alive = true;
    if (probe_wait) mbar_wait_bounded_n(bar_probe, 0, status, max_polls);  // nothing arrives: runs out
    auto wait = [&](uint32_t bar, unsigned& phase) {
        if (alive && !mbar_wait_bounded_n(bar, phase, status, max_polls)) {
            alive = false;
            cp_async_wait_all();  // this thread's copies land before anything else runs
        }
        phase ^= 1u;
    };

    // Copy assignments, fixed for the whole kernel: thread t takes the
    // (row, 16-byte column) slot t % NSLOT of a plane and the components
    // i = t / NSLOT, i + G, i + 2G, ... (G = NT / NSLOT groups of threads), so
    // a plane's copies cost one address add per component.
    constexpr int BSLOT = BH * L::BCH, BG = NT / BSLOT;  // box: slots, groups
    constexpr int FSLOT = TY * L::FCH, FG = NT / FSLOT;  // f tile
    static_assert(BG >= 1 && FG >= 1, "one copy slot per thread at most");
    const int bgrp = tid / BSLOT, fgrp = tid / FSLOT;
    int box_src = 0;
    uint32_t box_dst = 0;
    if (bgrp < BG) {
        const int slot = tid % BSLOT, r = slot / L::BCH, j = slot % L::BCH;
        int yy = y0 - 2 + r, xx = x0 - CH + j * CH;
        yy = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
        xx = xx < 0 ? xx + nx : (xx >= nx ? xx - nx : xx);
        box_src = yy * nx + xx;
        box_dst = smem_addr(box + (bgrp * BH + r) * BW + j * CH);
    }
    int f_src = 0;
    uint32_t f_dst = 0;
    if (fgrp < FG) {
        const int slot = tid % FSLOT, r = slot / L::FCH, j = slot % L::FCH;
        f_src = (y0 + r) * nx + x0 + j * CH;
        f_dst = smem_addr(ftile + (fgrp * TY + r) * TX + j * CH);
    }
    auto issue_box = [&](int zp) {
        if (bgrp < BG) {
            const int zw = zp < 0 ? zp + nz : (zp >= nz ? zp - nz : zp);
            const S* src = gs + (I)bgrp * npad + ((I)zw * plane + box_src);
            uint32_t dst = box_dst;
            for (int i = bgrp; i < Q; i += BG) {
                cp_async16(dst, src, keep_l2);
                src += (I)BG * npad;
                dst += BG * BH * BW * (int)sizeof(S);
            }
        }
        cp_async_arrive_noinc(bar_box);
    };
    auto issue_f = [&](int zp) {
        if (fgrp < FG) {
            const S* src = fs + (I)fgrp * npad + ((I)zp * plane + f_src);
            uint32_t dst = f_dst;
            for (int i = fgrp; i < Q; i += FG) {
                cp_async16(dst, src, drop_l2);
                src += (I)FG * npad;
                dst += FG * TY * TX * (int)sizeof(S);
            }
        }
        cp_async_arrive_noinc(bar_f);
    };

    // phi of plane zp over the tile + 2-halo from the box, into ring slot
    // `slot`; two x-adjacent sites per thread (216 pairs, one round). Each
    // site's sum over i keeps its order: phi is the same as in k_step_fused.
    auto phi_plane = [&](int slot) {
        constexpr int PW2 = PW / 2;
        for (int idx = tid; idx < PW2 * PH; idx += NT) {
            const int hx = 2 * (idx % PW2), hy = idx / PW2;
            const S* b = box + hy * BW + hx + (CH - 2);
            const bool interior = kKeepG && hx >= 2 && hx < TX + 2 && hy >= 2 && hy < TY + 2;
            S* keep = gring + ((size_t)slot * Q * TY + (hy - 2)) * TX + (hx - 2);
            R a0 = R(0), a1 = R(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if constexpr (sizeof(S) == 4) {
                    const float2 v = *reinterpret_cast<const float2*>(b + i * (BH * BW));
                    a0 += v.x;
                    a1 += v.y;
                } else {  // psi: the sum of the deviations
                    const unsigned v = *reinterpret_cast<const unsigned*>(b + i * (BH * BW));
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
            const R ph = kKeepG ? dref.Phi + c : c;
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

    // Prologue: phi(z0-2..z0+1), mu(z0-1), mu(z0); box of z0+2 in flight.
    issue_box(z0 - 2);
    wait(bar_box, phase_box);
    phi_plane(ps(z0 - 2));
    __syncthreads();  // box free
    issue_box(z0 - 1);
    wait(bar_box, phase_box);
    phi_plane(ps(z0 - 1));
    __syncthreads();
    issue_box(z0);
    wait(bar_box, phase_box);
    phi_plane(ps(z0));
    __syncthreads();  // phi(z0-2..z0) visible; box free
    issue_box(z0 + 1);
    mu_plane(ms(z0 - 1), ps(z0 - 2), ps(z0 - 1), ps(z0));
    wait(bar_box, phase_box);
    __syncthreads();  // phi(z0+1) reuses the slot mu(z0-1) read
    phi_plane(ps(z0 + 1));
    __syncthreads();  // phi(z0+1) visible; box free
    issue_box(z0 + 2);
    mu_plane(ms(z0), ps(z0 - 1), ps(z0), ps(z0 + 1));

    const int x = x0 + tx, y = y0 + ty;
    const int oxp = x + 1 == nx ? 1 - nx : 1, oxm = x == 0 ? nx - 1 : -1;
    const int oyp = y + 1 == ny ? (1 - ny) * nx : nx, oym = y == 0 ? (ny - 1) * nx : -nx;

    for (int k = z0; k < z0 + zc; ++k) {
        const int z = k;  // zc divides nz: k < nz
        const int s = z * plane + y * nx + x;
        // FP32: the collision's g re-read (an L2 hit) issued before the
        // passes, so that its latency overlaps them.
        S gpre[Q];
        if constexpr (kEarlyG) {
#pragma unroll
            for (int i = 0; i < Q; ++i) gpre[i] = ld_l2_hint_now(gs + (I)i * npad + s, drop_l2);
        }
        __syncthreads();  // collision k-1 done with the f tile and the ring slots of phi(k-1), mu(k-2)
        issue_f(k);
        wait(bar_box, phase_box);
        phi_plane(ps(k + 2));
        __syncthreads();  // phi(k+2) visible; box free
        if (k + 3 <= z0 + zc + 1) issue_box(k + 3);
        mu_plane(ms(k + 1), ps(k), ps(k + 1), ps(k + 2));
        wait(bar_f, phase_f);
        __syncthreads();  // mu(k+1) visible

        const int ozp = z + 1 == nz ? (1 - nz) * plane : plane, ozm = z == 0 ? (nz - 1) * plane : -plane;
        const R ring_c = phis[ps(k)][ty + 2][tx + 2];  // phi, or psi in the 16-bit forms
        const R ph = kKeepG ? dref.Phi + ring_c : ring_c;
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
        if (phi_out) {  // fields of the source state, for the adjoint
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
            const R ref = kKeepG ? R(0) : refs[i];  // deviations are stored as they are
            if constexpr (SR)
                __stcs(fd + (I)i * npad + dest(i), Prec<P>::encode_sr(f[i], ref, sr_key(sr, sr_st, 0, i, sr_w)));
            else
                __stcs(fd + (I)i * npad + dest(i), Prec<P>::encode(f[i], ref));
        }

        R gg[Q];
        if constexpr (kKeepG) {
#pragma unroll
            for (int i = 0; i < Q; ++i) gg[i] = to_float(gring[((size_t)ps(k) * Q + i) * (TY * TX) + ty * TX + tx]);
            collide_g_dev(gg, ring_c, ph, muc - dref.muP, ux, uy, uz, m, dref);
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) gg[i] = Prec<P>::decode(gpre[i], refs[Q + i]);
            collide_g(gg, ph, muc, ux, uy, uz, m);
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const R ref = kKeepG ? R(0) : refs[Q + i];
            if constexpr (SR)
                __stcs(gd + (I)i * npad + dest(i), Prec<P>::encode_sr(gg[i], ref, sr_key(sr, sr_st, 1, i, sr_w)));
            else
                __stcs(gd + (I)i * npad + dest(i), Prec<P>::encode(gg[i], ref));
        }
    }
    cp_async_wait_all();  // nothing of this CTA's is still in flight when it exits
}

template <int P>
bool staged_supported_p(int nx, int ny, int nz) {
    using L = StagedLayout<P>;
    return nx % L::TX == 0 && ny % L::TY == 0 && nz >= 4 && choose_zc(nx, ny, nz) > 0;
}

template <int P, class I, bool ISO, bool SR>
cudaError_t launch_staged(ld_ctx* c, const void* src, void* dst, void* fields) {
    using L = StagedLayout<P>;
    using S = typename L::S;
    using R = typename L::R;
    cudaError_t e = set_max_dynamic_smem_once<k_step_staged<P, I, ISO, SR>>((int)L::BYTES);
    if (e != cudaSuccess) return e;
    const Geom g{c->geom.nx, c->geom.ny, c->geom.nz, c->geom.n, c->geom.npad};
    const int zc = choose_zc(g.nx, g.ny, g.nz, c->num_sms, 3);
    const dim3 grid(g.nx / L::TX, g.ny / L::TY, g.nz / zc);
    k_step_staged<P, I, ISO, SR><<<grid, L::NT, L::BYTES, c->stream>>>(
        g, model_of<R>(c->prm), zc, (const S*)f_part(c, src), (const S*)g_part(c, src), (S*)f_part(c, dst),
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
