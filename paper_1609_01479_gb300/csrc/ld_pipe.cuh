// Fused single-pass step with TMA-staged planes (FP32 and 16-bit storage).
//
// Same decomposition as the register kernel in ld_fused.cuh -- a CTA owns a
// TX x TY column of sites and marches up a chunk of z-planes with rolling phi
// and mu rings in shared memory -- but the distributions reach shared memory
// through the copy engine (cp.async.bulk, completion counted on mbarriers),
// one plane ahead of use:
//   * the g box of each plane: 19 components x (TY+4) rows x (TX+2*CH)
//     values, i.e. the tile with a 2-row halo in y and a 16-byte chunk of
//     halo in x; rows that cross the periodic x edge are split into three
//     aligned pieces. It only feeds phi, so two boxes are resident;
//   * the f tile of each plane: 19 x TY rows x TX values (single-buffered in
//     FP32, where it is requested at the start of the plane's own iteration;
//     double-buffered one plane ahead in the 16-bit forms);
//   * 16-bit forms only: the g tile of each plane, double-buffered. In FP32
//     the collision reads its g tile with plain loads instead: the g box of
//     that plane brought those lines into L2 two iterations earlier under an
//     evict-last policy, and staging them would not fit next to the FP32
//     boxes at two CTAs per SM.
// 256-thread CTAs, two per SM, so that one CTA's barriers overlap the other's
// work. Threads compute phi (tile + 2-halo), mu (tile + 1-halo), force,
// velocity and both collisions, and push the post-collision values to
// x + c_i in the other buffer of the ping-pong pair with streaming stores.
#pragma once
#include "ld_common.cuh"
#include "ld_internal.h"
#include "ld_tma.cuh"

namespace ld {
namespace {

template <int P>
struct PipeLayout {
    using S = typename Prec<P>::store_t;
    using R = typename Prec<P>::real_t;
    static constexpr bool kStageG = sizeof(S) == 2;  // g tile staged by TMA (16-bit forms)
    static constexpr int TX = 32;
    static constexpr int TY = 8;
    static constexpr int NF = kStageG ? 2 : 1;  // f tile buffers
    static constexpr int NT = TX * TY;
    static constexpr int CH = 16 / (int)sizeof(S);  // values per 16-byte chunk
    static constexpr int BW = TX + 2 * CH;          // g box width
    static constexpr int BH = TY + 4;               // g box height
    static constexpr int GBOX = Q * BH * BW;        // values per g box
    static constexpr int FBOX = Q * TY * TX;        // values per f tile
    static constexpr int PW = TX + 4, PH = TY + 4;  // phi ring plane
    static constexpr int MW = TX + 2, MH = TY + 2;  // mu ring plane
    static constexpr size_t OFF_G = 0;
    static constexpr size_t OFF_F = OFF_G + 2 * (size_t)GBOX * sizeof(S);
    static constexpr size_t OFF_GI = OFF_F + NF * (size_t)FBOX * sizeof(S);
    static constexpr size_t OFF_PHI = OFF_GI + (kStageG ? 2 * (size_t)FBOX * sizeof(S) : 0);
    static constexpr size_t OFF_MU = OFF_PHI + 3 * (size_t)PH * PW * sizeof(R);
    static constexpr size_t OFF_REF = OFF_MU + 3 * (size_t)MH * MW * sizeof(R);
    static constexpr size_t OFF_BAR = (OFF_REF + 2 * Q * sizeof(float) + 15) / 16 * 16;
    static constexpr size_t BYTES = OFF_BAR + 6 * sizeof(unsigned long long);
    static constexpr uint32_t GBYTES = GBOX * sizeof(S);
    static constexpr uint32_t FBYTES = FBOX * sizeof(S);
    static_assert(Q * BH <= NT && Q * TY <= NT, "one copy job per thread per plane");
    static_assert((BW * sizeof(S)) % 16 == 0 && (TX * sizeof(S)) % 16 == 0, "16-byte rows");
    static_assert(OFF_F % 128 == 0 && OFF_GI % 128 == 0 && OFF_PHI % 16 == 0, "aligned boxes");
    static_assert(BYTES <= 113 * 1024, "two CTAs fit one SM's shared memory");
};

template <int P>
__global__ void __launch_bounds__(PipeLayout<P>::NT, 2)
    k_step_tma(Geom g, Model<typename Prec<P>::real_t> m, int zc, const typename Prec<P>::store_t* __restrict__ fs,
               const typename Prec<P>::store_t* __restrict__ gs, typename Prec<P>::store_t* __restrict__ fd,
               typename Prec<P>::store_t* __restrict__ gd, const float* __restrict__ ref_g, int* __restrict__ status,
               typename Prec<P>::real_t* __restrict__ phi_out, typename Prec<P>::real_t* __restrict__ mu_out) {
    using L = PipeLayout<P>;
    using S = typename L::S;
    using R = typename L::R;
    constexpr int TX = L::TX, TY = L::TY, NT = L::NT, CH = L::CH, BW = L::BW, BH = L::BH;
    constexpr int PW = L::PW, PH = L::PH, MW = L::MW, MH = L::MH;
    constexpr bool kStageG = L::kStageG;
    constexpr int NF = L::NF;
    extern __shared__ __align__(128) unsigned char smem[];
    S* G = reinterpret_cast<S*>(smem + L::OFF_G);    // [2][Q][BH][BW] g boxes (phi)
    S* F = reinterpret_cast<S*>(smem + L::OFF_F);    // [NF][Q][TY][TX] f tiles
    S* GI = reinterpret_cast<S*>(smem + L::OFF_GI);  // [2][Q][TY][TX] g tiles (16-bit forms)
    R* phis = reinterpret_cast<R*>(smem + L::OFF_PHI);  // [3][PH][PW]
    R* mus = reinterpret_cast<R*>(smem + L::OFF_MU);    // [3][MH][MW]
    float* refs = reinterpret_cast<float*>(smem + L::OFF_REF);
    // barriers: 0-1 g boxes, 2-3 f tiles, 4-5 g tiles
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem + L::OFF_BAR);

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * zc;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int plane = nx * ny;
    const long long npad = g.npad;
    const uint64_t keep_in_l2 = make_l2_evict_last_policy();

    if (tid < 2 * Q) refs[tid] = ref_g[tid];
    if (tid == 0) {
        for (int b = 0; b < 6; ++b) mbar_init(smem_addr(&bars[b]), 1);
        fence_mbar_init();
    }
    __syncthreads();

    // Barrier bookkeeping, identical in every thread: a bit per barrier for
    // "load issued, not yet waited for" and for the parity of its next phase.
    unsigned pending = 0, phase = 0;
    bool alive = true;

    auto zwrap = [&](int p) { return p < 0 ? p + nz : (p >= nz ? p - nz : p); };
    auto ywrap = [&](int y) { return y < 0 ? y + ny : (y >= ny ? y - ny : y); };
    auto gslot = [&](int p) { return (p - z0 + 2) & 1; };  // g box of plane p
    auto tslot = [&](int p) { return NF == 1 ? 0 : (p - z0) & 1; };  // f / g tiles of plane p
    auto ps = [&](int p) { return (p - z0 + 2) % 3; };     // phi ring slot
    auto ms = [&](int p) { return (p - z0 + 1) % 3; };     // mu ring slot

    auto issue_gbox = [&](int p) {
        const int s = gslot(p);
        const uint32_t bar = smem_addr(&bars[s]);
        if (tid == 0) mbar_arrive_expect_tx(bar, L::GBYTES);
        if (tid < Q * BH) {
            const int i = tid / BH, r = tid % BH;
            const S* row = gs + (long long)i * npad + (long long)zwrap(p) * plane + (long long)ywrap(y0 - 2 + r) * nx;
            const uint32_t dst = smem_addr(G + (size_t)s * L::GBOX + (size_t)(i * BH + r) * BW);
            const int xl = x0 - CH, xr = x0 + TX + CH;
            if (xl >= 0 && xr <= nx) {
                bulk_copy_g2s_hint(dst, row + xl, BW * sizeof(S), bar, keep_in_l2);
            } else {  // periodic images of the two edge chunks
                bulk_copy_g2s_hint(dst, row + (xl < 0 ? xl + nx : xl), CH * sizeof(S), bar, keep_in_l2);
                bulk_copy_g2s_hint(dst + CH * sizeof(S), row + x0, TX * sizeof(S), bar, keep_in_l2);
                const int xe = x0 + TX;
                bulk_copy_g2s_hint(dst + (CH + TX) * sizeof(S), row + (xe >= nx ? xe - nx : xe), CH * sizeof(S), bar,
                                   keep_in_l2);
            }
        }
        pending |= 1u << s;
    };
    // Tile (no halo) of plane p of `src` into `dst_base`, completing on barrier b.
    auto issue_tile = [&](const S* src_base, S* dst_base, int b, int p) {
        const uint32_t bar = smem_addr(&bars[b]);
        if (tid == 0) mbar_arrive_expect_tx(bar, L::FBYTES);
        if (tid < Q * TY) {
            const int i = tid / TY, r = tid % TY;
            const S* src = src_base + (long long)i * npad + (long long)p * plane + (long long)(y0 + r) * nx + x0;
            bulk_copy_g2s(smem_addr(dst_base + (size_t)(i * TY + r) * TX), src, TX * sizeof(S), bar);
        }
        pending |= 1u << b;
    };
    auto issue_tiles = [&](int p) {
        const int s = tslot(p);
        issue_tile(fs, F + (size_t)s * L::FBOX, 2 + s, p);
        if (kStageG) issue_tile(gs, GI + (size_t)s * L::FBOX, 4 + s, p);
    };
    auto wait_bar = [&](int b) {
        if (alive) alive = mbar_wait_bounded(smem_addr(&bars[b]), (phase >> b) & 1u, status);
        pending &= ~(1u << b);
        phase ^= 1u << b;
    };

    auto phi_plane = [&](int p) {
        const S* box = G + (size_t)gslot(p) * L::GBOX;
        R* dst = phis + ps(p) * (PH * PW);
        for (int idx = tid; idx < PH * PW; idx += NT) {
            const int hx = idx % PW, hy = idx / PW;
            const S* b = box + hy * BW + hx + (CH - 2);
            R acc = R(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) acc += Prec<P>::decode(b[i * (BH * BW)], refs[Q + i]);
            dst[idx] = acc;
        }
    };
    auto mu_plane = [&](int p) {
        const R* lo = phis + ps(p - 1) * (PH * PW);
        const R* mid = phis + ps(p) * (PH * PW);
        const R* hi = phis + ps(p + 1) * (PH * PW);
        R* dst = mus + ms(p) * (MH * MW);
        for (int idx = tid; idx < MH * MW; idx += NT) {
            const int mx = idx % MW, my = idx / MW;
            const int c = (my + 1) * PW + mx + 1;
            const R nb = mid[c + 1] + mid[c - 1] + mid[c + PW] + mid[c - PW] + hi[c] + lo[c];
            dst[idx] = chem_potential(mid[c], nb, m);
        }
    };

    // Prologue: phi(z0-2 .. z0+1), mu(z0-1), mu(z0); the g box of z0+2 and
    // the tiles of z0 in flight.
    issue_gbox(z0 - 2);
    issue_gbox(z0 - 1);
    if (NF == 2) issue_tiles(z0);
    wait_bar(gslot(z0 - 2));
    phi_plane(z0 - 2);
    __syncthreads();  // box slot of z0-2 takes z0
    issue_gbox(z0);
    wait_bar(gslot(z0 - 1));
    phi_plane(z0 - 1);
    __syncthreads();  // box slot of z0-1 takes z0+1
    issue_gbox(z0 + 1);
    wait_bar(gslot(z0));
    phi_plane(z0);
    __syncthreads();  // box slot of z0 takes z0+2; phi(z0-2..z0) visible
    issue_gbox(z0 + 2);
    mu_plane(z0 - 1);
    wait_bar(gslot(z0 + 1));
    __syncthreads();  // phi(z0+1) reuses the phi slot mu(z0-1) read
    phi_plane(z0 + 1);
    __syncthreads();
    mu_plane(z0);

    const int x = x0 + tx, y = y0 + ty;
    const int oxp = x + 1 == nx ? 1 - nx : 1, oxm = x == 0 ? nx - 1 : -1;
    const int oyp = y + 1 == ny ? (1 - ny) * nx : nx, oym = y == 0 ? (ny - 1) * nx : -nx;

    for (int k = z0; k < z0 + zc; ++k) {
        __syncthreads();  // phi(k+1) done with its box; collision k-1 done with its tiles and ring slots
        if (k + 3 <= z0 + zc + 1) issue_gbox(k + 3);
        if (NF == 1) issue_tiles(k);  // the single f buffer is free once collision k-1 is done
        else if (k + 1 < z0 + zc) issue_tiles(k + 1);
        wait_bar(gslot(k + 2));
        phi_plane(k + 2);
        __syncthreads();
        mu_plane(k + 1);
        __syncthreads();
        wait_bar(2 + tslot(k));

        const int ozp = k + 1 == nz ? (1 - nz) * plane : plane, ozm = k == 0 ? (nz - 1) * plane : -plane;
        const int s = k * plane + y * nx + x;
        const R ph = phis[ps(k) * (PH * PW) + (ty + 2) * PW + tx + 2];
        const R* mc = mus + ms(k) * (MH * MW) + (ty + 1) * MW + tx + 1;
        const R muc = mc[0];
        const R gmx = R(0.5) * (mc[1] - mc[-1]);
        const R gmy = R(0.5) * (mc[MW] - mc[-MW]);
        const R gmz = R(0.5) * (mus[ms(k + 1) * (MH * MW) + (ty + 1) * MW + tx + 1] -
                                mus[ms(k - 1) * (MH * MW) + (ty + 1) * MW + tx + 1]);
        const R Fx = -ph * gmx, Fy = -ph * gmy, Fz = -ph * gmz;
        if (phi_out) {  // fields of the source state, for the adjoint
            phi_out[s] = ph;
            mu_out[s] = muc;
        }

        const S* fb = F + (size_t)tslot(k) * L::FBOX + ty * TX + tx;
        R f[Q];
        R rho = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            f[i] = Prec<P>::decode(fb[i * (TY * TX)], refs[i]);
            rho += f[i];
            add_c(i, f[i], jx, jy, jz);
        }
        R ux, uy, uz;
        guo_velocity(rho, jx, jy, jz, Fx, Fy, Fz, ux, uy, uz);
        collide_f(f, rho, ux, uy, uz, Fx, Fy, Fz, m);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int d = s + (cx(i) > 0 ? oxp : (cx(i) < 0 ? oxm : 0)) + (cy(i) > 0 ? oyp : (cy(i) < 0 ? oym : 0)) +
                          (cz(i) > 0 ? ozp : (cz(i) < 0 ? ozm : 0));
            __stcs(fd + (long long)i * npad + d, Prec<P>::encode(f[i], refs[i]));
        }

        R gg[Q];
        if (kStageG) {
            wait_bar(4 + tslot(k));
            const S* gb = GI + (size_t)tslot(k) * L::FBOX + ty * TX + tx;
#pragma unroll
            for (int i = 0; i < Q; ++i) gg[i] = Prec<P>::decode(gb[i * (TY * TX)], refs[Q + i]);
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) gg[i] = Prec<P>::decode(__ldlu(gs + (long long)i * npad + s), refs[Q + i]);
        }
        collide_g(gg, ph, muc, ux, uy, uz, m);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int d = s + (cx(i) > 0 ? oxp : (cx(i) < 0 ? oxm : 0)) + (cy(i) > 0 ? oyp : (cy(i) < 0 ? oym : 0)) +
                          (cz(i) > 0 ? ozp : (cz(i) < 0 ? ozm : 0));
            __stcs(gd + (long long)i * npad + d, Prec<P>::encode(gg[i], refs[Q + i]));
        }
    }

    // After a failed wait, let every copy still in flight land (bounded)
    // before the CTA's shared memory is released.
    if (!alive) {
        for (int b = 0; b < 6; ++b)
            if (pending & (1u << b))
                for (int it = 0; it < kMaxWaitPolls && !mbar_try_wait(smem_addr(&bars[b]), (phase >> b) & 1u); ++it) {
                }
    }
}

// Planes per CTA: one CTA per SM is resident, and each CTA pays a prologue
// of about six planes (four extra phi planes and the first copy latency).
// Pick the divisor of nz among 64..4 that minimises
// waves x (planes per CTA + 6).
inline int pipe_zc(int cols, int nz, int num_sms) {
    int best = 0;
    long long best_cost = 0;
    for (int zc = 64; zc >= 4; zc /= 2) {
        if (nz % zc) continue;
        const long long ctas = (long long)cols * (nz / zc);
        const long long waves = (ctas + num_sms - 1) / num_sms;
        const long long cost = waves * (zc + 6);
        if (best == 0 || cost < best_cost) {
            best = zc;
            best_cost = cost;
        }
    }
    return best;
}

template <int P>
bool pipe_supported_p(int nx, int ny, int nz) {
    using L = PipeLayout<P>;
    return nx % L::TX == 0 && ny % L::TY == 0 && nz >= 4 && pipe_zc((nx / L::TX) * (ny / L::TY), nz, 1) > 0;
}

template <int P>
cudaError_t step_tma_p(ld_ctx* c, const void* src, void* dst, void* fields) {
    using L = PipeLayout<P>;
    using S = typename L::S;
    using R = typename L::R;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_step_tma<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::BYTES);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const Geom g{c->geom.nx, c->geom.ny, c->geom.nz, c->geom.n, c->geom.npad};
    const int zc = pipe_zc((g.nx / L::TX) * (g.ny / L::TY), g.nz, 2 * c->num_sms);  // two CTAs per SM
    const dim3 grid(g.nx / L::TX, g.ny / L::TY, g.nz / zc);
    k_step_tma<P><<<grid, L::NT, L::BYTES, c->stream>>>(g, model_of<R>(c->prm), zc, (const S*)f_part(c, src),
                                                        (const S*)g_part(c, src), (S*)f_part(c, dst),
                                                        (S*)g_part(c, dst), c->ref, c->status,
                                                        fields ? (R*)fields : nullptr,
                                                        fields ? (R*)fields + c->geom.npad : nullptr);
    return cudaGetLastError();
}

}  // namespace
}  // namespace ld
