// Fused single-pass step for the 16-bit deviation forms with two sites per
// thread and packed FP32 arithmetic.
//
// The decomposition is k_step_fused's (ld_fused.cuh): a CTA owns a 32 x 8
// column of sites and marches up a chunk of z-planes with rolling phi/psi
// and mu rings and a ring of the tile's g of the last three planes in shared
// memory. Here the CTA has 128 threads and each thread collides two
// x-adjacent sites (x, x + 1; x even). Their values travel together:
//   * one 32-bit load (or shared-memory read) brings the pair's deviations
//     of one direction, converted to a float2 in one step;
//   * the moments, the velocity and both collisions run on float2 values
//     with the packed FP32 instructions of sm_100 and later (__ffma2_rn,
//     __fadd2_rn, __fmul2_rn and sub.rn.f32x2: one instruction for both
//     sites), in deviation space as collide_f_dev / collide_g_dev;
//   * the 9 directions with c_x = 0 push both sites to one aligned pair of
//     the destination and store them with one 32-bit store of two rounded
//     16-bit values; the 10 with c_x != 0 are stored value by value.
// Each site sees the same operations as in collide_f_dev / collide_g_dev,
// except that the packed forms fix where a product and a sum fuse (the
// scalar kernel leaves that to the compiler); the results agree within FP32
// rounding. Round to nearest only (stochastic rounding runs k_step_fused).
// The same scheme for FP32 storage measured slower than k_step_fused (0.68 of
// the HBM roofline at 384^3 against 0.74): FP32 is bound by memory latency
// rather than by instructions, and two sites' values in registers leave a
// thread 128 registers, 16 warps per SM.
// Template only: instantiated for FP16-dev and BF16-dev by ld_prec_lp.cu.
#pragma once
#include "ld_async.cuh"
#include "ld_common.cuh"
#include "ld_fused.cuh"
#include "ld_internal.h"

namespace ld {
namespace {

// Packed FP32 pairs: both lanes rounded once, as two scalar operations would be.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;"
        : "=l"(r)
        : "l"(*reinterpret_cast<const unsigned long long*>(&a)), "l"(*reinterpret_cast<const unsigned long long*>(&b)));
    return *reinterpret_cast<const float2*>(&r);
}

// c_i . (ax, ay, az) for the first direction of an opposite pair (odd i):
// every such c_i has a +1 first nonzero component, so only adds and subtracts.
__device__ __forceinline__ float2 cdot2(int i, float2 ax, float2 ay, float2 az) {
    float2 s;
    bool any = false;
    if (cx(i) != 0) {
        s = ax;
        any = true;
    }
    if (cy(i) != 0) {
        s = any ? (cy(i) > 0 ? add2(s, ay) : sub2(s, ay)) : ay;
        any = true;
    }
    if (cz(i) != 0) s = any ? (cz(i) > 0 ? add2(s, az) : sub2(s, az)) : az;
    return s;
}

// j += v c_i, both lanes.
__device__ __forceinline__ void add_c2(int i, float2 v, float2& jx, float2& jy, float2& jz) {
    if (cx(i) > 0) jx = add2(jx, v);
    if (cx(i) < 0) jx = sub2(jx, v);
    if (cy(i) > 0) jy = add2(jy, v);
    if (cy(i) < 0) jy = sub2(jy, v);
    if (cz(i) > 0) jz = add2(jz, v);
    if (cz(i) < 0) jz = sub2(jz, v);
}

// collide_f_dev on a pair of sites. get(i) gives the pair's deviations of
// direction i, put(i, v) takes the collided ones; each opposite pair is read,
// collided and handed on before the next, so few values are live at once.
template <class Get, class Put>
__device__ __forceinline__ void collide_f_dev2(Get get, Put put, float2 delta, float2 rho, float2 ux, float2 uy,
                                               float2 uz, float2 Fx, float2 Fy, float2 Fz, const Model<float>& m,
                                               const DevRefs& d) {
    const float2 uu = fma2(ux, ux, fma2(uy, uy, mul2(uz, uz)));
    const float2 uF = fma2(ux, Fx, fma2(uy, Fy, mul2(uz, Fz)));
    const float2 keep = f2(1.0f - m.omega_f), om = f2(m.omega_f);
    const float2 m15uu = mul2(f2(-1.5f), uu);
    float2 moving = f2(0.0f);
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const float w = wgt<float>(i), pw = m.force_pre * w;
        const float2 cu = cdot2(i, ux, uy, uz);
        const float2 cF = cdot2(i, Fx, Fy, Fz);
        const float2 wr = mul2(f2(w), rho);
        const float2 eq_sym = fma2(wr, fma2(f2(4.5f), mul2(cu, cu), m15uu), fma2(f2(w), delta, f2(d.ef[dir_class(i)])));
        const float2 eq_anti = mul2(mul2(f2(3.0f), wr), cu);
        const float2 src_sym = fma2(f2(9.0f * pw), mul2(cu, cF), mul2(f2(-3.0f * pw), uF));
        const float2 src_anti = mul2(f2(3.0f * pw), cF);
        const float2 sym = fma2(om, eq_sym, src_sym);
        const float2 anti = fma2(om, eq_anti, src_anti);
        put(i, fma2(keep, get(i), add2(sym, anti)));
        put(i + 1, fma2(keep, get(i + 1), sub2(sym, anti)));
        moving = add2(moving, eq_sym);
    }
    const float2 eq0 = fma2(f2(-2.0f), moving, delta);
    const float2 src0 = mul2(f2(m.force_pre * wgt<float>(0) * -3.0f), uF);
    put(0, fma2(keep, get(0), fma2(om, eq0, src0)));
}

// collide_g_dev on a pair of sites, with get/put as in collide_f_dev2.
template <class Get, class Put>
__device__ __forceinline__ void collide_g_dev2(Get get, Put put, float2 psi, float2 phi, float2 dmu, float2 ux,
                                               float2 uy, float2 uz, const Model<float>& m, const DevRefs& d) {
    const float2 uu = fma2(ux, ux, fma2(uy, uy, mul2(uz, uz)));
    const float2 ddev = fma2(f2(m.Gamma), dmu, mul2(f2(-1.0f / 3.0f), psi));  // dev - dhat
    const float2 base = fma2(f2(-1.5f), mul2(phi, uu), psi);
    const float2 keep = f2(1.0f - m.omega_g), om = f2(m.omega_g);
    const float2 phi45 = mul2(f2(4.5f), phi);
    float2 moving = f2(0.0f);
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const float w = wgt<float>(i);
        const float2 cu = cdot2(i, ux, uy, uz);
        float2 inner = fma2(phi45, mul2(cu, cu), base);
        if (c2(i) == 2) inner = fma2(f2(4.5f), ddev, inner);  // (|c_i|^2 - 1) = 1 for the diagonals, 0 on the axes
        const float2 eq_sym = fma2(f2(w), inner, f2(d.eg[dir_class(i)]));
        const float2 eq_anti = mul2(mul2(f2(3.0f * w), phi), cu);
        const float2 sym = mul2(om, eq_sym), anti = mul2(om, eq_anti);
        put(i, fma2(keep, get(i), add2(sym, anti)));
        put(i + 1, fma2(keep, get(i + 1), sub2(sym, anti)));
        moving = add2(moving, eq_sym);
    }
    const float2 eq0 = fma2(f2(-2.0f), moving, psi);
    put(0, fma2(keep, get(0), mul2(om, eq0)));
}

// Two 16-bit values <-> float2 (low half = the lower address).
template <int P>
__device__ __forceinline__ float2 unpack2(unsigned v) {
    if constexpr (P == LD_FP16DEV) {
        __half2 h;
        memcpy(&h, &v, 4);
        return __half22float2(h);
    } else {
        __nv_bfloat162 b;
        memcpy(&b, &v, 4);
        return __bfloat1622float2(b);
    }
}
template <int P>
__device__ __forceinline__ unsigned pack2(float2 a) {
    unsigned v;
    if constexpr (P == LD_FP16DEV) {
        const __half2 h = __float22half2_rn(a);
        memcpy(&v, &h, 4);
    } else {
        const __nv_bfloat162 b = __float22bfloat162_rn(a);
        memcpy(&v, &b, 4);
    }
    return v;
}

// CTAs of 16 x TY threads (16 pairs x TY rows of a 32 x TY tile); resident
// CTAs per SM chosen so that a thread has 128 registers (fewer spill).
// Issue the plane's f loads before the psi pass (true) or after its own loads
// (false), to be used after the mu pass.
constexpr bool kPairFBeforePhi = false;
// The psi pass on four-site quads (one round of 8-byte loads for 128 threads)
// rather than pairs (two rounds of 4-byte loads), per storage form. Measured
// at 384^3 / 256^3 (fraction of HBM): BF16-dev 0.593 / 0.578 with quads
// against 0.568 / 0.539; FP16-dev 0.563 / 0.548 against 0.569 / 0.538 (its
// quad kernel keeps a 12-byte spill at 128 registers).
template <int P>
__host__ __device__ constexpr bool phi_quads() {
    return P == LD_BF16DEV;
}

template <int TY>
constexpr int pair_ctas_per_sm() {
    return TY == 8 ? 4 : 2;
}

template <int P, class I, bool ISO, int TY, bool SR = false>
__global__ void __launch_bounds__(16 * TY, pair_ctas_per_sm<TY>())
    k_step_fused2(Geom g, Model<float> m, int nchunks, const typename Prec<P>::store_t* __restrict__ fs,
                  const typename Prec<P>::store_t* __restrict__ gs, typename Prec<P>::store_t* __restrict__ fd,
                  typename Prec<P>::store_t* __restrict__ gd, const float* __restrict__ ref_g,
                  float* __restrict__ phi_out, float* __restrict__ mu_out, SrStream sr, int* __restrict__ status) {
    using S = typename Prec<P>::store_t;
    static_assert(sizeof(S) == 2, "16-bit deviation forms");
    constexpr int TX = kTX, NT = 16 * TY;
    constexpr int PW = TX + 4, PH = TY + 4;  // psi ring plane
    constexpr int MW = TX + 2, MH = TY + 2;  // mu ring plane
    __shared__ float phis[3][PH][PW];        // psi = phi - Phi
    __shared__ float mus[3][MH][MW];
    __shared__ DevRefs dref;
    extern __shared__ __align__(16) unsigned char keep_smem[];
    S* gring = reinterpret_cast<S*>(keep_smem);  // [3][Q][TY][TX], slot = psi slot of the plane

    const int tid = threadIdx.x;
    const int tp = tid % (TX / 2), ty = tid / (TX / 2);
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = chunk_begin(blockIdx.z, g.nz, nchunks), z1 = chunk_begin(blockIdx.z + 1, g.nz, nchunks);
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int plane = nx * ny;
    const I npad = (I)g.npad;
    if (tid == 0) dref = dev_refs_of(ref_g, m);
    const uint64_t keep_l2 = make_l2_evict_last_policy(), drop_l2 = make_l2_evict_first_policy();
    __syncthreads();

    // psi of plane zp over the tile + 2-halo: two x-adjacent sites from one
    // 32-bit load per direction; the tile's own pairs also go to the g ring.
    auto phi_plane = [&](int zp, int slot) {
        const int zoff = wrap_once(zp, nz) * plane;
        if constexpr (phi_quads<P>()) {
            // four x-adjacent sites from one 8-byte load per direction, over
            // x0-4 .. x0+TX+3 (quads aligned to four sites; the outermost
            // two sites on each side are loaded and not kept)
            constexpr int QQ = (TX + 8) / 4;
            for (int idx = tid; idx < QQ * PH; idx += NT) {
                const int qx = 4 * (idx % QQ), hy = idx / QQ;
                const int s = zoff + wrap_once(y0 + hy - 2, ny) * nx + wrap_once(x0 + qx - 4, nx);  // multiple of 4
                const bool sok = site_ok(s, g.n, status) && site_ok(s + 3, g.n, status);
                const bool interior = qx >= 4 && qx < TX + 4 && hy >= 2 && hy < TY + 2;
                S* keep = gring + ((size_t)slot * Q * TY + (hy - 2)) * TX + (qx - 4);
                float a[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const uint2 v = sok ? ld_l2_hint_quad(gs + i * npad + s, keep_l2) : make_uint2(0u, 0u);
                    const unsigned short h[4] = {(unsigned short)(v.x & 0xffffu), (unsigned short)(v.x >> 16),
                                                 (unsigned short)(v.y & 0xffffu), (unsigned short)(v.y >> 16)};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if constexpr (P == LD_FP16DEV)
                            a[j] = add_f16(a[j], h[j]);
                        else
                            a[j] = add_bf16(a[j], h[j]);
                    }
                    if (interior) *reinterpret_cast<uint2*>(keep + i * (TY * TX)) = v;
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int hx = qx - 2 + j;  // psi frame: x0-2 .. x0+TX+1
                    if (hx >= 0 && hx < PW) phis[slot][hy][hx] = a[j];
                }
            }
            return;
        }
        constexpr int PW2 = PW / 2;
        for (int idx = tid; idx < PW2 * PH; idx += NT) {
            const int hx = 2 * (idx % PW2), hy = idx / PW2;
            const int s = zoff + wrap_once(y0 + hy - 2, ny) * nx + wrap_once(x0 + hx - 2, nx);  // even
            const bool sok = site_ok(s, g.n, status) && site_ok(s + 1, g.n, status);
            const bool interior = hx >= 2 && hx < TX + 2 && hy >= 2 && hy < TY + 2;
            S* keep = gring + ((size_t)slot * Q * TY + (hy - 2)) * TX + (hx - 2);
            float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const unsigned v = sok ? ld_l2_hint_pair(gs + i * npad + s, keep_l2) : 0u;
                if constexpr (P == LD_FP16DEV) {
                    a0 = add_f16(a0, (unsigned short)(v & 0xffffu));
                    a1 = add_f16(a1, (unsigned short)(v >> 16));
                } else {
                    a0 = add_bf16(a0, (unsigned short)(v & 0xffffu));
                    a1 = add_bf16(a1, (unsigned short)(v >> 16));
                }
                if (interior) *reinterpret_cast<unsigned*>(keep + i * (TY * TX)) = v;
            }
            phis[slot][hy][hx] = a0;
            phis[slot][hy][hx + 1] = a1;
        }
    };
    auto mu_plane = [&](int slot, int lo, int mid, int hi) {
        for (int idx = tid; idx < MW * MH; idx += NT) {
            const int mx = idx % MW, my = idx / MW;
            const int hx = mx + 1, hy = my + 1;
            const float c = phis[mid][hy][hx];
            float lap;
            if constexpr (ISO) {
                auto nb = [&](int i) { return phis[cz(i) > 0 ? hi : (cz(i) < 0 ? lo : mid)][hy + cy(i)][hx + cx(i)]; };
                lap = lap19(c, nb);
            } else {
                const float nb = phis[mid][hy][hx + 1] + phis[mid][hy][hx - 1] + phis[mid][hy + 1][hx]
                               + phis[mid][hy - 1][hx] + phis[hi][hy][hx] + phis[lo][hy][hx];
                lap = sub_rn(nb, mul_rn(6.0f, c));
            }
            mus[slot][my][mx] = chem_potential_lap(dref.Phi + c, lap, m);
        }
    };
    auto ps = [&](int zp) { return (zp - z0 + 2) % 3; };
    auto ms = [&](int zp) { return (zp - z0 + 1) % 3; };

    phi_plane(z0 - 2, ps(z0 - 2));
    phi_plane(z0 - 1, ps(z0 - 1));
    phi_plane(z0, ps(z0));
    __syncthreads();
    mu_plane(ms(z0 - 1), ps(z0 - 2), ps(z0 - 1), ps(z0));
    __syncthreads();  // psi(z0+1) reuses the slot mu(z0-1) just read
    phi_plane(z0 + 1, ps(z0 + 1));
    __syncthreads();
    mu_plane(ms(z0), ps(z0 - 1), ps(z0), ps(z0 + 1));

    const int tx = 2 * tp;  // the pair's first column in the tile
    const int x = x0 + tx, y = y0 + ty;
    // x is even and nx is even: x + 1 never wraps; x - 1 wraps when x = 0,
    // x + 2 when x + 2 = nx
    const int oxm0 = x == 0 ? nx - 1 : -1, oxp1 = x + 2 == nx ? 1 - nx : 1;
    const int oyp = y + 1 == ny ? (1 - ny) * nx : nx, oym = y == 0 ? (ny - 1) * nx : -nx;

    for (int k = z0; k < z1; ++k) {
        const int z = k;
        const int s = z * plane + y * nx + x;  // even: the pair (s, s + 1)
        const bool cok = site_ok(s, g.n, status) && site_ok(s + 1, g.n, status);
        unsigned fpre[Q];  // issued before or after the psi pass's own loads, used after the mu pass
        auto load_f = [&]() {
#pragma unroll
            for (int i = 0; i < Q; ++i) fpre[i] = cok ? ld_l2_hint_pair_now(fs + i * npad + s, drop_l2) : 0u;
        };
        if constexpr (kPairFBeforePhi) load_f();
        __syncthreads();  // previous collision done with psi(k-1) and mu(k-2) slots
        phi_plane(k + 2, ps(k + 2));
        if constexpr (!kPairFBeforePhi) load_f();
        __syncthreads();
        mu_plane(ms(k + 1), ps(k), ps(k + 1), ps(k + 2));
        __syncthreads();

        const int ozp = z + 1 == nz ? (1 - nz) * plane : plane, ozm = z == 0 ? (nz - 1) * plane : -plane;
        // per site: phi, mu, the force
        float2 psi, ph, muc, Fx, Fy, Fz;
        {
            const int mc = ms(k), mp = ms(k + 1), mm = ms(k - 1);
            float gx[2], gy[2], gz[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int cxl = tx + e;
                if constexpr (ISO) {
                    auto nb = [&](int i) {
                        return mus[cz(i) > 0 ? mp : (cz(i) < 0 ? mm : mc)][ty + 1 + cy(i)][cxl + 1 + cx(i)];
                    };
                    grad19(nb, gx[e], gy[e], gz[e]);
                } else {
                    gx[e] = 0.5f * (mus[mc][ty + 1][cxl + 2] - mus[mc][ty + 1][cxl]);
                    gy[e] = 0.5f * (mus[mc][ty + 2][cxl + 1] - mus[mc][ty][cxl + 1]);
                    gz[e] = 0.5f * (mus[mp][ty + 1][cxl + 1] - mus[mm][ty + 1][cxl + 1]);
                }
            }
            psi = make_float2(phis[ps(k)][ty + 2][tx + 2], phis[ps(k)][ty + 2][tx + 3]);
            ph = add2(f2(dref.Phi), psi);
            muc = make_float2(mus[mc][ty + 1][tx + 1], mus[mc][ty + 1][tx + 2]);
            Fx = make_float2(-ph.x * gx[0], -ph.y * gx[1]);
            Fy = make_float2(-ph.x * gy[0], -ph.y * gy[1]);
            Fz = make_float2(-ph.x * gz[0], -ph.y * gz[1]);
        }
        if (phi_out && cok) {  // fields of the source state, for the adjoint
            *reinterpret_cast<float2*>(phi_out + s) = ph;
            *reinterpret_cast<float2*>(mu_out + s) = muc;
        }
        // destination of direction i for site e of the pair
        auto dest = [&](int i, int e) {
            const int ox = cx(i) > 0 ? (e == 0 ? 1 : oxp1) : (cx(i) < 0 ? (e == 0 ? oxm0 : -1) : 0);
            return s + e + ox + (cy(i) > 0 ? oyp : (cy(i) < 0 ? oym : 0)) + (cz(i) > 0 ? ozp : (cz(i) < 0 ? ozm : 0));
        };
        // SR: the random 16 bits of (site, distribution a, direction i) are
        // those sr_key gives (one splitmix64 word per four directions, from
        // the site's stream position); the collisions hand the directions over
        // as 1..18 and then 0, so each site keeps its current word and the
        // group it belongs to.
        unsigned long long srw[2] = {0ull, 0ull};
        int srg[2] = {-1, -1};
        auto sr_bits = [&](int e, int a, int i) -> unsigned {
            const int grp = 5 * a + (i >> 2);
            if (srg[e] != grp) {
                const unsigned long long st = sr.base + (unsigned long long)(s + e) * kSrGamma;
                srw[e] = sr_mix(st + (unsigned long long)grp * sr.stride);
                srg[e] = grp;
            }
            return (unsigned)(srw[e] >> (16 * (i & 3))) & 0xffffu;
        };
        auto bits_of = [](S h) -> unsigned {
            unsigned short u;
            memcpy(&u, &h, 2);
            return u;
        };
        // store the pair's values of distribution a, direction i (paired when c_x = 0)
        auto store = [&](S* base, int a, int i, float2 v) {
            S lo, hi;
            if constexpr (SR) {
                lo = Prec<P>::encode_sr(v.x, 0.0f, sr_bits(0, a, i));
                hi = Prec<P>::encode_sr(v.y, 0.0f, sr_bits(1, a, i));
            }
            if (cx(i) == 0) {
                const int d = dest(i, 0);  // even; site 1 goes to d + 1
                const unsigned packed = SR ? (bits_of(lo) | (bits_of(hi) << 16)) : pack2<P>(v);
                if (site_ok(d, g.n, status) && site_ok(d + 1, g.n, status))
                    __stcs(reinterpret_cast<unsigned*>(base + i * npad + d), packed);
            } else {
                if constexpr (!SR) {
                    lo = Prec<P>::encode(v.x, 0.0f);
                    hi = Prec<P>::encode(v.y, 0.0f);
                }
                const int d0 = dest(i, 0), d1 = dest(i, 1);
                if (site_ok(d0, g.n, status)) __stcs(base + i * npad + d0, lo);
                if (site_ok(d1, g.n, status)) __stcs(base + i * npad + d1, hi);
            }
        };

        // moments of f from the packed pairs (unpacked again where collided,
        // so that 19 packed registers rather than 38 unpacked ones stay live)
        float2 delta = f2(0.0f), jx = f2(0.0f), jy = f2(0.0f), jz = f2(0.0f);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const float2 v = unpack2<P>(fpre[i]);
            delta = add2(delta, v);
            add_c2(i, v, jx, jy, jz);
        }
        const float2 rho = add2(f2(dref.R), delta);
        const float2 inv = make_float2(__frcp_rn(rho.x), __frcp_rn(rho.y));
        const float2 ux = mul2(fma2(f2(0.5f), Fx, jx), inv);
        const float2 uy = mul2(fma2(f2(0.5f), Fy, jy), inv);
        const float2 uz = mul2(fma2(f2(0.5f), Fz, jz), inv);
        collide_f_dev2([&](int i) { return unpack2<P>(fpre[i]); }, [&](int i, float2 v) { store(fd, 0, i, v); }, delta,
                       rho, ux, uy, uz, Fx, Fy, Fz, m, dref);
        const unsigned* gt = reinterpret_cast<const unsigned*>(gring + (size_t)ps(k) * Q * (TY * TX) + ty * TX + tx);
        collide_g_dev2([&](int i) { return unpack2<P>(gt[i * (TY * TX / 2)]); }, [&](int i, float2 v) { store(gd, 1, i, v); },
                       psi, ph, sub2(muc, f2(dref.muP)), ux, uy, uz, m, dref);
    }
}

// Use the pair kernel for the 16-bit forms wherever k_step_fused would run
// (round to nearest); rows per tile: 8 (four CTAs of 128 threads per SM;
// 16 rows with two CTAs of 256 measured slower).
constexpr bool kPairs16 = true;
constexpr int kPairRows = 8;

template <int P, class I, bool ISO, int TY, bool SR>
cudaError_t launch_fused2(ld_ctx* c, const void* src, void* dst, void* fields) {
    using S = typename Prec<P>::store_t;
    constexpr size_t kRingBytes = 3 * (size_t)Q * TY * kTX * sizeof(S);
    cudaError_t e = set_max_dynamic_smem_once<k_step_fused2<P, I, ISO, TY, SR>>((int)kRingBytes);
    if (e != cudaSuccess) return e;
    const Geom g{c->geom.nx, c->geom.ny, c->geom.nz, c->geom.n, c->geom.npad};
    const int nchunks = choose_chunks(g.nx, g.ny, g.nz, TY, c->num_sms, pair_ctas_per_sm<TY>());
    const dim3 grid(g.nx / kTX, g.ny / TY, nchunks);
    k_step_fused2<P, I, ISO, TY, SR><<<grid, 16 * TY, kRingBytes, c->stream>>>(
        g, model_of<float>(c->prm), nchunks, (const S*)f_part(c, src), (const S*)g_part(c, src), (S*)f_part(c, dst),
        (S*)g_part(c, dst), c->ref, fields ? (float*)fields : nullptr, fields ? (float*)fields + c->geom.npad : nullptr,
        sr_stream(c->prm.seed, c->sr_step, c->geom.n), c->status);
    return cudaGetLastError();
}

template <int P, class I, bool ISO>
cudaError_t launch_fused2_rows(ld_ctx* c, const void* src, void* dst, void* fields) {
    const bool sr = c->prm.rounding == LD_ROUND_STOCHASTIC;
    if constexpr (kPairRows == 16) {
        if (c->geom.ny % 16 == 0)
            return sr ? launch_fused2<P, I, ISO, 16, true>(c, src, dst, fields)
                      : launch_fused2<P, I, ISO, 16, false>(c, src, dst, fields);
    }
    return sr ? launch_fused2<P, I, ISO, 8, true>(c, src, dst, fields)
              : launch_fused2<P, I, ISO, 8, false>(c, src, dst, fields);
}

template <int P>
cudaError_t step_fused2_p(ld_ctx* c, const void* src, void* dst, void* fields) {
    const bool small = (long long)Q * c->geom.npad <= 0x7fffffffLL;
    if (c->prm.stencil == LD_STENCIL_19)
        return small ? launch_fused2_rows<P, int, true>(c, src, dst, fields)
                     : launch_fused2_rows<P, long long, true>(c, src, dst, fields);
    return small ? launch_fused2_rows<P, int, false>(c, src, dst, fields)
                 : launch_fused2_rows<P, long long, false>(c, src, dst, fields);
}

}  // namespace
}  // namespace ld
