// Shared device-side definitions of the D3Q19 binary-fluid step: velocity
// set, storage codecs of the four precisions, per-site equilibria, Guo
// forcing and collision. Included by every kernel translation unit.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ld.h"
#include "ld_internal.h"

namespace ld {

constexpr int Q = 19;

// D3Q19 (Qian, d'Humieres & Lallemand 1992): rest, six axis vectors, twelve
// face diagonals in (v, -v) pairs. Written as constexpr selectors so that
// fully unrolled loops fold every c_i to an immediate.
__host__ __device__ constexpr int cx(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int cy(int i) {
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
         : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int cz(int i) {
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
         : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
__host__ __device__ constexpr int c2(int i) { return cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i); }
template <class R>
__host__ __device__ constexpr R wgt(int i) {
    return i == 0 ? R(1) / R(3) : (i <= 6 ? R(1) / R(18) : R(1) / R(36));
}

// ---------------------------------------------------------------------------
// Storage precisions. real_t is the arithmetic type; store_t the stored one.
// The 16-bit forms store the deviation from a per-direction reference value.
// decode/encode work in real_t inside the step; decode_d/encode_d convert
// to and from double for initialisation, I/O and the FP64 totals.
template <int P> struct Prec;
template <> struct Prec<LD_FP64> {
    using store_t = double;
    using real_t = double;
    static constexpr bool kDev = false;
    __device__ static double decode(store_t v, double) { return v; }
    __device__ static store_t encode(double x, double) { return x; }
    __device__ static double decode_d(store_t v, float) { return v; }
    __device__ static store_t encode_d(double x, float) { return x; }
};
template <> struct Prec<LD_FP32> {
    using store_t = float;
    using real_t = float;
    static constexpr bool kDev = false;
    __device__ static float decode(store_t v, float) { return v; }
    __device__ static store_t encode(float x, float) { return x; }
    __device__ static double decode_d(store_t v, float) { return v; }
    __device__ static store_t encode_d(double x, float) { return (float)x; }
};
template <> struct Prec<LD_FP16DEV> {
    using store_t = __half;
    using real_t = float;
    static constexpr bool kDev = true;
    __device__ static float decode(store_t v, float ref) { return ref + __half2float(v); }
    __device__ static store_t encode(float x, float ref) { return __float2half_rn(x - ref); }
    __device__ static store_t encode_sr(float x, float ref, unsigned k);
    __device__ static double decode_d(store_t v, float ref) { return (double)ref + (double)__half2float(v); }
    __device__ static store_t encode_d(double x, float ref) { return __double2half(x - (double)ref); }
};
template <> struct Prec<LD_BF16DEV> {
    using store_t = __nv_bfloat16;
    using real_t = float;
    static constexpr bool kDev = true;
    __device__ static float decode(store_t v, float ref) { return ref + __bfloat162float(v); }
    __device__ static store_t encode(float x, float ref) { return __float2bfloat16_rn(x - ref); }
    __device__ static store_t encode_sr(float x, float ref, unsigned k);
    __device__ static double decode_d(store_t v, float ref) { return (double)ref + (double)__bfloat162float(v); }
    __device__ static store_t encode_d(double x, float ref) { return __double2bfloat16(x - (double)ref); }
};

// Stochastic rounding of the FP32 deviation h to a 16-bit format with the
// 16-bit random integer k (Connolly, Higham & Mary 2021, mode 1): lo = h
// rounded toward zero, hi = the next value away from zero, and hi is taken
// when k (|hi| - |lo|) < 65536 (|h| - |lo|). Both sides of the comparison are
// exact in FP32 (|hi| - |lo| is a power of two, |h| - |lo| is exact by
// Sterbenz's lemma or because lo = 0), so the decision is a function of h and
// k alone. Exact values, NaN and the largest finite magnitude are kept.
__device__ __forceinline__ bool sr_up(float h, float lo, float hi, unsigned k) {
    const float gap = __fsub_rn(fabsf(hi), fabsf(lo));
    const float d = __fsub_rn(fabsf(h), fabsf(lo));
    return __fmul_rn((float)k, gap) < __fmul_rn(d, 65536.0f);
}
__device__ __forceinline__ __half Prec<LD_FP16DEV>::encode_sr(float x, float ref, unsigned k) {
    const float h = x - ref;
    const __half lo = __float2half_rz(h);
    const float lof = __half2float(lo);
    const unsigned short b = __half_as_ushort(lo);
    if (lof == h || (b & 0x7fffu) == 0x7bffu) return lo;
    const __half hi = __ushort_as_half((unsigned short)(b + 1));
    return sr_up(h, lof, __half2float(hi), k) ? hi : lo;
}
__device__ __forceinline__ __nv_bfloat16 Prec<LD_BF16DEV>::encode_sr(float x, float ref, unsigned k) {
    const float h = x - ref;
    const __nv_bfloat16 lo = __float2bfloat16_rz(h);
    const float lof = __bfloat162float(lo);
    const unsigned short b = __bfloat16_as_ushort(lo);
    if (lof == h || (b & 0x7fffu) == 0x7f7fu) return lo;
    const __nv_bfloat16 hi = __ushort_as_bfloat16((unsigned short)(b + 1));
    return sr_up(h, lof, __bfloat162float(hi), k) ? hi : lo;
}

// Random words of stochastic rounding: SplitMix64 (Steele, Lea & Flood 2014)
// used as a counter-based generator. The word of counter c is the output
// mix of the state seed + (c + 1) gamma; c = ((2t + a) 5 + q) N + s for step
// t, array a (0 f, 1 g), quarter q = i / 4 of the directions and site s.
constexpr unsigned long long kSrGamma = 0x9E3779B97F4A7C15ull;
__device__ __forceinline__ unsigned long long sr_mix(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
// The step's stream: state of (a, q, s) = base + s gamma + (5a + q) stride,
// with base = seed + gamma + 10 t N gamma and stride = N gamma (mod 2^64).
struct SrStream {
    unsigned long long base, stride;
};
inline SrStream sr_stream(unsigned long long seed, unsigned long long t, long long n) {
    const unsigned long long ng = (unsigned long long)n * kSrGamma;
    return SrStream{seed + kSrGamma + 10ull * t * ng, ng};
}
// 16-bit random integer of direction i of array a at a site whose stream
// state is st = base + s gamma; w caches the word of the current quarter
// (the loops over i are unrolled, so i % 4 == 0 refreshes it).
__device__ __forceinline__ unsigned sr_key(const SrStream& r, unsigned long long st, int a, int i,
                                           unsigned long long& w) {
    if ((i & 3) == 0) w = sr_mix(st + (unsigned long long)(5 * a + (i >> 2)) * r.stride);
    return (unsigned)(w >> (16 * (i & 3))) & 0xffffu;
}

// Debug builds (compiled with -DLD_DEBUG_BOUNDS): the step kernels check the
// site index of every global load and store against [0, n) first; an index
// outside sets kStatusBounds and the access is skipped (a load reads 0), so
// a wrong index is reported instead of faulting. Release builds compile the
// checks away.
#ifdef LD_DEBUG_BOUNDS
constexpr bool kDebugBounds = true;
#else
constexpr bool kDebugBounds = false;
#endif
__device__ __forceinline__ bool site_ok(long long s, long long n, int* status) {
    if constexpr (!kDebugBounds) return true;
    if (s >= 0 && s < n) return true;
    atomicOr(status, kStatusBounds);
    return false;
}

// Lattice geometry. npad: component stride of every SoA array (>= n, a
// multiple of 64 so each component starts 256-byte aligned for 32-bit data).
struct Geom {
    int nx, ny, nz;
    long long n, npad;
};

// Model constants in the arithmetic type.
template <class R>
struct Model {
    R A, B, kappa, Gamma;
    R omega_f, omega_g;  // 1/tau
    R force_pre;         // 1 - 1/(2 tau_f)
    int iso;             // 1: 19-point isotropic stencils (LD_STENCIL_19)
    int trt;             // 1: two-relaxation-time collision of f (LD_COLLISION_TRT)
    R omega_m;           // TRT: 1/tau- of the odd parts
    R force_pre_m;       // TRT: 1 - 1/(2 tau-)
};

// Model constants from the C-ABI parameters.
template <class R>
inline Model<R> model_of(const ld_params& p) {
    Model<R> m;
    m.A = (R)p.A;
    m.B = (R)p.B;
    m.kappa = (R)p.kappa;
    m.Gamma = (R)p.Gamma;
    m.omega_f = (R)(1.0 / p.tau_f);
    m.omega_g = (R)(1.0 / p.tau_g);
    m.force_pre = (R)(1.0 - 0.5 / p.tau_f);
    m.iso = p.stencil == LD_STENCIL_19 ? 1 : 0;
    m.trt = p.collision == LD_COLLISION_TRT ? 1 : 0;
    const double tau_m = m.trt ? 0.5 + p.magic / (p.tau_f - 0.5) : p.tau_f;
    m.omega_m = (R)(1.0 / tau_m);
    m.force_pre_m = (R)(1.0 - 0.5 / tau_m);
    return m;
}

// Reference values of the deviation codec: ref[i] for f, ref[19 + i] for g.
constexpr int kRefCount = 2 * Q;

__device__ __forceinline__ int wrap_inc(int a, int n) { return a + 1 == n ? 0 : a + 1; }
__device__ __forceinline__ int wrap_dec(int a, int n) { return a == 0 ? n - 1 : a - 1; }

// ---------------------------------------------------------------------------
// Per-site physics (one site, registers only).

// Explicitly rounded products and sums: the compiler may not contract these
// into fused multiply-adds, so every kernel that forms mu gets the same bits.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }

// mu = A phi + B phi^3 - kappa lap; operations in that order, each rounded once.
template <class R>
__device__ __forceinline__ R chem_potential_lap(R phi, R lap, const Model<R>& m) {
    const R cubic = mul_rn(mul_rn(mul_rn(m.B, phi), phi), phi);
    return sub_rn(add_rn(mul_rn(m.A, phi), cubic), mul_rn(m.kappa, lap));
}

// The same with the 7-point lap = (sum of the six axis neighbours' phi) - 6 phi.
template <class R>
__device__ __forceinline__ R chem_potential(R phi, R nb_sum, const Model<R>& m) {
    return chem_potential_lap(phi, sub_rn(nb_sum, mul_rn(R(6), phi)), m);
}

// 19-point isotropic forms on the D3Q19 neighbourhood. nb(i) is h(x + c_i).
//   lap h  = sum_{i=1..18} 6 w_i (h(x + c_i) - h(x)),  6 w_i = 1/3 (axis), 1/6 (diagonal)
//   grad h = sum_{i=1..18} 3 w_i c_i h(x + c_i),       3 w_i = 1/6 (axis), 1/12 (diagonal)
// Summed in velocity order with every operation rounded once, so that each
// kernel that forms them gets the same bits (and FP64 follows the plain
// operation order); components with c_ia = 0 contribute nothing.
template <class R>
__device__ __forceinline__ R lap19_coef(int i) {
    return i <= 6 ? R(1) / R(3) : R(1) / R(6);
}
template <class R>
__device__ __forceinline__ R grad19_coef(int i) {
    return i <= 6 ? R(1) / R(6) : R(1) / R(12);
}
template <class R, class F>
__device__ __forceinline__ R lap19(R h0, F nb) {
    R sum = R(0);
#pragma unroll
    for (int i = 1; i < Q; ++i) sum = add_rn(sum, mul_rn(lap19_coef<R>(i), sub_rn(nb(i), h0)));
    return sum;
}
template <class R, class F>
__device__ __forceinline__ void grad19(F nb, R& gx, R& gy, R& gz) {
    gx = gy = gz = R(0);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const R t = mul_rn(grad19_coef<R>(i), nb(i));
        if (cx(i) > 0) gx = add_rn(gx, t);
        if (cx(i) < 0) gx = sub_rn(gx, t);
        if (cy(i) > 0) gy = add_rn(gy, t);
        if (cy(i) < 0) gy = sub_rn(gy, t);
        if (cz(i) > 0) gz = add_rn(gz, t);
        if (cz(i) < 0) gz = sub_rn(gz, t);
    }
}

// c_i . (ax, ay, az) over the nonzero components of c_i only, in x, y, z
// order. Equal, bit for bit, to the full three-term sum (adding a zero
// product changes nothing) without the multiplies by 0 and +-1 that IEEE
// arithmetic does not let the compiler drop.
template <class R>
__device__ __forceinline__ R cdot(int i, R ax, R ay, R az) {
    R s = R(0);
    bool any = false;
    if (cx(i) != 0) {
        s = cx(i) > 0 ? ax : -ax;
        any = true;
    }
    if (cy(i) != 0) {
        s = any ? (cy(i) > 0 ? s + ay : s - ay) : (cy(i) > 0 ? ay : -ay);
        any = true;
    }
    if (cz(i) != 0) s = any ? (cz(i) > 0 ? s + az : s - az) : (cz(i) > 0 ? az : -az);
    return s;
}

// Accumulate v c_i into (jx, jy, jz), skipping zero components.
template <class R>
__device__ __forceinline__ void add_c(int i, R v, R& jx, R& jy, R& jz) {
    if (cx(i) > 0) jx += v;
    if (cx(i) < 0) jx -= v;
    if (cy(i) > 0) jy += v;
    if (cy(i) < 0) jy -= v;
    if (cz(i) > 0) jz += v;
    if (cz(i) < 0) jz -= v;
}

// Guo velocity from the moments and the force: u = (j + F/2) / rho. FP64
// divides (the rounding the FP64 path is held to); FP32 multiplies by the
// correctly rounded reciprocal.
__device__ __forceinline__ void guo_velocity(double rho, double jx, double jy, double jz, double Fx, double Fy,
                                             double Fz, double& ux, double& uy, double& uz) {
    ux = (jx + 0.5 * Fx) / rho;
    uy = (jy + 0.5 * Fy) / rho;
    uz = (jz + 0.5 * Fz) / rho;
}
__device__ __forceinline__ void guo_velocity(float rho, float jx, float jy, float jz, float Fx, float Fy, float Fz,
                                             float& ux, float& uy, float& uz) {
    const float inv = __frcp_rn(rho);
    ux = (jx + 0.5f * Fx) * inv;
    uy = (jy + 0.5f * Fy) * inv;
    uz = (jz + 0.5f * Fz) * inv;
}

// BGK + Guo collision of f in place.
//
// The generic template evaluates the equilibrium and the source term
// direction by direction, in the operation order of the formulas above.
// FP64 and FP32 (also the arithmetic of the 16-bit forms) use specialisations
// on opposite pairs (i, i+1), c_{i+1} = -c_i: c.u and c.F change sign within
// a pair, so
//   feq_(i,i+1) = w rho (1 - 3/2 u.u + 9/2 (c.u)^2) +- 3 w rho c.u
//   src_(i,i+1) = pre w (9 (c.u)(c.F) - 3 u.F)        +- 3 pre w c.F
// and each pair shares its symmetric part. In FP32 the rest equilibrium is
// rho minus the 18 moving ones (the same value in exact arithmetic): the
// nearest floats to 1/3, 1/18, 1/36 sum to 1 + 1.5e-8, and the formula for
// every direction would add that much mass to each site at every step.
template <class R>
__device__ __forceinline__ void collide_f(R (&f)[Q], R rho, R ux, R uy, R uz, R Fx, R Fy, R Fz,
                                          const Model<R>& m) {
    const R uu = ux * ux + uy * uy + uz * uz;
    const R uF = ux * Fx + uy * Fy + uz * Fz;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const R cu = cdot(i, ux, uy, uz);
        const R cF = cdot(i, Fx, Fy, Fz);
        const R feq = wgt<R>(i) * rho * (R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu);
        const R src = m.force_pre * wgt<R>(i) * (R(3) * (cF - uF) + R(9) * cu * cF);
        f[i] = f[i] - m.omega_f * (f[i] - feq) + src;
    }
    // c_0 = 0: feq_0 = w_0 rho (1 - 3/2 u.u), src_0 = pre w_0 (-3 u.F)
    const R feq0 = wgt<R>(0) * rho * (R(1) - R(1.5) * uu);
    const R src0 = m.force_pre * wgt<R>(0) * (R(3) * (-uF));
    f[0] = f[0] - m.omega_f * (f[0] - feq0) + src0;
}

// FP64 on opposite pairs too (with the g collision's pair form, about 35 %
// fewer FP64 operations per site than direction by direction, where the FP64
// pipe is the bound); the rest
// equilibrium from its formula, the FP64 weights summing to 1 within an ulp.
template <>
__device__ __forceinline__ void collide_f<double>(double (&f)[Q], double rho, double ux, double uy, double uz,
                                                  double Fx, double Fy, double Fz, const Model<double>& m) {
    const double uu = ux * ux + uy * uy + uz * uz;
    const double uF = ux * Fx + uy * Fy + uz * Fz;
    const double base = 1.0 - 1.5 * uu;
    const double keep = 1.0 - m.omega_f;
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const double w = wgt<double>(i);
        const double wr = w * rho, pw = m.force_pre * w;
        const double cu = cdot(i, ux, uy, uz);
        const double cF = cdot(i, Fx, Fy, Fz);
        const double feq_sym = wr * (base + 4.5 * cu * cu);
        const double feq_anti = 3.0 * wr * cu;
        const double src_sym = pw * (9.0 * cu * cF - 3.0 * uF);
        const double src_anti = 3.0 * pw * cF;
        const double sym = m.omega_f * feq_sym + src_sym;
        const double anti = m.omega_f * feq_anti + src_anti;
        f[i] = keep * f[i] + (sym + anti);
        f[i + 1] = keep * f[i + 1] + (sym - anti);
    }
    const double feq0 = wgt<double>(0) * rho * base;
    const double src0 = m.force_pre * wgt<double>(0) * (-3.0 * uF);
    f[0] = keep * f[0] + (m.omega_f * feq0 + src0);
}

template <>
__device__ __forceinline__ void collide_f<float>(float (&f)[Q], float rho, float ux, float uy, float uz, float Fx,
                                                 float Fy, float Fz, const Model<float>& m) {
    const float uu = ux * ux + uy * uy + uz * uz;
    const float uF = ux * Fx + uy * Fy + uz * Fz;
    const float base = 1.0f - 1.5f * uu;
    const float keep = 1.0f - m.omega_f;
    float moving = 0.0f;  // sum of the symmetric equilibrium parts (each counted once)
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const float w = wgt<float>(i);
        const float wr = w * rho, pw = m.force_pre * w;
        const float cu = cdot(i, ux, uy, uz);
        const float cF = cdot(i, Fx, Fy, Fz);
        const float feq_sym = wr * (base + 4.5f * cu * cu);
        const float feq_anti = 3.0f * wr * cu;
        const float src_sym = pw * (9.0f * cu * cF - 3.0f * uF);
        const float src_anti = 3.0f * pw * cF;
        const float sym = m.omega_f * feq_sym + src_sym;
        const float anti = m.omega_f * feq_anti + src_anti;
        f[i] = keep * f[i] + (sym + anti);
        f[i + 1] = keep * f[i + 1] + (sym - anti);
        moving += feq_sym;
    }
    const float feq0 = rho - 2.0f * moving;
    const float src0 = m.force_pre * wgt<float>(0) * (-3.0f * uF);
    f[0] = keep * f[0] + (m.omega_f * feq0 + src0);
}

// ---------------------------------------------------------------------------
// Arithmetic in deviation space (the 16-bit storage forms).
//
// The stored values are h_i = f_i - r_i and h_i = g_i - q_i with fixed
// references r_i (~ w_i rho0) and q_i (~ geq_i(phibar, 0, mubar)). A collision
// written on the deviations needs no decode of the form r_i + h_i and no
// encode of the form f_i - r_i: with R = sum r_i and delta = sum h_i,
//   rho = R + delta,  j = sum_i c_i h_i  (r_i = r_-i, so the references cancel)
//   f*_i - r_i = (1 - w_f) h_i + w_f (feq_i - r_i) + S_i,
//   feq_i - r_i = w_i delta + (w_i R - r_i) + w_i rho (3 c.u + 9/2 (c.u)^2 - 3/2 u.u),
// and with Phi = sum q_i, psi = sum h_i (phi = Phi + psi), dhat any constant,
//   g*_i - q_i = (1 - w_g) h_i + w_g (geq_i - q_i),
//   geq_i - q_i = w_i [psi - 3/2 phi u.u + 9/2 (dev - dhat)(|c_i|^2 - 1) + 3 phi c.u
//                      + 9/2 phi (c.u)^2] + (w_i (Phi + 9/2 dhat (|c_i|^2 - 1)) - q_i),
// dev = Gamma mu - phi/3. Both are the same step as collide_f / collide_g in
// exact arithmetic; the constant terms in parentheses (a few units in the
// last place of the references) are formed once, in FP64. The rest values
// come by difference, so sum_i h*_i equals the conserved delta (f, plus the
// Guo source's rounding) and psi (g) exactly as in collide_f / collide_g.
struct DevRefs {
    float R;      // sum_i r_i
    float ef[3];  // w_i R - r_i for the rest, axis and diagonal directions
    float Phi;    // sum_i q_i
    float muP;    // A Phi + B Phi^3
    float dhat;   // Gamma muP - Phi/3
    float eg[3];  // w_i (Phi + 9/2 dhat (|c_i|^2 - 1)) - q_i per class
};

// Class of a direction: 0 rest, 1 axis, 2 diagonal.
__host__ __device__ constexpr int dir_class(int i) { return i == 0 ? 0 : (i <= 6 ? 1 : 2); }

// The constants from the 38 stored references (f then g), in FP64.
__device__ inline DevRefs dev_refs_of(const float* ref, const Model<float>& m) {
    double R = 0.0, Phi = 0.0;
    for (int i = 0; i < Q; ++i) {
        R += (double)ref[i];
        Phi += (double)ref[Q + i];
    }
    const double muP = (double)m.A * Phi + (double)m.B * Phi * Phi * Phi;
    const double dhat = (double)m.Gamma * muP - Phi / 3.0;
    DevRefs d;
    d.R = (float)R;
    d.Phi = (float)Phi;
    d.muP = (float)muP;
    d.dhat = (float)dhat;
    const int rep[3] = {0, 1, 7};
    for (int k = 0; k < 3; ++k) {
        const int i = rep[k];
        d.ef[k] = (float)(wgt<double>(i) * R - (double)ref[i]);
        d.eg[k] = (float)(wgt<double>(i) * (Phi + 4.5 * dhat * (c2(i) - 1)) - (double)ref[Q + i]);
    }
    return d;
}

// BGK + Guo collision of the f deviations in place; delta = sum_i h_i,
// rho = R + delta.
__device__ __forceinline__ void collide_f_dev(float (&h)[Q], float delta, float rho, float ux, float uy, float uz,
                                              float Fx, float Fy, float Fz, const Model<float>& m, const DevRefs& d) {
    const float uu = ux * ux + uy * uy + uz * uz;
    const float uF = ux * Fx + uy * Fy + uz * Fz;
    const float keep = 1.0f - m.omega_f;
    float moving = 0.0f;  // sum of the symmetric parts of feq_i - r_i over the pairs
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const float w = wgt<float>(i);
        const float wr = w * rho, pw = m.force_pre * w;
        const float cu = cdot(i, ux, uy, uz);
        const float cF = cdot(i, Fx, Fy, Fz);
        const float eq_sym = w * delta + d.ef[dir_class(i)] + wr * (4.5f * cu * cu - 1.5f * uu);
        const float eq_anti = 3.0f * wr * cu;
        const float src_sym = pw * (9.0f * cu * cF - 3.0f * uF);
        const float src_anti = 3.0f * pw * cF;
        const float sym = m.omega_f * eq_sym + src_sym;
        const float anti = m.omega_f * eq_anti + src_anti;
        h[i] = keep * h[i] + (sym + anti);
        h[i + 1] = keep * h[i + 1] + (sym - anti);
        moving += eq_sym;
    }
    const float eq0 = delta - 2.0f * moving;
    const float src0 = m.force_pre * wgt<float>(0) * (-3.0f * uF);
    h[0] = keep * h[0] + (m.omega_f * eq0 + src0);
}

// BGK collision of the g deviations in place; psi = sum_i h_i, phi = Phi + psi,
// dmu = mu - muP.
__device__ __forceinline__ void collide_g_dev(float (&h)[Q], float psi, float phi, float dmu, float ux, float uy,
                                              float uz, const Model<float>& m, const DevRefs& d) {
    const float uu = ux * ux + uy * uy + uz * uz;
    const float ddev = m.Gamma * dmu - psi / 3.0f;  // dev - dhat
    const float base = psi - 1.5f * phi * uu;
    const float keep = 1.0f - m.omega_g;
    float moving = 0.0f;
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const float w = wgt<float>(i);
        const float cu = cdot(i, ux, uy, uz);
        const float eq_sym = w * (base + 4.5f * ddev * float(c2(i) - 1) + 4.5f * phi * cu * cu) + d.eg[dir_class(i)];
        const float eq_anti = 3.0f * w * phi * cu;
        const float sym = m.omega_g * eq_sym, anti = m.omega_g * eq_anti;
        h[i] = keep * h[i] + (sym + anti);
        h[i + 1] = keep * h[i + 1] + (sym - anti);
        moving += eq_sym;
    }
    const float eq0 = psi - 2.0f * moving;
    h[0] = keep * h[0] + m.omega_g * eq0;
}

// A stored value as float (exact for every storage type of the FP32 arithmetic).
__device__ __forceinline__ float to_float(float v) { return v; }
__device__ __forceinline__ float to_float(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_float(__nv_bfloat16 v) { return __bfloat162float(v); }

// acc + (a 16-bit value), rounded once: the value converts exactly, so this
// equals float(v) + acc; one instruction instead of a conversion and an add.
__device__ __forceinline__ float add_f16(float acc, unsigned short bits) {
    float r;
    asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(r) : "h"(bits), "f"(acc));
    return r;
}
__device__ __forceinline__ float add_bf16(float acc, unsigned short bits) {
    float r;
    asm("add.rn.f32.bf16 %0, %1, %2;" : "=f"(r) : "h"(bits), "f"(acc));
    return r;
}

// Two-relaxation-time collision of f in place (LD_COLLISION_TRT). Each
// opposite pair (i, i+1), c_{i+1} = -c_i, splits into even and odd parts:
//   f+- = (f_i +- f_{i+1})/2,  feq+ = w rho (1 - 3/2 u.u + 9/2 (c.u)^2), feq- = 3 w rho c.u,
//   S+ = w (9 (c.u)(c.F) - 3 u.F),  S- = 3 w c.F   (the Guo source without prefactor),
//   new+ = f+ - omega+ (f+ - feq+) + (1 - omega+/2) S+,
//   new- = f- - omega- (f- - feq-) + (1 - omega-/2) S-,
//   f_i = new+ + new-,  f_{i+1} = new+ - new-.
// The rest population has only an even part. In FP32 its equilibrium is rho
// minus the 18 moving ones (as in collide_f), which keeps mass exact.
template <class R>
__device__ __forceinline__ void collide_f_trt(R (&f)[Q], R rho, R ux, R uy, R uz, R Fx, R Fy, R Fz,
                                              const Model<R>& m) {
    const R uu = ux * ux + uy * uy + uz * uz;
    const R uF = ux * Fx + uy * Fy + uz * Fz;
    R moving = R(0);
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const R w = wgt<R>(i);
        const R cu = cdot(i, ux, uy, uz);
        const R cF = cdot(i, Fx, Fy, Fz);
        const R ep = w * rho * (R(1) + R(4.5) * cu * cu - R(1.5) * uu);
        const R em = R(3) * w * rho * cu;
        const R sp = w * (R(9) * cu * cF - R(3) * uF);
        const R sm = R(3) * w * cF;
        const R fp = R(0.5) * (f[i] + f[i + 1]), fm = R(0.5) * (f[i] - f[i + 1]);
        const R np = fp - m.omega_f * (fp - ep) + m.force_pre * sp;
        const R nm = fm - m.omega_m * (fm - em) + m.force_pre_m * sm;
        f[i] = np + nm;
        f[i + 1] = np - nm;
        moving += ep;
    }
    const R feq0 = sizeof(R) == 4 ? rho - R(2) * moving : wgt<R>(0) * rho * (R(1) - R(1.5) * uu);
    const R s0 = wgt<R>(0) * (R(3) * (-uF));
    f[0] = f[0] - m.omega_f * (f[0] - feq0) + m.force_pre * s0;
}

// BGK collision of g in place: the generic template direction by direction;
// FP64 and FP32 on opposite pairs (FP32 with the rest equilibrium phi minus
// the moving ones, as in collide_f).
template <class R>
__device__ __forceinline__ void collide_g(R (&g)[Q], R phi, R mu, R ux, R uy, R uz, const Model<R>& m) {
    const R uu = ux * ux + uy * uy + uz * uz;
    const R dev = m.Gamma * mu - phi / R(3);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const R cu = cdot(i, ux, uy, uz);
        const R geq = wgt<R>(i) * (phi + R(3) * phi * cu + R(4.5) * dev * R(c2(i) - 1)
                                   + R(4.5) * phi * cu * cu - R(1.5) * phi * uu);
        g[i] = g[i] - m.omega_g * (g[i] - geq);
    }
    // c_0 = 0, |c_0|^2 - 1 = -1: geq_0 = w_0 (phi - 9/2 dev - 3/2 phi u.u)
    const R geq0 = wgt<R>(0) * ((phi - R(4.5) * dev) - R(1.5) * phi * uu);
    g[0] = g[0] - m.omega_g * (g[0] - geq0);
}

template <>
__device__ __forceinline__ void collide_g<double>(double (&g)[Q], double phi, double mu, double ux, double uy,
                                                  double uz, const Model<double>& m) {
    const double uu = ux * ux + uy * uy + uz * uz;
    const double dev = m.Gamma * mu - phi / 3.0;
    const double pbase = phi * (1.0 - 1.5 * uu);
    const double keep = 1.0 - m.omega_g;
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const double w = wgt<double>(i);
        const double cu = cdot(i, ux, uy, uz);
        const double geq_sym = w * (pbase + 4.5 * dev * double(c2(i) - 1) + 4.5 * phi * cu * cu);
        const double geq_anti = 3.0 * w * phi * cu;
        const double sym = m.omega_g * geq_sym, anti = m.omega_g * geq_anti;
        g[i] = keep * g[i] + (sym + anti);
        g[i + 1] = keep * g[i + 1] + (sym - anti);
    }
    const double geq0 = wgt<double>(0) * ((phi - 4.5 * dev) - 1.5 * phi * uu);
    g[0] = keep * g[0] + m.omega_g * geq0;
}

template <>
__device__ __forceinline__ void collide_g<float>(float (&g)[Q], float phi, float mu, float ux, float uy, float uz,
                                                 const Model<float>& m) {
    const float uu = ux * ux + uy * uy + uz * uz;
    const float dev = m.Gamma * mu - phi / 3.0f;
    const float pbase = phi * (1.0f - 1.5f * uu);
    const float keep = 1.0f - m.omega_g;
    float moving = 0.0f;
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const float w = wgt<float>(i);
        const float cu = cdot(i, ux, uy, uz);
        const float geq_sym = w * (pbase + 4.5f * dev * float(c2(i) - 1) + 4.5f * phi * cu * cu);
        const float geq_anti = 3.0f * w * phi * cu;
        const float sym = m.omega_g * geq_sym, anti = m.omega_g * geq_anti;
        g[i] = keep * g[i] + (sym + anti);
        g[i + 1] = keep * g[i + 1] + (sym - anti);
        moving += geq_sym;
    }
    const float geq0 = phi - 2.0f * moving;
    g[0] = keep * g[0] + m.omega_g * geq0;
}

}  // namespace ld
