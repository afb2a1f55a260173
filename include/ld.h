/*
 * ld.h -- C ABI of the binary-fluid D3Q19 lattice-Boltzmann library (sm_103a).
 *
 * One timestep of the grid application ported in Gray & Stratford, "A
 * Lightweight Approach to Performance Portability with targetDP" (Sec. 2.1.1,
 * the Ludwig components "Order Parameter Gradients", "Chemical stress",
 * "Collision" and "Propagation"), in its binary-fluid form:
 *
 *   rho = sum_i f_i,  j = sum_i f_i c_i,  phi = sum_i g_i      (moments)
 *   mu  = A phi + B phi^3 - kappa lap(phi)       (7-point Laplacian by default)
 *   F   = -phi grad(mu)                           (2-point central difference by default)
 *   u   = (j + F/2) / rho                         (Guo, Zheng & Shi 2002)
 *   f*_i = f_i - (f_i - feq_i(rho,u))/tau_f + (1 - 1/(2 tau_f)) w_i [3(c_i-u) + 9(c_i.u)c_i].F
 *   g*_i = g_i - (g_i - geq_i(phi,u,mu))/tau_g
 *   f_i(x + c_i, t+1) = f*_i(x, t),  g likewise                (propagation)
 *
 * with feq_i = w_i rho [1 + 3c.u + 9/2 (c.u)^2 - 3/2 u.u] and
 * geq_i = w_i [phi + 3 phi c.u + 9/2 (Gamma mu - phi/3)(|c_i|^2 - 1)
 *              + 9/2 phi (c.u)^2 - 3/2 phi u.u],
 * on a periodic nx*ny*nz lattice, D3Q19 velocity set in the order: rest,
 * +x,-x,+y,-y,+z,-z, then the face diagonals in (v,-v) pairs
 * (++0,--0,+-0,-+0, +0+,-0-,+0-,-0+, 0++,0--,0+-,0-+).
 * The lines above are the default step; ld_params selects 19-point
 * stencils (LD_STENCIL_19), the force -div P (LD_FORCE_STRESS) and a
 * two-relaxation-time collision of f (LD_COLLISION_TRT), described with
 * their enums below.
 *
 * Conventions shared by every call:
 *   - Site order s = x + nx*(y + ny*z), x fastest. Scalar fields are double[N],
 *     vector fields double[3][N] (component-major), distributions
 *     double[19][N]; N = nx*ny*nz.
 *   - Every array pointer is a DEVICE pointer (cudaMalloc'd or torch-owned);
 *     host pointers are rejected with LD_EINVAL. The library never allocates
 *     or frees device memory: the caller provides one workspace of
 *     ld_workspace_bytes() bytes (256-byte aligned) and keeps it alive until
 *     ld_destroy(). The library owns only the host-side context.
 *   - Calls are stream-ordered on the CUDA stream given to ld_create() (or
 *     ld_set_stream()); they do not synchronise the host unless stated.
 *   - Return 0 (LD_OK) on success or a negative LD_E* code; ld_last_error()
 *     gives a message. No call aborts, exits or traps the device.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef LD_H
#define LD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Storage precision of the distributions (arithmetic in parentheses).
 * LD_FP64: double (double).  LD_FP32: float (float).
 * LD_FP16DEV / LD_BF16DEV: half / bfloat16 deviations from a fixed reference
 * (float): f_i = w_i rho0 + h_i, g_i = geq_i(phibar, 0, A phibar + B phibar^3) + h_i,
 * phibar the mean of the initial phi; stores round to nearest even. */
enum { LD_FP64 = 0, LD_FP32 = 1, LD_FP16DEV = 2, LD_BF16DEV = 3 };

/* Step kernel selection.
 * LD_KERNEL_GENERIC: three launches per step (phi, mu, collide+propagate); any lattice.
 * LD_KERNEL_FUSED: one launch per step that reads and writes each distribution
 *   once from HBM; phi and mu rings in shared memory, distributions through
 *   registers (nx % 32 == 0, ny % 8 == 0, nz % 4 == 0).
 * LD_KERNEL_FUSED_STAGED: the fused step with each plane's distributions
 *   staged in shared memory one plane ahead by asynchronous 16-byte copies
 *   (cp.async, completion tracked on mbarriers with bounded waits); FP32 and
 *   the 16-bit forms only (nx % 32 == 0, ny % 8 == 0, nz % 4 == 0); every
 *   stencil and rounding option of FUSED.
 * LD_KERNEL_AUTO: FUSED when the lattice admits it, else GENERIC; always
 * GENERIC for LD_FP64, which is bound by the FP64 pipe, where the generic
 * launches do less FP64 work per site (no halo phi sums). */
enum { LD_KERNEL_AUTO = 0, LD_KERNEL_GENERIC = 1, LD_KERNEL_FUSED = 2, LD_KERNEL_FUSED_STAGED = 3 };

/* Stencils of the order-parameter gradients (mu's Laplacian, the force's
 * gradient of mu, the grad phi output). The paper names these kernels
 * ("Order Parameter Gradients", Sec. 2.1.1) without their forms.
 * LD_STENCIL_7: 7-point Laplacian and 2-point central difference (default).
 * LD_STENCIL_19: 19-point isotropic forms on the D3Q19 neighbourhood,
 *   lap h = sum_i 6 w_i (h(x + c_i) - h(x)), grad h = sum_i 3 w_i c_i h(x + c_i),
 *   whose leading truncation errors do not depend on direction. */
enum { LD_STENCIL_7 = 0, LD_STENCIL_19 = 1 };

/* Form of the force on the fluid (the "Chemical stress" kernel of a Ludwig
 * timestep, Sec. 2.1.1 of the paper, which gives no formula).
 * LD_FORCE_POTENTIAL: F = -phi grad(mu) (default).
 * LD_FORCE_STRESS: F = -div P, the divergence of the chemical stress
 *   P_ab = [A phi^2/2 + 3B phi^4/4 - kappa phi lap(phi) - kappa/2 |grad phi|^2] delta_ab
 *          + kappa d_a phi d_b phi,
 *   with the selected stencils; equal to -phi grad(mu) in the continuum, it
 *   conserves total momentum exactly on the lattice. GENERIC kernel only
 *   (AUTO picks it; FUSED and FUSED_STAGED give LD_EINVAL); no adjoint
 *   (ld_adjoint_workspace_bytes returns 0, ld_adjoint_attach LD_EINVAL).
 *   Fixed at ld_create (its 6 stress fields are part of the workspace). */
enum { LD_FORCE_POTENTIAL = 0, LD_FORCE_STRESS = 1 };

/* Collision of f (the "Collision" kernel of Sec. 2.1.1; the paper gives no
 * formula).
 * LD_COLLISION_BGK: one relaxation time tau_f, Guo forcing (default).
 * LD_COLLISION_TRT: two relaxation times. The even and odd parts of each
 *   opposite pair, f+- = (f_i +- f_-i)/2, and likewise of f^eq and of the Guo
 *   source, relax with omega+ = 1/tau_f and omega- = 1/tau-, where
 *   tau- = 1/2 + magic/(tau_f - 1/2); the source parts carry (1 - omega+/2)
 *   and (1 - omega-/2). The shear viscosity is still (tau_f - 1/2)/3.
 *   GENERIC kernel only (AUTO picks it; FUSED and FUSED_STAGED give LD_EINVAL);
 *   no adjoint. Fixed at ld_create. */
enum { LD_COLLISION_BGK = 0, LD_COLLISION_TRT = 1 };

/* Rounding of the 16-bit storage forms (LD_FP16DEV, LD_BF16DEV) when a step
 * stores its collided values; ld_init and ld_set_distributions always round
 * to nearest. The paper fixes no storage precision; these are two readings.
 * LD_ROUND_NEAREST: round to nearest even (default).
 * LD_ROUND_STOCHASTIC: stochastic rounding (Connolly, Higham & Mary 2021,
 *   "mode 1"). The deviation h (FP32) is rounded toward zero to lo; hi is the
 *   next 16-bit value away from zero; the stored value is hi when
 *   k * (|hi| - |lo|) < 65536 * (|h| - |lo|), else lo, for a 16-bit random
 *   integer k: P(hi) = (|h| - |lo|)/(|hi| - |lo|) (to 2^-16), so the stored
 *   value is h in expectation. Exact values and the largest finite
 *   magnitude are kept. k comes from SplitMix64 (Steele, Lea & Flood 2014:
 *   state increment gamma = 0x9E3779B97F4A7C15 and its 64-bit output mix),
 *   counter based: for step t (steps taken since ld_init), array a (0 = f,
 *   1 = g), direction i and site s (x + nx*(y + ny*z), N sites), the word is
 *   the SplitMix64 output of state seed + (c + 1)*gamma (mod 2^64) with
 *   c = ((2t + a)*5 + i/4)*N + s, and k is its bits 16*(i%4) .. 16*(i%4)+15
 *   (the value collided at site s in direction i). Fixed seed: bitwise
 *   reproducible runs. 16-bit forms only; not with ld_step_between or the
 *   adjoint (LD_EINVAL), whose recomputation would
 *   need the step counter of the saved state. Fixed at ld_create. */
enum { LD_ROUND_NEAREST = 0, LD_ROUND_STOCHASTIC = 1 };

enum {
    LD_OK = 0,
    LD_EINVAL = -1,     /* bad argument: dims < 4, null/host pointer, tau <= 1/2, small workspace */
    LD_ECUDA = -2,      /* a CUDA runtime call or kernel launch failed */
    LD_ENONFINITE = -3, /* ld_check found a NaN or Inf in the state */
    LD_ESTATE = -4      /* call out of order (e.g. ld_step before ld_init) */
};

typedef struct {
    double A, B, kappa, Gamma; /* free energy and mobility parameter */
    double tau_f, tau_g;       /* relaxation times, each > 1/2 */
    double rho0;               /* reference density (default rho, f deviation reference) */
    int precision;             /* LD_FP64 .. LD_BF16DEV */
    int kernel;                /* LD_KERNEL_AUTO / GENERIC / FUSED / FUSED_STAGED */
    int stencil;               /* LD_STENCIL_7 / LD_STENCIL_19 */
    int force;                 /* LD_FORCE_POTENTIAL / LD_FORCE_STRESS */
    int collision;             /* LD_COLLISION_BGK / LD_COLLISION_TRT */
    double magic;              /* TRT: (tau_f - 1/2)(tau- - 1/2) > 0 (3/16 is usual) */
    int rounding;              /* LD_ROUND_NEAREST / LD_ROUND_STOCHASTIC */
    unsigned long long seed;   /* stochastic rounding: seed of the random stream */
} ld_params;

typedef struct ld_ctx ld_ctx;

/* Bytes of device workspace a context of this size and precision needs
 * (two distribution buffers, phi/mu scratch, reduction partials). 0 on bad
 * arguments. */
size_t ld_workspace_bytes(int nx, int ny, int nz, const ld_params* p);

/* Create a context on the caller's workspace (device, >= ld_workspace_bytes,
 * 256-byte aligned) and CUDA stream (cudaStream_t, or NULL for the legacy
 * default stream). Lattice dims must each be >= 4. *out receives the context. */
int ld_create(int nx, int ny, int nz, const ld_params* p, void* dev_workspace, size_t bytes,
              void* cuda_stream, ld_ctx** out);

/* Release the host context (the workspace stays the caller's). NULL is a no-op. */
int ld_destroy(ld_ctx* ctx);

/* Change the stream later calls are ordered on. */
int ld_set_stream(ld_ctx* ctx, void* cuda_stream);

/* Replace A, B, kappa, Gamma, tau_f, tau_g, the stencil, magic and the seed
 * of stochastic rounding (precision, kernel, rho0, force, collision and
 * rounding must stay as created: LD_EINVAL otherwise). Takes effect at the
 * next launch. */
int ld_set_params(ld_ctx* ctx, const ld_params* p);

/* Initial state (equilibrium, no force): f = feq(rho, u), g = geq(phi, u, mu(phi))
 * with mu from the selected stencil's Laplacian of phi. phi: device double[N];
 * rho: device double[N] or NULL (rho0 everywhere); u: device double[3][N] or
 * NULL (at rest). Also fixes the deviation reference of LD_FP16DEV/LD_BF16DEV
 * and sets the step counter t of stochastic rounding to 0. */
int ld_init(ld_ctx* ctx, const double* phi, const double* rho, const double* u);

/* ld_init for a lattice that is one part of a larger one (a slab of a
 * domain decomposition): the 16-bit storage forms take their g deviation
 * reference from phi_mean, the mean phi of the whole lattice, instead of the
 * mean of this part's phi, so that every part stores deviations from the
 * same reference as the whole lattice would. Otherwise as ld_init (the
 * reference has no effect on FP64 and FP32). LD_EINVAL for a non-finite
 * phi_mean. */
int ld_init_with_reference(ld_ctx* ctx, const double* phi, const double* rho, const double* u, double phi_mean);

/* FP64 sum of a device double[n] (any n >= 1, independent of the context's
 * lattice) into device sum[0], in the fixed order ld_init sums phi for its
 * mean: the whole lattice's mean phi for ld_init_with_reference, bit for bit
 * the one ld_init of the whole lattice would take. Uses the context's
 * reduction scratch; stream-ordered. */
int ld_field_sum(ld_ctx* ctx, long long n, const double* x, double* sum);

/* Halo exchange of a domain decomposition (the paper's Sec. 2.1.1: each
 * sub-domain is surrounded by halo regions filled from its neighbours).
 * ld_pack_planes copies the f and g of nplanes whole z-planes of the current
 * state, starting at plane z0 (taken modulo nz, the range wrapping
 * periodically), into dev_buf as [38][nplanes][ny][nx] values of the storage
 * precision (f components 0..18, then g); ld_unpack_planes writes such a
 * buffer into those planes. ld_planes_bytes gives the buffer size (0 for a
 * NULL context or nplanes < 1). Stream-ordered device-to-device copies; the
 * buffer is caller-owned device memory. LD_EINVAL for nplanes outside 1..nz
 * or a host buffer; LD_ESTATE before the state is initialised. */
size_t ld_planes_bytes(const ld_ctx* ctx, int nplanes);
int ld_pack_planes(ld_ctx* ctx, int z0, int nplanes, void* dev_buf);
int ld_unpack_planes(ld_ctx* ctx, int z0, int nplanes, const void* dev_buf);

/* The step kernel a context runs (LD_KERNEL_AUTO resolved for its lattice,
 * precision and options): LD_KERNEL_GENERIC, LD_KERNEL_FUSED or
 * LD_KERNEL_FUSED_STAGED; LD_EINVAL for a NULL context. */
int ld_step_kernel(const ld_ctx* ctx);

/* Advance nsteps >= 0 full timesteps (moments, phi stencil and mu, force,
 * collisions of f and g, propagation). Each step adds 1 to the step counter
 * of stochastic rounding. Asynchronous. */
int ld_step(ld_ctx* ctx, int nsteps);

/* Macroscopic fields of the current (pre-collision) state. Each output may be
 * NULL. rho, phi: double[N]; u = (j + F/2)/rho with the selected force:
 * double[3][N]; grad_phi (the selected stencil's gradient): double[3][N]; totals: double[5] =
 * {sum rho, sum phi, sum jx, sum jy, sum jz}, each summed in FP64 in a fixed
 * order (bitwise reproducible run to run). Asynchronous. */
int ld_moments(ld_ctx* ctx, double* rho, double* u, double* phi, double* grad_phi, double* totals);

/* Synchronise the stream and return LD_ENONFINITE if the state holds a NaN
 * or Inf (tested through the FP64 totals), LD_ECUDA if a kernel recorded that
 * it gave up waiting for its shared-memory copies (the steps since then are
 * invalid; ld_init clears the record), else LD_OK. Blocks the host. */
int ld_check(ld_ctx* ctx);

/* Test setting of the failure detection of ld_check (the paper has no
 * counterpart; it exercises the bounded waits of LD_KERNEL_FUSED_STAGED
 * without faulting or hanging the GPU). max_polls (>= 1) bounds every
 * barrier wait of the staged step kernel (default 2^24 polls). With probe
 * != 0 each of its threads also waits once per step on a barrier that
 * nothing arrives on, and no copy is tracked by: that wait gives up after
 * max_polls polls and records the failure that ld_check then reports, while
 * the step itself completes. LD_EINVAL for max_polls < 1. */
int ld_test_bounded_wait(ld_ctx* ctx, int max_polls, int probe);

/* Copy the current pre-collision distributions out as double[19][N] each
 * (decoded from the storage precision). Either pointer may be NULL. */
int ld_get_distributions(ld_ctx* ctx, double* f, double* g);

/* Overwrite the state with given pre-collision distributions double[19][N]
 * (encoded to the storage precision, rounding to nearest even). The
 * deviation reference of the 16-bit forms is the one fixed by ld_init, or
 * rho0-only (g reference 0) if ld_init was never called. */
int ld_set_distributions(ld_ctx* ctx, const double* f, const double* g);

/* Propagation alone on the stored bits (no collision): reverse = 0 applies
 * f_i(x + c_i) <- f_i(x); reverse = 1 applies the transpose
 * f_i(x) <- f_i(x + c_i). A permutation of raw storage values: bit-exact in
 * every precision. */
int ld_propagate(ld_ctx* ctx, int reverse);

/* Checkpoint: bytes of one saved state, and device-to-device save/restore of
 * it (caller-owned device buffer of ld_state_bytes()). Asynchronous. */
size_t ld_state_bytes(const ld_ctx* ctx);
int ld_save_state(ld_ctx* ctx, void* dev_buf);
int ld_load_state(ld_ctx* ctx, const void* dev_buf);

/* One full step from a saved state to another (both device buffers of
 * ld_state_bytes() bytes, distinct, 16-byte aligned: the step kernels move
 * rows of the state with bulk copies), without touching the context's own
 * state: used to recompute a checkpointed segment into a tape of states.
 * LD_EINVAL for host, equal or misaligned buffers, and with
 * LD_ROUND_STOCHASTIC.
 * fields_out (device, ld_fields_bytes(), or NULL) receives the phi and mu
 * fields of the source state ([phi npad][mu npad] in the arithmetic type),
 * which ld_adjoint_step can then reuse instead of recomputing them. */
size_t ld_fields_bytes(const ld_ctx* ctx);
int ld_step_between(ld_ctx* ctx, const void* src_state, void* dst_state, void* fields_out);

/* ---- Adjoint (reverse mode) of the step above, the derivative of a scalar
 * loss of the final phi with respect to the initial phi, kappa and tau_f.
 * The paper has no adjoint; these calls are the exact transpose of the
 * linearised step equations at the top of this file:
 *   reverse propagation fbar*_i(x) = fbar_i(x + c_i) (and g), then the adjoint
 *   of both collisions and of u = (j+F/2)/rho and F = -phi grad(mu), whose
 *   non-local parts are the transposed gradient and the (symmetric)
 *   Laplacian of the selected stencil; gbar_i = (1 - 1/tau_g) gbar*_i + phibar.
 * Defined for LD_FORCE_POTENTIAL with LD_COLLISION_BGK and LD_ROUND_NEAREST
 * only.
 * The adjoint state is held in the arithmetic type (FP64 for LD_FP64,
 * FP32 otherwise); parameter sums are FP64 in a fixed order. */

/* Bytes of the adjoint workspace (two adjoint states, per-site scratch,
 * per-block partials), and attaching one (device, 256-byte aligned). */
size_t ld_adjoint_workspace_bytes(const ld_ctx* ctx);
int ld_adjoint_attach(ld_ctx* ctx, void* dev_workspace, size_t bytes);

/* Adjoint state at the final time T from dL/dphi_T (device double[N]):
 * fbar = 0, gbar_i = dL/dphi_T (phi_T = sum_i g_i). */
int ld_adjoint_seed(ld_ctx* ctx, const double* phibar);

/* Map the adjoint state at t+1 to the one at t, given the forward state at
 * time t (a device state buffer as written by ld_save_state or
 * ld_step_between) and optionally its phi/mu fields from ld_step_between
 * (NULL: computed here). Adds dL/dkappa and dL/dtau_f of this step into
 * grad_params[0..1] (device doubles; NULL to skip). The context's current
 * kappa and tau_f must be those of the forward run. */
int ld_adjoint_step(ld_ctx* ctx, const void* state_t, const void* fields_t, double* grad_params);

/* Adjoint of ld_init (rho = rho0 implied; u0 the initial velocity or NULL):
 * writes dL/dphi0 (device double[N]) from the adjoint state at t = 0 and adds
 * the initialiser's dL/dkappa into grad_params[0] (NULL to skip). */
int ld_adjoint_init(ld_ctx* ctx, const double* phi0, const double* u0, double* grad_phi0, double* grad_params);

/* Read or overwrite the current adjoint state as device double[19][N] each. */
int ld_adjoint_get(ld_ctx* ctx, double* fbar, double* gbar);
int ld_adjoint_set(ld_ctx* ctx, const double* fbar, const double* gbar);

/* FP64 totals {sum rho, sum phi, sum jx, sum jy, sum jz} of distributions
 * given as device double[19][N] each (N = nx*ny*nz, the layout of
 * ld_get_distributions), written to device totals[5], on cuda_stream.
 * The paper has no counterpart to this call. It serves callers that cannot
 * allocate device memory or provide a workspace -- e.g. a monitoring or
 * checkpoint hook that must leave a running simulation's device-memory
 * footprint unchanged, or code running inside another library's allocator
 * callback: it allocates nothing, and keeps its partial sums in a fixed
 * static device array (160 KiB, held by every GPU that loads the library
 * until exit). Limit: N <= 67,108,864 sites (LD_EINVAL beyond). The first
 * call on a device looks up that array's address, with that device current,
 * and caches it; make that first call before any stream capture. The cached
 * address belongs to the device's primary context: after cudaDeviceReset on
 * that device the call is invalid for the rest of the process. Calls share
 * the array: calls that overlap on the GPU race. f and g must each hold at
 * least 19*N doubles and totals 5; only the size limit is checked here, the
 * extent of the buffers is the caller's to ensure. Summation order is fixed
 * (bitwise reproducible). No context needed; errors are read with
 * ld_last_error(NULL). */
int ld_totals_static(int nx, int ny, int nz, const double* f, const double* g, double* totals, void* cuda_stream);

/* FP64 throughput probe: the ceiling of the FP64 step, which is bound by
 * the FP64 pipe, measured on the current GPU. The paper bounds each kernel
 * by the platform's measured STREAM bandwidth and peak double-precision rate
 * (Sec. 4, Table 1 and its roofline ridge points); this call supplies the
 * second for this GPU. Launches `blocks` CTAs of 256 threads on
 * cuda_stream, each thread running 8 independent chains of `iters` FP64
 * operations: op 0 fused multiply-add, 1 add, 2 multiply (one instruction
 * each). The caller times the launch (CUDA events) and divides
 * blocks * 256 * 8 * iters by the time. sink: device double[blocks], never
 * written in practice (it keeps the chains live). LD_EINVAL for op outside
 * 0..2, blocks or iters < 1, or a host sink. Context-free; errors via
 * ld_last_error(NULL). */
int ld_probe_fp64_rate(int op, int blocks, int iters, double* sink, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Liquid crystal: the paper's Ludwig test case (Sec. 2.1.1: "Order Parameter
 * Gradients", "Chemical stress", "Collision", "Propagation", "LC Update",
 * "Advection"; the paper cites the Beris-Edwards model and the Landau-de
 * Gennes free energy without printing them). A symmetric traceless Q-tensor,
 * stored as its five components (xx, xy, xz, yy, yz; zz = -xx - yy), on the
 * same periodic D3Q19 lattice as a fluid of distributions f. One step:
 *   H_ab = -A0 (1 - gamma/3) Q_ab + A0 gamma (Q_ac Q_cb - delta_ab Q_cd Q_cd/3)
 *          - A0 gamma (Q_cd Q_cd) Q_ab + kappa lap(Q_ab)        (molecular field)
 *   sigma_ab = f delta_ab - kappa d_a Q_cd d_b Q_cd - xi H_ac (Q_cb + delta_cb/3)
 *          - xi (Q_ac + delta_ac/3) H_cb + 2 xi (Q_ab + delta_ab/3) Q_cd H_cd
 *          + Q_ac H_cb - H_ac Q_cb                                  (chemical stress)
 *   with f = A0/2 (1 - gamma/3) Q:Q - A0 gamma/3 tr(Q^3) + A0 gamma/4 (Q:Q)^2
 *          + kappa/2 |grad Q|^2;
 *   F_a = d_b sigma_ab, u = (j + F/2)/rho, BGK + Guo collision of f, propagation;
 *   Q <- Q + Gamma H + S(W, Q) - u.grad(Q), W_ab = d_b u_a,
 *   S = (xi D + Om)(Q + I/3) + (Q + I/3)(xi D - Om) - 2 xi (Q + I/3) tr(Q W),
 * d the central difference, lap the 7-point Laplacian, advection first-order
 * upwind, dt = 1. FP64 or FP32 storage and arithmetic. The same conventions
 * as the binary-fluid calls: device pointers, caller-owned workspace,
 * stream-ordered, error codes with messages from ld_last_error(NULL).
 * Step kernels (lc_params.kernel):
 *   LD_KERNEL_GENERIC: three launches, one thread per site (H and sigma;
 *     F, u, collision and push; Q update); any lattice.
 *   LD_KERNEL_FUSED: two launches. A z-marching launch keeps Q and sigma of
 *     three planes in shared memory and collides and pushes f, writing only f
 *     and u; the Q update recomputes H from Q. nx % 32 == 0, ny % 8 == 0.
 *   LD_KERNEL_AUTO: FUSED for FP32 where the lattice admits it, else GENERIC.
 * Both give the same values: the same operations in the same order. */
typedef struct {
    double A0, gamma, kappa; /* Landau-de Gennes bulk scale, ordering parameter, elastic constant */
    double Gamma, xi;        /* rotational diffusion constant, flow-aligning parameter */
    double tau_f, rho0;      /* fluid relaxation time (> 1/2), reference density */
    int precision;           /* LD_FP64 or LD_FP32 */
    int kernel;              /* LD_KERNEL_AUTO, LD_KERNEL_GENERIC or LD_KERNEL_FUSED */
} lc_params;
typedef struct lc_ctx lc_ctx;

/* Workspace of an nx*ny*nz liquid-crystal lattice (each dim >= 3); 0 for
 * invalid arguments. */
size_t lc_workspace_bytes(int nx, int ny, int nz, const lc_params* params);
/* Create a context over a 256-byte aligned device workspace of at least
 * lc_workspace_bytes() bytes, on cuda_stream. LD_EINVAL for kernel
 * LD_KERNEL_FUSED on a lattice that does not admit it. */
int lc_create(int nx, int ny, int nz, const lc_params* params, void* dev_workspace, size_t bytes, void* cuda_stream,
              lc_ctx** out);
/* Initial state: Q from device double[5][N]; f = feq(rho, u) with rho
 * double[N] (NULL: rho0) and u double[3][N] (NULL: rest). */
int lc_init(lc_ctx* ctx, const double* q, const double* rho, const double* u);
/* Advance nsteps >= 0 coupled steps (three launches each with
 * LD_KERNEL_GENERIC, two with LD_KERNEL_FUSED). */
int lc_step(lc_ctx* ctx, int nsteps);
/* The step kernel a context runs (LD_KERNEL_AUTO resolved):
 * LD_KERNEL_GENERIC or LD_KERNEL_FUSED; LD_EINVAL for a NULL context. */
int lc_step_kernel(const lc_ctx* ctx);
/* Current state as device doubles, each output may be NULL: q [5][N], rho
 * [N], u [3][N] (the velocity (j + F/2)/rho with the force of the current
 * Q), h [5][N] (molecular field), f [19][N]. */
int lc_fields(lc_ctx* ctx, double* q, double* rho, double* u, double* h, double* f);
int lc_destroy(lc_ctx* ctx);

/* Message for an error code, and the last error recorded on a context. */
const char* ld_strerror(int code);
const char* ld_last_error(const ld_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* LD_H */
