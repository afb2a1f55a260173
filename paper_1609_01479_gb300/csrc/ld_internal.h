// Host-side internals shared by the library's translation units: the
// context layout and the kernel launchers each .cu file provides.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <atomic>

#include "ld.h"

namespace ld {

struct GeomH {
    int nx, ny, nz;
    long long n, npad;
};

// Row-ordered launches: one block per segment of kRowThreads sites of one
// x-row (row r = y + ny z), so consecutive blocks cover consecutive addresses.
constexpr int kRowThreads = 128;
inline long long row_segments(const GeomH& g) {
    return (long long)g.ny * g.nz * ((g.nx + kRowThreads - 1) / kRowThreads);
}

// Fixed reduction grid: per-block partials then one ordered final pass, so
// every FP64 sum is bitwise reproducible.
constexpr int kRedBlocks = 1024;
constexpr int kRedThreads = 256;
constexpr int kRedFields = 8;  // partial slots per block

// Status bits written by kernels into the workspace status word (read by
// ld_check).
constexpr int kStatusWaitTimeout = 1;  // a bounded wait gave up
constexpr int kStatusBounds = 2;       // debug builds: a site index fell outside the lattice

// Poll limit of a kernel's barrier waits (mbarrier try_wait polls). Each
// poll returns after at most a short hardware-defined suspension, so this
// bounds a wait to well under a few seconds.
constexpr int kDefaultWaitPolls = 1 << 24;

}  // namespace ld

struct ld_ctx {
    ld::GeomH geom;
    ld_params prm;
    int prec;
    size_t store_bytes;  // bytes per stored distribution value
    size_t real_bytes;   // bytes of the arithmetic type
    char* ws;
    size_t ws_bytes;
    void* dist[2];  // each buffer: f[19][npad] then g[19][npad]
    int cur;        // index of the buffer holding the current state
    void* phi;      // real_t[npad] scratch
    void* mu;       // real_t[npad] scratch
    void* stress;   // real_t[6][npad] chemical stress (LD_FORCE_STRESS), else NULL
    double* partials;  // kRedBlocks * kRedFields doubles
    double* totals;    // 8 doubles scratch
    float* ref;        // 38 floats: f then g deviation references
    int* status;       // device status word (kernel wait timeouts)
    int wait_polls;    // poll limit of the staged kernel's barrier waits
    int wait_probe;    // test setting: the staged kernel also waits on a barrier nothing arrives on
    cudaStream_t stream;
    bool initialized;
    int step_kernel;  // ld::StepKernel
    unsigned long long sr_step;  // step counter t of stochastic rounding (0 at ld_init)
    // adjoint (attached with ld_adjoint_attach): two adjoint states
    // fbar[19][npad] + gbar[19][npad] in the arithmetic type, per-site scratch,
    // per-block FP64 partials (2 per block)
    bool adj_ready;
    int adj_cur;
    void* adj[2];
    void* adj_gmb;   // 3 x npad
    void* adj_mub;   // npad
    void* adj_phib;  // npad
    void* adj_p[2];  // per-site part of gbar of each adjoint state (npad)
    double* adj_part;
    int num_sms;      // multiprocessors of the current device
    char last_error[256];
};

namespace ld {

size_t dist_bytes(const ld_ctx* c);  // one buffer (f and g)

// ld_api.cu: record a context-free error message (returned by
// ld_last_error(NULL)) and return `code`; device-pointer test used by every
// entry point.
int report_error(int code, const char* fmt, ...);
bool is_device_pointer(const void* p);
// A state buffer (a ping-pong buffer or a saved state) holds f[19][npad]
// then g[19][npad] in the storage precision.
inline void* f_part(const ld_ctx*, const void* state) { return const_cast<void*>(state); }
inline void* g_part(const ld_ctx* c, const void* state) {
    return static_cast<char*>(const_cast<void*>(state)) + dist_bytes(c) / 2;
}
inline void* f_of(const ld_ctx* c, int buf) { return f_part(c, c->dist[buf]); }
inline void* g_of(const ld_ctx* c, int buf) { return g_part(c, c->dist[buf]); }

// Launchers per storage precision. The FP64 set (ld_prec_f64.cu) is compiled
// without fused multiply-add contraction so that its roundings follow the
// plain operation order of the formulas; the FP32/FP16/BF16 set
// (ld_prec_lp.cu) lets the compiler contract.
#define LD_PRECISION_LAUNCHERS(NS)                                                                \
    namespace NS {                                                                                \
    cudaError_t init(ld_ctx* c, const double* phi, const double* rho, const double* u,           \
                     const double* ref_mean);                                                     \
    cudaError_t phi_mu(ld_ctx* c, const void* state);                                             \
    cudaError_t collide_generic(ld_ctx* c, const void* src, void* dst, void* fields);             \
    cudaError_t macros(ld_ctx* c, double* rho, double* u, double* phi, double* grad_phi);         \
    cudaError_t totals(ld_ctx* c, double* totals);                                                \
    cudaError_t decode(ld_ctx* c, double* f, double* g);                                          \
    cudaError_t encode(ld_ctx* c, const double* f, const double* g);                              \
    cudaError_t step_fused_regs(ld_ctx* c, const void* src, void* dst, void* fields);             \
    cudaError_t step_staged(ld_ctx* c, const void* src, void* dst, void* fields);                 \
    cudaError_t adj_step(ld_ctx* c, const void* state_t, const void* fields_t, double* grad);     \
    cudaError_t adj_seed(ld_ctx* c, const double* phibar);                                        \
    cudaError_t adj_init(ld_ctx* c, const double* phi0, const double* u0, double* gphi0, double* grad); \
    cudaError_t adj_io(ld_ctx* c, int to_double, double* fbar, double* gbar);                     \
    bool regs_supported(int nx, int ny, int nz);                                                  \
    bool staged_supported(int nx, int ny, int nz, int prec);                                      \
    }
LD_PRECISION_LAUNCHERS(f64)
LD_PRECISION_LAUNCHERS(lp)
#undef LD_PRECISION_LAUNCHERS

// Precision-independent (ld_prec_lp.cu).
cudaError_t launch_propagate(ld_ctx* c, int reverse);
// FP64 sum of a device double[n] into out[0], in the fixed order ld_init
// uses for the mean of phi (the context's reduction scratch).
cudaError_t launch_field_sum(ld_ctx* c, long long n, const double* x, double* out);
cudaError_t launch_default_refs(ld_ctx* c);

// Raise a kernel's dynamic shared-memory limit to `bytes` on the current
// device, once per device (the attribute belongs to the device's context).
// Safe to call from several host threads: a repeated setting is harmless.
template <auto Kernel>
cudaError_t set_max_dynamic_smem_once(int bytes) {
    static std::atomic<unsigned long long> done{0};  // bit d: set on device d (d < 64)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
    return e;
}

// Step kernels (ld_ctx::step_kernel).
enum StepKernel { kStepGeneric = 1, kStepStaged = 2, kStepRegs = 3 };
// The kernel a request resolves to for this lattice and precision, or 0 if
// the requested one cannot run it.
int choose_step_kernel(int nx, int ny, int nz, int prec, int requested);

inline bool is_f64(const ld_ctx* c) { return c->prec == LD_FP64; }
// ref_mean: host pointer to the mean phi the 16-bit forms' g references are
// taken from, or null for the mean of the given phi.
inline cudaError_t launch_init(ld_ctx* c, const double* phi, const double* rho, const double* u,
                               const double* ref_mean = nullptr) {
    return is_f64(c) ? f64::init(c, phi, rho, u, ref_mean) : lp::init(c, phi, rho, u, ref_mean);
}
inline cudaError_t launch_phi_mu(ld_ctx* c, const void* state) {
    return is_f64(c) ? f64::phi_mu(c, state) : lp::phi_mu(c, state);
}
inline cudaError_t launch_macros(ld_ctx* c, double* rho, double* u, double* phi, double* gphi) {
    return is_f64(c) ? f64::macros(c, rho, u, phi, gphi) : lp::macros(c, rho, u, phi, gphi);
}
inline cudaError_t launch_totals(ld_ctx* c, double* t) { return is_f64(c) ? f64::totals(c, t) : lp::totals(c, t); }
inline cudaError_t launch_decode(ld_ctx* c, double* f, double* g) {
    return is_f64(c) ? f64::decode(c, f, g) : lp::decode(c, f, g);
}
inline cudaError_t launch_encode(ld_ctx* c, const double* f, const double* g) {
    return is_f64(c) ? f64::encode(c, f, g) : lp::encode(c, f, g);
}
inline cudaError_t launch_adj_step(ld_ctx* c, const void* st, const void* fields, double* grad) {
    return is_f64(c) ? f64::adj_step(c, st, fields, grad) : lp::adj_step(c, st, fields, grad);
}
inline cudaError_t launch_adj_seed(ld_ctx* c, const double* pb) {
    return is_f64(c) ? f64::adj_seed(c, pb) : lp::adj_seed(c, pb);
}
inline cudaError_t launch_adj_init(ld_ctx* c, const double* phi0, const double* u0, double* gphi0, double* grad) {
    return is_f64(c) ? f64::adj_init(c, phi0, u0, gphi0, grad) : lp::adj_init(c, phi0, u0, gphi0, grad);
}
inline cudaError_t launch_adj_io(ld_ctx* c, int to_double, double* fbar, double* gbar) {
    return is_f64(c) ? f64::adj_io(c, to_double, fbar, gbar) : lp::adj_io(c, to_double, fbar, gbar);
}

// One full step from the state in `src` to the state in `dst` (distinct
// buffers) with the context's step kernel; when `fields` is not null the phi
// and mu of the source state are also written there ([phi npad][mu npad],
// arithmetic type).
inline cudaError_t launch_step(ld_ctx* c, const void* src, void* dst, void* fields = nullptr) {
    if (c->step_kernel == kStepGeneric)
        return is_f64(c) ? f64::collide_generic(c, src, dst, fields) : lp::collide_generic(c, src, dst, fields);
    if (c->step_kernel == kStepStaged)
        return is_f64(c) ? f64::step_staged(c, src, dst, fields) : lp::step_staged(c, src, dst, fields);
    return is_f64(c) ? f64::step_fused_regs(c, src, dst, fields) : lp::step_fused_regs(c, src, dst, fields);
}

}  // namespace ld
