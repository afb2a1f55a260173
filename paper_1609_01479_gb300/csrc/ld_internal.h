// Host-side internals shared by the library's translation units: the
// context layout and the kernel launchers each .cu file provides.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "ld.h"

namespace ld {

struct GeomH {
    int nx, ny, nz;
    long long n, npad;
};

// Fixed reduction grid: per-block partials then one ordered final pass, so
// every FP64 sum is bitwise reproducible.
constexpr int kRedBlocks = 1024;
constexpr int kRedThreads = 256;
constexpr int kRedFields = 8;  // partial slots per block

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
    double* partials;  // kRedBlocks * kRedFields doubles
    double* totals;    // 8 doubles scratch
    float* ref;        // 38 floats: f then g deviation references
    int* status;       // device status word (kernel wait timeouts)
    cudaStream_t stream;
    bool initialized;
    int step_kernel;  // ld::StepKernel
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
inline void* f_of(const ld_ctx* c, int buf) { return c->dist[buf]; }
inline void* g_of(const ld_ctx* c, int buf) {
    return static_cast<char*>(c->dist[buf]) + dist_bytes(c) / 2;
}

// Launchers per storage precision. The FP64 set (ld_prec_f64.cu) is compiled
// without fused multiply-add contraction so that its roundings follow the
// plain operation order of the formulas; the FP32/FP16/BF16 set
// (ld_prec_lp.cu) lets the compiler contract.
#define LD_PRECISION_LAUNCHERS(NS)                                                                \
    namespace NS {                                                                                \
    cudaError_t init(ld_ctx* c, const double* phi, const double* rho, const double* u);          \
    cudaError_t phi_mu(ld_ctx* c, int buf);                                                       \
    cudaError_t collide_generic(ld_ctx* c);                                                       \
    cudaError_t macros(ld_ctx* c, double* rho, double* u, double* phi, double* grad_phi);         \
    cudaError_t totals(ld_ctx* c, double* totals);                                                \
    cudaError_t decode(ld_ctx* c, double* f, double* g);                                          \
    cudaError_t encode(ld_ctx* c, const double* f, const double* g);                              \
    cudaError_t step_fused_regs(ld_ctx* c);                                                       \
    cudaError_t step_tma(ld_ctx* c);                                                              \
    bool regs_supported(int nx, int ny, int nz);                                                  \
    bool tma_supported(int nx, int ny, int nz, int prec);                                         \
    }
LD_PRECISION_LAUNCHERS(f64)
LD_PRECISION_LAUNCHERS(lp)
#undef LD_PRECISION_LAUNCHERS

// Precision-independent (ld_prec_lp.cu).
cudaError_t launch_propagate(ld_ctx* c, int reverse);
cudaError_t launch_default_refs(ld_ctx* c);

// Step kernels (ld_ctx::step_kernel).
enum StepKernel { kStepGeneric = 1, kStepTma = 2, kStepRegs = 3 };
// The kernel a request resolves to for this lattice and precision, or 0 if
// the requested one cannot run it.
int choose_step_kernel(int nx, int ny, int nz, int prec, int requested);

inline bool is_f64(const ld_ctx* c) { return c->prec == LD_FP64; }
inline cudaError_t launch_init(ld_ctx* c, const double* phi, const double* rho, const double* u) {
    return is_f64(c) ? f64::init(c, phi, rho, u) : lp::init(c, phi, rho, u);
}
inline cudaError_t launch_phi_mu(ld_ctx* c, int buf) { return is_f64(c) ? f64::phi_mu(c, buf) : lp::phi_mu(c, buf); }
inline cudaError_t launch_collide_generic(ld_ctx* c) {
    return is_f64(c) ? f64::collide_generic(c) : lp::collide_generic(c);
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
inline cudaError_t launch_step_fused(ld_ctx* c) {
    if (c->step_kernel == kStepTma) return is_f64(c) ? f64::step_tma(c) : lp::step_tma(c);
    return is_f64(c) ? f64::step_fused_regs(c) : lp::step_fused_regs(c);
}

}  // namespace ld
