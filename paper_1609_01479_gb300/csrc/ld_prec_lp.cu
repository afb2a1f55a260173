// FP32, FP16-deviation and BF16-deviation instantiations of the step
// kernels, and the launches that do not depend on the precision.
#include "ld_fused.cuh"
#include "ld_fused2.cuh"
#include "ld_generic.cuh"
#include "ld_staged.cuh"
#include "ld_adjoint.cuh"

namespace ld {
namespace lp {

#define LD_LP_DISPATCH(fn, ...)                              \
    switch (c->prec) {                                       \
        case LD_FP32: return fn<LD_FP32>(__VA_ARGS__);       \
        case LD_FP16DEV: return fn<LD_FP16DEV>(__VA_ARGS__); \
        case LD_BF16DEV: return fn<LD_BF16DEV>(__VA_ARGS__); \
        default: return cudaErrorInvalidValue;               \
    }

cudaError_t init(ld_ctx* c, const double* phi, const double* rho, const double* u, const double* ref_mean) {
    LD_LP_DISPATCH(init_p, c, phi, rho, u, ref_mean);
}
cudaError_t phi_mu(ld_ctx* c, const void* state) { LD_LP_DISPATCH(phi_mu_p, c, state); }
cudaError_t collide_generic(ld_ctx* c, const void* src, void* dst, void* fields) {
    LD_LP_DISPATCH(collide_p, c, src, dst, fields);
}
cudaError_t macros(ld_ctx* c, double* rho, double* u, double* phi, double* gphi) {
    LD_LP_DISPATCH(macros_p, c, rho, u, phi, gphi);
}
cudaError_t totals(ld_ctx* c, double* t) { LD_LP_DISPATCH(totals_p, c, t); }
cudaError_t decode(ld_ctx* c, double* f, double* g) { LD_LP_DISPATCH(decode_p, c, f, g); }
cudaError_t encode(ld_ctx* c, const double* f, const double* g) { LD_LP_DISPATCH(encode_p, c, f, g); }
cudaError_t step_fused_regs(ld_ctx* c, const void* src, void* dst, void* fields) {
    // the 16-bit forms (either rounding): two sites per thread, packed FP32
    if (kPairs16) {
        if (c->prec == LD_FP16DEV) return step_fused2_p<LD_FP16DEV>(c, src, dst, fields);
        if (c->prec == LD_BF16DEV) return step_fused2_p<LD_BF16DEV>(c, src, dst, fields);
    }
    LD_LP_DISPATCH(step_fused_p, c, src, dst, fields);
}
cudaError_t step_staged(ld_ctx* c, const void* src, void* dst, void* fields) {
    LD_LP_DISPATCH(step_staged_p, c, src, dst, fields);
}
bool regs_supported(int nx, int ny, int nz) { return fused_supported_impl(nx, ny, nz); }
cudaError_t adj_step(ld_ctx* c, const void* st, const void* fields, double* grad) {
    LD_LP_DISPATCH(adj_step_p, c, st, fields, grad);
}
cudaError_t adj_seed(ld_ctx* c, const double* pb) { LD_LP_DISPATCH(adj_seed_p, c, pb); }
cudaError_t adj_init(ld_ctx* c, const double* phi0, const double* u0, double* gphi0, double* grad) {
    LD_LP_DISPATCH(adj_init_p, c, phi0, u0, gphi0, grad);
}
cudaError_t adj_io(ld_ctx* c, int to_double, double* fbar, double* gbar) {
    LD_LP_DISPATCH(adj_io_p, c, to_double, fbar, gbar);
}
bool staged_supported(int nx, int ny, int nz, int prec) {
    switch (prec) {
        case LD_FP32: return staged_supported_p<LD_FP32>(nx, ny, nz);
        case LD_FP16DEV: return staged_supported_p<LD_FP16DEV>(nx, ny, nz);
        case LD_BF16DEV: return staged_supported_p<LD_BF16DEV>(nx, ny, nz);
        default: return false;
    }
}

#undef LD_LP_DISPATCH

}  // namespace lp

cudaError_t launch_propagate(ld_ctx* c, int reverse) { return propagate_raw(c, reverse); }
cudaError_t launch_field_sum(ld_ctx* c, long long n, const double* x, double* out) {
    k_sum_field<<<kRedBlocks, kRedThreads, 0, c->stream>>>(n, x, c->partials);
    k_finalize<<<1, kRedBlocks, 0, c->stream>>>(c->partials, 1, out);
    return cudaGetLastError();
}
cudaError_t launch_default_refs(ld_ctx* c) { return default_refs(c); }
int choose_step_kernel(int nx, int ny, int nz, int prec, int requested) {
    const bool f64p = prec == LD_FP64;
    const bool staged = f64p ? f64::staged_supported(nx, ny, nz, prec) : lp::staged_supported(nx, ny, nz, prec);
    const bool regs = f64p ? f64::regs_supported(nx, ny, nz) : lp::regs_supported(nx, ny, nz);
    switch (requested) {
        case LD_KERNEL_GENERIC: return kStepGeneric;
        case LD_KERNEL_FUSED: return regs ? kStepRegs : 0;
        case LD_KERNEL_FUSED_STAGED: return staged ? kStepStaged : 0;
        // FP64 is bound by the FP64 pipe, and the three row-ordered launches
        // do less FP64 work per site than the fused step (no halo phi sums)
        case LD_KERNEL_AUTO: return regs && !f64p ? kStepRegs : kStepGeneric;
        default: return 0;
    }
}

}  // namespace ld
