// FP64 instantiation of the step kernels. Built with -fmad=false: every
// product and sum rounds separately (no fused multiply-add contraction), in
// the operation order each kernel writes -- the formulas' own order, or the
// opposite-pair forms of the collisions (ld_common.cuh).
#include "ld_fused.cuh"
#include "ld_generic.cuh"
#include "ld_adjoint.cuh"

namespace ld {
namespace f64 {

cudaError_t init(ld_ctx* c, const double* phi, const double* rho, const double* u, const double* ref_mean) {
    return init_p<LD_FP64>(c, phi, rho, u, ref_mean);
}
cudaError_t phi_mu(ld_ctx* c, const void* state) { return phi_mu_p<LD_FP64>(c, state); }
cudaError_t collide_generic(ld_ctx* c, const void* src, void* dst, void* fields) {
    return collide_p<LD_FP64>(c, src, dst, fields);
}
cudaError_t macros(ld_ctx* c, double* rho, double* u, double* phi, double* gphi) {
    return macros_p<LD_FP64>(c, rho, u, phi, gphi);
}
cudaError_t totals(ld_ctx* c, double* t) { return totals_p<LD_FP64>(c, t); }
cudaError_t decode(ld_ctx* c, double* f, double* g) { return decode_p<LD_FP64>(c, f, g); }
cudaError_t encode(ld_ctx* c, const double* f, const double* g) { return encode_p<LD_FP64>(c, f, g); }
cudaError_t step_fused_regs(ld_ctx* c, const void* src, void* dst, void* fields) {
    return step_fused_p<LD_FP64>(c, src, dst, fields);
}
// FP64 staging would not fit shared memory at the occupancy the FP64 pipe needs
cudaError_t step_staged(ld_ctx*, const void*, void*, void*) { return cudaErrorNotSupported; }
bool regs_supported(int nx, int ny, int nz) { return fused_supported_impl(nx, ny, nz); }
cudaError_t adj_step(ld_ctx* c, const void* st, const void* fields, double* grad) {
    return adj_step_p<LD_FP64>(c, st, fields, grad);
}
cudaError_t adj_seed(ld_ctx* c, const double* pb) { return adj_seed_p<LD_FP64>(c, pb); }
cudaError_t adj_init(ld_ctx* c, const double* phi0, const double* u0, double* gphi0, double* grad) {
    return adj_init_p<LD_FP64>(c, phi0, u0, gphi0, grad);
}
cudaError_t adj_io(ld_ctx* c, int to_double, double* fbar, double* gbar) {
    return adj_io_p<LD_FP64>(c, to_double, fbar, gbar);
}
bool staged_supported(int, int, int, int) { return false; }

}  // namespace f64
}  // namespace ld
