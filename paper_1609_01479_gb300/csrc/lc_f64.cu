// FP64 instantiation of the liquid-crystal kernels. Built with -fmad=false:
// every product and sum rounds separately, in the order the kernels write.
#include "lc_kernels.cuh"

namespace lc {
namespace f64 {
cudaError_t init(lc_ctx* c, const double* q, const double* rho, const double* u) {
    return lc_init_t<double>(c, q, rho, u);
}
cudaError_t step(lc_ctx* c) { return lc_step_t<double>(c); }
cudaError_t out(lc_ctx* c, double* q, double* rho, double* u, double* h, double* f) {
    return lc_out_t<double>(c, q, rho, u, h, f);
}
}  // namespace f64
}  // namespace lc
