// FP32 instantiation of the liquid-crystal kernels (FP32 storage and
// arithmetic; the compiler may contract products and sums).
#include "lc_kernels.cuh"

namespace lc {
namespace f32 {
cudaError_t init(lc_ctx* c, const double* q, const double* rho, const double* u) {
    return lc_init_t<float>(c, q, rho, u);
}
cudaError_t step(lc_ctx* c) { return lc_step_t<float>(c); }
cudaError_t out(lc_ctx* c, double* q, double* rho, double* u, double* h, double* f) {
    return lc_out_t<float>(c, q, rho, u, h, f);
}
}  // namespace f32
}  // namespace lc
