// ld_probe_fp64_rate: the FP64 instruction throughput of the current GPU,
// the ceiling the FP64 step is measured against.
//
// The paper bounds each kernel by the machine's measured STREAM bandwidth
// and its peak double-precision rate (Sec. 4, Table 1, and the roofline
// ridge points that follow). The FP64 step on this GPU is bound by the FP64
// pipe, not by HBM, so that peak is measured here rather than taken from a
// data sheet: every thread runs eight independent chains of one FP64
// operation (fused multiply-add, add or multiply, each rounded once by its
// intrinsic), enough to keep the pipe busy at full occupancy.
#include "ld.h"
#include "ld_internal.h"

namespace {

constexpr int kChains = 8;

template <int OP>
__global__ void __launch_bounds__(256) k_fp64_rate(int iters, double seed, double* __restrict__ sink) {
    double a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + 1e-3 * (threadIdx.x + c);
    const double m = 0.999999999, k = 1e-12;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if (OP == 0) a[c] = __fma_rn(a[c], m, k);
            if (OP == 1) a[c] = __dadd_rn(a[c], k);
            if (OP == 2) a[c] = __dmul_rn(a[c], m);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == 12345.678) sink[blockIdx.x] = s;  // keeps the chains live; never true for these inputs
}

}  // namespace

extern "C" int ld_probe_fp64_rate(int op, int blocks, int iters, double* sink, void* cuda_stream) {
    if (op < 0 || op > 2 || blocks < 1 || iters < 1)
        return ld::report_error(LD_EINVAL, "ld_probe_fp64_rate: op in 0..2, blocks and iters >= 1");
    if (!ld::is_device_pointer(sink))
        return ld::report_error(LD_EINVAL, "ld_probe_fp64_rate: sink must be a device pointer of blocks doubles");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (op == 0) k_fp64_rate<0><<<blocks, 256, 0, s>>>(iters, 1.0, sink);
    if (op == 1) k_fp64_rate<1><<<blocks, 256, 0, s>>>(iters, 1.0, sink);
    if (op == 2) k_fp64_rate<2><<<blocks, 256, 0, s>>>(iters, 1.0, sink);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ld::report_error(LD_ECUDA, "ld_probe_fp64_rate: %s", cudaGetErrorString(e));
    return LD_OK;
}
