// Host-side internals of the liquid-crystal context: its layout and the
// launchers each precision's translation unit provides.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "ld.h"

struct lc_ctx {
    int nx, ny, nz;
    long long n, npad;
    lc_params prm;
    size_t real_bytes;  // 8 (FP64) or 4 (FP32)
    void* f[2];         // distributions [19][npad], ping-pong
    void* q[2];         // Q components [5][npad], ping-pong
    void* h;            // molecular field [5][npad]
    void* sigma;        // chemical stress [9][npad]
    void* u;            // velocity [3][npad]
    int kernel;         // LD_KERNEL_GENERIC or LD_KERNEL_FUSED (resolved at create)
    int num_sms;
    int cur;
    bool initialized;
    cudaStream_t stream;
};

namespace lc {
#define LC_PRECISION_LAUNCHERS(NS)                                                            \
    namespace NS {                                                                            \
    cudaError_t init(lc_ctx* c, const double* q, const double* rho, const double* u);          \
    cudaError_t step(lc_ctx* c);                                                              \
    cudaError_t out(lc_ctx* c, double* q, double* rho, double* u, double* h, double* f);     \
    }
bool fused_supported(int nx, int ny, int nz);
LC_PRECISION_LAUNCHERS(f64)
LC_PRECISION_LAUNCHERS(f32)
#undef LC_PRECISION_LAUNCHERS
}  // namespace lc
