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
    cudaStream_t stream;
    bool initialized;
    bool fused;  // step uses the fused kernel
    char last_error[256];
};

namespace ld {

size_t dist_bytes(const ld_ctx* c);  // one buffer (f and g)
inline void* f_of(const ld_ctx* c, int buf) { return c->dist[buf]; }
inline void* g_of(const ld_ctx* c, int buf) {
    return static_cast<char*>(c->dist[buf]) + dist_bytes(c) / 2;
}

// ld_generic.cu
cudaError_t launch_init(ld_ctx* c, const double* phi, const double* rho, const double* u);
cudaError_t launch_phi_mu(ld_ctx* c, int buf);  // phi and mu scratch of buffer buf
cudaError_t launch_collide_generic(ld_ctx* c);  // one step, cur -> 1-cur (phi, mu ready)
cudaError_t launch_macros(ld_ctx* c, double* rho, double* u, double* phi, double* grad_phi);
cudaError_t launch_totals(ld_ctx* c, double* totals);
cudaError_t launch_decode(ld_ctx* c, double* f, double* g);
cudaError_t launch_encode(ld_ctx* c, const double* f, const double* g);
cudaError_t launch_propagate(ld_ctx* c, int reverse);
cudaError_t launch_default_refs(ld_ctx* c);

// ld_fused.cu
bool fused_supported(int nx, int ny, int nz);
cudaError_t launch_step_fused(ld_ctx* c);  // one step, cur -> 1-cur

}  // namespace ld
