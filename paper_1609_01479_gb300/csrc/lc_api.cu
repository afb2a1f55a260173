// C ABI of the liquid-crystal timestep (declared in include/ld.h): argument
// checks, the workspace layout and the launch order of each call.
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#include "lc_internal.h"
#include "ld_internal.h"

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
long long npad_of(long long n) { return (n + 63) / 64 * 64; }

bool lc_params_ok(const lc_params* p, const char** why) {
    if (!p) return *why = "params is NULL", false;
    if (p->precision != LD_FP64 && p->precision != LD_FP32) return *why = "precision must be LD_FP64 or LD_FP32", false;
    if (p->kernel != LD_KERNEL_AUTO && p->kernel != LD_KERNEL_GENERIC && p->kernel != LD_KERNEL_FUSED)
        return *why = "kernel must be LD_KERNEL_AUTO, LD_KERNEL_GENERIC or LD_KERNEL_FUSED", false;
    if (!(p->tau_f > 0.5)) return *why = "tau_f must exceed 1/2", false;
    if (!(p->rho0 > 0.0)) return *why = "rho0 must be positive", false;
    if (!isfinite(p->A0) || !isfinite(p->gamma) || !isfinite(p->kappa) || !isfinite(p->Gamma) || !isfinite(p->xi))
        return *why = "A0, gamma, kappa, Gamma, xi must be finite", false;
    return true;
}

bool lc_dims_ok(int nx, int ny, int nz) {
    return nx >= 3 && ny >= 3 && nz >= 3 && (long long)nx * ny * nz < (1LL << 31);
}

// f ping-pong (2 x 19 npad), Q ping-pong (2 x 5 npad), H (5), sigma (9), u (3).
size_t lc_layout(int nx, int ny, int nz, int precision, size_t off[7]) {
    const long long npad = npad_of((long long)nx * ny * nz);
    const size_t rb = precision == LD_FP64 ? 8 : 4;
    const size_t comps[7] = {19, 19, 5, 5, 5, 9, 3};
    size_t o = 0;
    for (int k = 0; k < 7; ++k) {
        off[k] = o;
        o += align_up(comps[k] * (size_t)npad * rb);
    }
    return o;
}

bool opt_dev(const void* p) { return p == nullptr || ld::is_device_pointer(p); }

}  // namespace

namespace lc {
bool fused_supported(int nx, int ny, int nz) { return nx % 32 == 0 && ny % 8 == 0 && nz >= 3; }
}  // namespace lc

extern "C" {

size_t lc_workspace_bytes(int nx, int ny, int nz, const lc_params* p) {
    const char* why = nullptr;
    size_t off[7];
    if (!lc_dims_ok(nx, ny, nz) || !lc_params_ok(p, &why)) return 0;
    return lc_layout(nx, ny, nz, p->precision, off);
}

int lc_create(int nx, int ny, int nz, const lc_params* p, void* ws, size_t bytes, void* cuda_stream, lc_ctx** out) {
    const char* why = nullptr;
    if (!out) return ld::report_error(LD_EINVAL, "lc_create: out is NULL");
    *out = nullptr;
    if (!lc_dims_ok(nx, ny, nz)) return ld::report_error(LD_EINVAL, "lc_create: each dim must be >= 3");
    if (!lc_params_ok(p, &why)) return ld::report_error(LD_EINVAL, "lc_create: %s", why);
    if (!ld::is_device_pointer(ws)) return ld::report_error(LD_EINVAL, "lc_create: workspace is not a device pointer");
    if ((uintptr_t)ws % kAlign) return ld::report_error(LD_EINVAL, "lc_create: workspace must be 256-byte aligned");
    const bool fused_ok = lc::fused_supported(nx, ny, nz);
    if (p->kernel == LD_KERNEL_FUSED && !fused_ok)
        return ld::report_error(LD_EINVAL, "lc_create: LD_KERNEL_FUSED needs nx %% 32 == 0 and ny %% 8 == 0");
    size_t off[7];
    const size_t need = lc_layout(nx, ny, nz, p->precision, off);
    if (bytes < need)
        return ld::report_error(LD_EINVAL, "lc_create: workspace of %zu bytes is smaller than the %zu needed", bytes, need);
    lc_ctx* c = (lc_ctx*)calloc(1, sizeof(lc_ctx));
    if (!c) return ld::report_error(LD_EINVAL, "lc_create: host allocation of the context failed");
    c->nx = nx;
    c->ny = ny;
    c->nz = nz;
    c->n = (long long)nx * ny * nz;
    c->npad = npad_of(c->n);
    c->prm = *p;
    c->real_bytes = p->precision == LD_FP64 ? 8 : 4;
    char* w = (char*)ws;
    c->f[0] = w + off[0];
    c->f[1] = w + off[1];
    c->q[0] = w + off[2];
    c->q[1] = w + off[3];
    c->h = w + off[4];
    c->sigma = w + off[5];
    c->u = w + off[6];
    c->kernel = p->kernel == LD_KERNEL_GENERIC ? LD_KERNEL_GENERIC
              : p->kernel == LD_KERNEL_FUSED     ? LD_KERNEL_FUSED
              : (fused_ok && p->precision == LD_FP32 ? LD_KERNEL_FUSED : LD_KERNEL_GENERIC);
    int dev = 0, sms = 0;
    c->num_sms = cudaGetDevice(&dev) == cudaSuccess &&
                         cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0
                     ? sms
                     : 152;
    c->cur = 0;
    c->initialized = false;
    c->stream = (cudaStream_t)cuda_stream;
    *out = c;
    return LD_OK;
}

int lc_destroy(lc_ctx* c) {
    free(c);
    return LD_OK;
}

int lc_step_kernel(const lc_ctx* c) { return c ? c->kernel : LD_EINVAL; }

int lc_init(lc_ctx* c, const double* q, const double* rho, const double* u) {
    if (!c) return ld::report_error(LD_EINVAL, "lc_init: context is NULL");
    if (!ld::is_device_pointer(q)) return ld::report_error(LD_EINVAL, "lc_init: q must be a device pointer");
    if (!opt_dev(rho) || !opt_dev(u)) return ld::report_error(LD_EINVAL, "lc_init: rho and u must be device pointers or NULL");
    c->cur = 0;
    const cudaError_t e = c->prm.precision == LD_FP64 ? lc::f64::init(c, q, rho, u) : lc::f32::init(c, q, rho, u);
    if (e != cudaSuccess) return ld::report_error(LD_ECUDA, "lc_init: %s", cudaGetErrorString(e));
    c->initialized = true;
    return LD_OK;
}

int lc_step(lc_ctx* c, int nsteps) {
    if (!c) return ld::report_error(LD_EINVAL, "lc_step: context is NULL");
    if (!c->initialized) return ld::report_error(LD_ESTATE, "lc_step: state not initialised (call lc_init first)");
    if (nsteps < 0) return ld::report_error(LD_EINVAL, "lc_step: nsteps must be >= 0");
    for (int t = 0; t < nsteps; ++t) {
        const cudaError_t e = c->prm.precision == LD_FP64 ? lc::f64::step(c) : lc::f32::step(c);
        if (e != cudaSuccess) return ld::report_error(LD_ECUDA, "lc_step: %s", cudaGetErrorString(e));
        c->cur ^= 1;
    }
    return LD_OK;
}

int lc_fields(lc_ctx* c, double* q, double* rho, double* u, double* h, double* f) {
    if (!c) return ld::report_error(LD_EINVAL, "lc_fields: context is NULL");
    if (!c->initialized) return ld::report_error(LD_ESTATE, "lc_fields: state not initialised (call lc_init first)");
    if (!opt_dev(q) || !opt_dev(rho) || !opt_dev(u) || !opt_dev(h) || !opt_dev(f))
        return ld::report_error(LD_EINVAL, "lc_fields: outputs must be device pointers or NULL");
    const cudaError_t e =
        c->prm.precision == LD_FP64 ? lc::f64::out(c, q, rho, u, h, f) : lc::f32::out(c, q, rho, u, h, f);
    if (e != cudaSuccess) return ld::report_error(LD_ECUDA, "lc_fields: %s", cudaGetErrorString(e));
    return LD_OK;
}

}  // extern "C"
