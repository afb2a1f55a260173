// C ABI of the library (declared in include/ld.h): argument checks, the
// workspace layout, and the order of kernel launches for each call.
#include <math.h>
#include <stdint.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <nvtx3/nvToolsExt.h>

#include "ld.h"
#include "ld_internal.h"

namespace {

thread_local char g_last_error[256] = "";

constexpr size_t kAlign = 256;
constexpr int kQ = 19;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

size_t store_bytes_of(int prec) {
    switch (prec) {
        case LD_FP64: return 8;
        case LD_FP32: return 4;
        case LD_FP16DEV:
        case LD_BF16DEV: return 2;
        default: return 0;
    }
}
size_t real_bytes_of(int prec) { return prec == LD_FP64 ? 8 : 4; }

long long npad_of(long long n) { return (n + 63) / 64 * 64; }

struct Layout {
    size_t dist, phi, mu, stress, partials, totals, ref, status, total;
};

Layout layout_of(int nx, int ny, int nz, int prec, int force) {
    const long long npad = npad_of((long long)nx * ny * nz);
    Layout L;
    size_t off = 0;
    const size_t dist_one = align_up(2 * kQ * npad * store_bytes_of(prec));
    L.dist = off;
    off += 2 * dist_one;
    L.phi = off;
    off += align_up(npad * real_bytes_of(prec));
    L.mu = off;
    off += align_up(npad * real_bytes_of(prec));
    L.stress = off;  // six stress fields, only for the stress form of the force
    if (force == LD_FORCE_STRESS) off += align_up(6 * npad * real_bytes_of(prec));
    L.partials = off;
    off += align_up(sizeof(double) * ld::kRedBlocks * ld::kRedFields);
    L.totals = off;
    off += align_up(sizeof(double) * 8);
    L.ref = off;
    off += align_up(sizeof(float) * 2 * kQ);
    L.status = off;
    off += align_up(sizeof(int));
    L.total = off;
    return L;
}

int fail(ld_ctx* c, int code, const char* fmt, ...) {
    char* buf = c ? c->last_error : g_last_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 256, fmt, ap);
    va_end(ap);
    if (c) strncpy(g_last_error, c->last_error, sizeof(g_last_error) - 1);
    return code;
}

int cuda_fail(ld_ctx* c, cudaError_t e, const char* where) {
    return fail(c, LD_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

bool params_ok(const ld_params* p, const char** why) {
    if (!p) return *why = "params is NULL", false;
    if (!(p->tau_f > 0.5) || !(p->tau_g > 0.5)) return *why = "tau_f and tau_g must exceed 1/2", false;
    if (!(p->rho0 > 0.0)) return *why = "rho0 must be positive", false;
    if (!isfinite(p->A) || !isfinite(p->B) || !isfinite(p->kappa) || !isfinite(p->Gamma))
        return *why = "A, B, kappa, Gamma must be finite", false;
    if (p->precision < LD_FP64 || p->precision > LD_BF16DEV) return *why = "unknown precision", false;
    if (p->kernel < LD_KERNEL_AUTO || p->kernel > LD_KERNEL_FUSED_STAGED) return *why = "unknown kernel", false;
    if (p->stencil != LD_STENCIL_7 && p->stencil != LD_STENCIL_19) return *why = "unknown stencil", false;
    if (p->force != LD_FORCE_POTENTIAL && p->force != LD_FORCE_STRESS) return *why = "unknown force form", false;
    if (p->force == LD_FORCE_STRESS && (p->kernel == LD_KERNEL_FUSED || p->kernel == LD_KERNEL_FUSED_STAGED))
        return *why = "the stress form of the force runs on the generic kernel only", false;
    if (p->collision != LD_COLLISION_BGK && p->collision != LD_COLLISION_TRT) return *why = "unknown collision", false;
    if (p->collision == LD_COLLISION_TRT) {
        if (!(p->magic > 0.0) || !isfinite(p->magic)) return *why = "the TRT magic parameter must be positive", false;
        if (p->kernel == LD_KERNEL_FUSED || p->kernel == LD_KERNEL_FUSED_STAGED)
            return *why = "the TRT collision runs on the generic kernel only", false;
    }
    if (p->rounding != LD_ROUND_NEAREST && p->rounding != LD_ROUND_STOCHASTIC) return *why = "unknown rounding", false;
    if (p->rounding == LD_ROUND_STOCHASTIC && p->precision != LD_FP16DEV && p->precision != LD_BF16DEV)
        return *why = "stochastic rounding applies to the 16-bit storage forms only", false;
    return true;
}

bool dims_ok(int nx, int ny, int nz) {
    if (nx < 4 || ny < 4 || nz < 4) return false;
    // every index and offset fits the 64-bit arithmetic; keep n within 2^31 sites
    return (long long)nx * ny * nz < (1LL << 31);
}

// Device (or managed) memory only; host memory, pinned or not, is rejected.
bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool opt_device(const void* p) { return p == nullptr || is_device_ptr(p); }

int check_ready(ld_ctx* c) {
    if (!c) return fail(nullptr, LD_EINVAL, "context is NULL");
    if (!c->initialized) return fail(c, LD_ESTATE, "state not initialised (call ld_init or ld_load_state first)");
    return LD_OK;
}

}  // namespace

namespace ld {
size_t dist_bytes(const ld_ctx* c) { return 2 * kQ * (size_t)c->geom.npad * c->store_bytes; }

int report_error(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return code;
}

bool is_device_pointer(const void* p) { return is_device_ptr(p); }
}  // namespace ld

extern "C" {

size_t ld_workspace_bytes(int nx, int ny, int nz, const ld_params* p) {
    const char* why = nullptr;
    if (!dims_ok(nx, ny, nz) || !params_ok(p, &why)) return 0;
    return layout_of(nx, ny, nz, p->precision, p->force).total;
}

int ld_create(int nx, int ny, int nz, const ld_params* p, void* dev_workspace, size_t bytes, void* cuda_stream,
              ld_ctx** out) {
    const char* why = nullptr;
    if (!out) return fail(nullptr, LD_EINVAL, "out is NULL");
    *out = nullptr;
    if (!dims_ok(nx, ny, nz)) return fail(nullptr, LD_EINVAL, "lattice %dx%dx%d: each dim must be >= 4", nx, ny, nz);
    if (!params_ok(p, &why)) return fail(nullptr, LD_EINVAL, "%s", why);
    const Layout L = layout_of(nx, ny, nz, p->precision, p->force);
    if (!is_device_ptr(dev_workspace)) return fail(nullptr, LD_EINVAL, "workspace is not a device pointer");
    if ((uintptr_t)dev_workspace % kAlign) return fail(nullptr, LD_EINVAL, "workspace must be 256-byte aligned");
    if (bytes < L.total)
        return fail(nullptr, LD_EINVAL, "workspace of %zu bytes is smaller than the %zu needed", bytes, L.total);
    // the stress form of the force and the TRT collision run on the generic kernel
    const int step_kernel = p->force == LD_FORCE_STRESS || p->collision == LD_COLLISION_TRT
                                ? ld::kStepGeneric
                                : ld::choose_step_kernel(nx, ny, nz, p->precision, p->kernel);
    if (step_kernel == 0)
        return fail(nullptr, LD_EINVAL,
                    "fused kernels need nx %% 32 == 0, ny %% 8 == 0, nz %% 4 == 0 (staged: FP32/FP16DEV/BF16DEV only)");

    ld_ctx* c = (ld_ctx*)calloc(1, sizeof(ld_ctx));
    if (!c) return fail(nullptr, LD_EINVAL, "host allocation of the context failed");
    c->geom.nx = nx;
    c->geom.ny = ny;
    c->geom.nz = nz;
    c->geom.n = (long long)nx * ny * nz;
    c->geom.npad = npad_of(c->geom.n);
    c->prm = *p;
    c->prec = p->precision;
    c->store_bytes = store_bytes_of(p->precision);
    c->real_bytes = real_bytes_of(p->precision);
    c->ws = (char*)dev_workspace;
    c->ws_bytes = bytes;
    const size_t dist_one = align_up(2 * kQ * c->geom.npad * c->store_bytes);
    c->dist[0] = c->ws + L.dist;
    c->dist[1] = c->ws + L.dist + dist_one;
    c->cur = 0;
    c->sr_step = 0;
    c->phi = c->ws + L.phi;
    c->mu = c->ws + L.mu;
    c->stress = p->force == LD_FORCE_STRESS ? c->ws + L.stress : nullptr;
    c->partials = (double*)(c->ws + L.partials);
    c->totals = (double*)(c->ws + L.totals);
    c->ref = (float*)(c->ws + L.ref);
    c->status = (int*)(c->ws + L.status);
    c->wait_polls = ld::kDefaultWaitPolls;
    c->wait_probe = 0;
    c->stream = (cudaStream_t)cuda_stream;
    c->initialized = false;
    c->step_kernel = step_kernel;
    {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
            c->num_sms = sms;
        else
            c->num_sms = 152;
    }
    c->last_error[0] = '\0';
    cudaError_t e = cudaMemsetAsync(c->status, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = ld::launch_default_refs(c);
    if (e != cudaSuccess) {
        int rc = cuda_fail(nullptr, e, "ld_create");
        free(c);
        return rc;
    }
    *out = c;
    return LD_OK;
}

int ld_destroy(ld_ctx* c) {
    free(c);
    return LD_OK;
}

int ld_set_stream(ld_ctx* c, void* cuda_stream) {
    if (!c) return fail(nullptr, LD_EINVAL, "context is NULL");
    c->stream = (cudaStream_t)cuda_stream;
    return LD_OK;
}

int ld_set_params(ld_ctx* c, const ld_params* p) {
    const char* why = nullptr;
    if (!c) return fail(nullptr, LD_EINVAL, "context is NULL");
    if (!params_ok(p, &why)) return fail(c, LD_EINVAL, "%s", why);
    if (p->precision != c->prm.precision || p->kernel != c->prm.kernel || p->rho0 != c->prm.rho0 ||
        p->force != c->prm.force || p->collision != c->prm.collision || p->rounding != c->prm.rounding)
        return fail(c, LD_EINVAL,
                    "precision, kernel, rho0, the force form, the collision and the rounding are fixed at ld_create");
    c->prm = *p;
    return LD_OK;
}

}  // extern "C"

namespace {
int init_common(ld_ctx* c, const double* phi, const double* rho, const double* u, const double* ref_mean,
                const char* where) {
    if (!c) return fail(nullptr, LD_EINVAL, "context is NULL");
    if (!is_device_ptr(phi)) return fail(c, LD_EINVAL, "phi must be a device pointer");
    if (!opt_device(rho) || !opt_device(u)) return fail(c, LD_EINVAL, "rho and u must be device pointers or NULL");
    if (ref_mean && !isfinite(*ref_mean)) return fail(c, LD_EINVAL, "the reference mean must be finite");
    c->cur = 0;
    c->sr_step = 0;
    cudaError_t e = cudaMemsetAsync(c->status, 0, sizeof(int), c->stream);  // a fresh state has no failed wait
    if (e == cudaSuccess) e = ld::launch_init(c, phi, rho, u, ref_mean);
    if (e != cudaSuccess) return cuda_fail(c, e, where);
    c->initialized = true;
    return LD_OK;
}

// z-planes [z0, z0 + nplanes) of the current state as at most two runs of
// whole planes that do not wrap: (first plane, count) pairs.
int plane_runs(const ld_ctx* c, int z0, int nplanes, int run_z[2], int run_n[2]) {
    const int nz = c->geom.nz;
    const int z = ((z0 % nz) + nz) % nz;
    run_z[0] = z;
    run_n[0] = nplanes <= nz - z ? nplanes : nz - z;
    run_z[1] = 0;
    run_n[1] = nplanes - run_n[0];
    return run_n[1] > 0 ? 2 : 1;
}

// Copy whole planes between the current state (38 components, pitch npad)
// and a packed buffer [38][nplanes][ny][nx] in the storage precision.
int copy_planes(ld_ctx* c, int z0, int nplanes, void* buf, bool pack, const char* where) {
    int rc = check_ready(c);
    if (rc) return rc;
    if (nplanes < 1 || nplanes > c->geom.nz) return fail(c, LD_EINVAL, "%s: nplanes must be in 1..nz", where);
    if (!is_device_ptr(buf)) return fail(c, LD_EINVAL, "%s: the buffer must be a device pointer", where);
    const size_t S = c->store_bytes;
    const size_t plane_bytes = (size_t)c->geom.nx * c->geom.ny * S;
    const size_t pitch_state = (size_t)c->geom.npad * S, pitch_buf = (size_t)nplanes * plane_bytes;
    char* state = static_cast<char*>(c->dist[c->cur]);
    int rz[2], rn[2];
    const int runs = plane_runs(c, z0, nplanes, rz, rn);
    size_t done = 0;
    for (int r = 0; r < runs; ++r) {
        char* st = state + (size_t)rz[r] * plane_bytes;
        char* bf = static_cast<char*>(buf) + done;
        const size_t width = (size_t)rn[r] * plane_bytes;
        const cudaError_t e = pack ? cudaMemcpy2DAsync(bf, pitch_buf, st, pitch_state, width, 2 * kQ,
                                                       cudaMemcpyDeviceToDevice, c->stream)
                                   : cudaMemcpy2DAsync(st, pitch_state, bf, pitch_buf, width, 2 * kQ,
                                                       cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, where);
        done += width;
    }
    return LD_OK;
}
}  // namespace

extern "C" {

int ld_init(ld_ctx* c, const double* phi, const double* rho, const double* u) {
    return init_common(c, phi, rho, u, nullptr, "ld_init");
}

int ld_init_with_reference(ld_ctx* c, const double* phi, const double* rho, const double* u, double phi_mean) {
    return init_common(c, phi, rho, u, &phi_mean, "ld_init_with_reference");
}

int ld_field_sum(ld_ctx* c, long long n, const double* x, double* sum) {
    if (!c) return fail(nullptr, LD_EINVAL, "context is NULL");
    if (n < 1) return fail(c, LD_EINVAL, "n must be >= 1");
    if (!is_device_ptr(x) || !is_device_ptr(sum)) return fail(c, LD_EINVAL, "x and sum must be device pointers");
    const cudaError_t e = ld::launch_field_sum(c, n, x, sum);
    if (e != cudaSuccess) return cuda_fail(c, e, "ld_field_sum");
    return LD_OK;
}

size_t ld_planes_bytes(const ld_ctx* c, int nplanes) {
    if (!c || nplanes < 1) return 0;
    return 2 * kQ * (size_t)nplanes * c->geom.nx * c->geom.ny * c->store_bytes;
}

int ld_pack_planes(ld_ctx* c, int z0, int nplanes, void* dev_buf) {
    return copy_planes(c, z0, nplanes, dev_buf, true, "ld_pack_planes");
}

int ld_unpack_planes(ld_ctx* c, int z0, int nplanes, const void* dev_buf) {
    return copy_planes(c, z0, nplanes, const_cast<void*>(dev_buf), false, "ld_unpack_planes");
}

int ld_step(ld_ctx* c, int nsteps) {
    int rc = check_ready(c);
    if (rc) return rc;
    if (nsteps < 0) return fail(c, LD_EINVAL, "nsteps must be >= 0");
    nvtxRangePushA("ld_step");
    for (int t = 0; t < nsteps; ++t) {
        cudaError_t e = ld::launch_step(c, c->dist[c->cur], c->dist[1 - c->cur]);
        if (e != cudaSuccess) {
            nvtxRangePop();
            return cuda_fail(c, e, "ld_step");
        }
        c->cur ^= 1;
        ++c->sr_step;
    }
    nvtxRangePop();
    return LD_OK;
}

int ld_step_kernel(const ld_ctx* c) {
    if (!c) return LD_EINVAL;
    switch (c->step_kernel) {
        case ld::kStepGeneric: return LD_KERNEL_GENERIC;
        case ld::kStepRegs: return LD_KERNEL_FUSED;
        case ld::kStepStaged: return LD_KERNEL_FUSED_STAGED;
        default: return LD_EINVAL;
    }
}

int ld_test_bounded_wait(ld_ctx* c, int max_polls, int probe) {
    if (!c) return fail(nullptr, LD_EINVAL, "context is NULL");
    if (max_polls < 1) return fail(c, LD_EINVAL, "max_polls must be >= 1");
    c->wait_polls = max_polls;
    c->wait_probe = probe ? 1 : 0;
    return LD_OK;
}

int ld_moments(ld_ctx* c, double* rho, double* u, double* phi, double* grad_phi, double* totals) {
    int rc = check_ready(c);
    if (rc) return rc;
    if (!opt_device(rho) || !opt_device(u) || !opt_device(phi) || !opt_device(grad_phi) || !opt_device(totals))
        return fail(c, LD_EINVAL, "outputs must be device pointers or NULL");
    cudaError_t e = cudaSuccess;
    if (rho || u || phi || grad_phi) e = ld::launch_macros(c, rho, u, phi, grad_phi);
    if (e == cudaSuccess && totals) e = ld::launch_totals(c, totals);
    if (e != cudaSuccess) return cuda_fail(c, e, "ld_moments");
    return LD_OK;
}

int ld_check(ld_ctx* c) {
    int rc = check_ready(c);
    if (rc) return rc;
    double host[5];
    int status = 0;
    cudaError_t e = ld::launch_totals(c, c->totals);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, c->totals, sizeof(host), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ld_check");
    if (status & ld::kStatusBounds) return fail(c, LD_ECUDA, "a kernel caught a site index outside the lattice (debug build, status %d)", status);
    if (status) return fail(c, LD_ECUDA, "a kernel gave up waiting for its shared-memory copies (status %d)", status);
    for (int k = 0; k < 5; ++k)
        if (!isfinite(host[k])) return fail(c, LD_ENONFINITE, "state holds a non-finite value (total %d)", k);
    return LD_OK;
}

int ld_get_distributions(ld_ctx* c, double* f, double* g) {
    int rc = check_ready(c);
    if (rc) return rc;
    if (!opt_device(f) || !opt_device(g)) return fail(c, LD_EINVAL, "f and g must be device pointers or NULL");
    cudaError_t e = ld::launch_decode(c, f, g);
    if (e != cudaSuccess) return cuda_fail(c, e, "ld_get_distributions");
    return LD_OK;
}

int ld_set_distributions(ld_ctx* c, const double* f, const double* g) {
    if (!c) return fail(nullptr, LD_EINVAL, "context is NULL");
    if (!is_device_ptr(f) || !is_device_ptr(g)) return fail(c, LD_EINVAL, "f and g must be device pointers");
    cudaError_t e = ld::launch_encode(c, f, g);
    if (e != cudaSuccess) return cuda_fail(c, e, "ld_set_distributions");
    c->initialized = true;
    return LD_OK;
}

int ld_propagate(ld_ctx* c, int reverse) {
    int rc = check_ready(c);
    if (rc) return rc;
    cudaError_t e = ld::launch_propagate(c, reverse ? 1 : 0);
    if (e != cudaSuccess) return cuda_fail(c, e, "ld_propagate");
    c->cur ^= 1;
    return LD_OK;
}

size_t ld_state_bytes(const ld_ctx* c) {
    if (!c) return 0;
    return align_up(ld::dist_bytes(c)) + align_up(sizeof(float) * 2 * kQ);
}

int ld_save_state(ld_ctx* c, void* dev_buf) {
    int rc = check_ready(c);
    if (rc) return rc;
    if (!is_device_ptr(dev_buf)) return fail(c, LD_EINVAL, "buffer must be a device pointer");
    const size_t db = ld::dist_bytes(c);
    cudaError_t e = cudaMemcpyAsync(dev_buf, c->dist[c->cur], db, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((char*)dev_buf + align_up(db), c->ref, sizeof(float) * 2 * kQ, cudaMemcpyDeviceToDevice,
                            c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ld_save_state");
    return LD_OK;
}

int ld_load_state(ld_ctx* c, const void* dev_buf) {
    if (!c) return fail(nullptr, LD_EINVAL, "context is NULL");
    if (!is_device_ptr(dev_buf)) return fail(c, LD_EINVAL, "buffer must be a device pointer");
    const size_t db = ld::dist_bytes(c);
    cudaError_t e = cudaMemcpyAsync(c->dist[c->cur], dev_buf, db, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->ref, (const char*)dev_buf + align_up(db), sizeof(float) * 2 * kQ,
                            cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ld_load_state");
    c->initialized = true;
    return LD_OK;
}

// ---------------------------------------------------------------------------
// Adjoint

}  // extern "C"

namespace {
struct AdjLayout {
    size_t adj, gmb, mub, phib, pfield, part, total;
};
AdjLayout adj_layout_of(const ld_ctx* c) {
    const size_t npad = (size_t)c->geom.npad;
    const size_t rb = c->real_bytes;
    const size_t nblk = (size_t)((c->geom.n + 255) / 256);
    AdjLayout L;
    size_t off = 0;
    L.adj = off;
    off += 2 * align_up(2 * kQ * npad * rb);
    L.gmb = off;
    off += align_up(3 * npad * rb);
    L.mub = off;
    off += align_up(npad * rb);
    L.phib = off;
    off += align_up(npad * rb);
    L.pfield = off;
    off += 2 * align_up(npad * rb);
    L.part = off;
    off += align_up(2 * nblk * sizeof(double));
    L.total = off;
    return L;
}
int check_adj(ld_ctx* c) {
    if (!c) return fail(nullptr, LD_EINVAL, "context is NULL");
    if (!c->adj_ready) return fail(c, LD_ESTATE, "no adjoint workspace attached (call ld_adjoint_attach)");
    return LD_OK;
}
}  // namespace

extern "C" {

size_t ld_adjoint_workspace_bytes(const ld_ctx* c) {
    return c && c->prm.force == LD_FORCE_POTENTIAL && c->prm.collision == LD_COLLISION_BGK &&
                   c->prm.rounding == LD_ROUND_NEAREST
               ? adj_layout_of(c).total
               : 0;
}

int ld_adjoint_attach(ld_ctx* c, void* dev_workspace, size_t bytes) {
    if (!c) return fail(nullptr, LD_EINVAL, "context is NULL");
    if (c->prm.force != LD_FORCE_POTENTIAL || c->prm.collision != LD_COLLISION_BGK)
        return fail(c, LD_EINVAL, "the adjoint is built for the BGK collision with F = -phi grad(mu) only");
    if (c->prm.rounding != LD_ROUND_NEAREST)
        return fail(c, LD_EINVAL, "the adjoint's recomputation needs round-to-nearest storage");
    const AdjLayout L = adj_layout_of(c);
    if (!is_device_ptr(dev_workspace)) return fail(c, LD_EINVAL, "adjoint workspace is not a device pointer");
    if ((uintptr_t)dev_workspace % kAlign) return fail(c, LD_EINVAL, "adjoint workspace must be 256-byte aligned");
    if (bytes < L.total)
        return fail(c, LD_EINVAL, "adjoint workspace of %zu bytes is smaller than the %zu needed", bytes, L.total);
    char* w = (char*)dev_workspace;
    const size_t one = align_up(2 * kQ * (size_t)c->geom.npad * c->real_bytes);
    c->adj[0] = w + L.adj;
    c->adj[1] = w + L.adj + one;
    c->adj_gmb = w + L.gmb;
    c->adj_mub = w + L.mub;
    c->adj_phib = w + L.phib;
    c->adj_p[0] = w + L.pfield;
    c->adj_p[1] = w + L.pfield + align_up((size_t)c->geom.npad * c->real_bytes);
    c->adj_part = (double*)(w + L.part);
    c->adj_cur = 0;
    c->adj_ready = true;
    return LD_OK;
}

size_t ld_fields_bytes(const ld_ctx* c) { return c ? align_up(2 * (size_t)c->geom.npad * c->real_bytes) : 0; }

int ld_step_between(ld_ctx* c, const void* src_state, void* dst_state, void* fields_out) {
    int rc = check_ready(c);
    if (rc) return rc;
    if (c->prm.rounding != LD_ROUND_NEAREST)
        return fail(c, LD_EINVAL, "ld_step_between has no step counter for stochastic rounding");
    if (!is_device_ptr(src_state) || !is_device_ptr(dst_state) || src_state == dst_state)
        return fail(c, LD_EINVAL, "src and dst must be distinct device state buffers");
    if ((uintptr_t)src_state % 16 || (uintptr_t)dst_state % 16)
        return fail(c, LD_EINVAL, "src and dst state buffers must be 16-byte aligned");
    if (!opt_device(fields_out)) return fail(c, LD_EINVAL, "fields_out must be a device pointer or NULL");
    cudaError_t e = ld::launch_step(c, src_state, dst_state, fields_out);
    if (e != cudaSuccess) return cuda_fail(c, e, "ld_step_between");
    return LD_OK;
}

int ld_adjoint_seed(ld_ctx* c, const double* phibar) {
    int rc = check_adj(c);
    if (rc) return rc;
    if (!is_device_ptr(phibar)) return fail(c, LD_EINVAL, "phibar must be a device pointer");
    cudaError_t e = ld::launch_adj_seed(c, phibar);
    if (e != cudaSuccess) return cuda_fail(c, e, "ld_adjoint_seed");
    return LD_OK;
}

int ld_adjoint_step(ld_ctx* c, const void* state_t, const void* fields_t, double* grad_params) {
    int rc = check_adj(c);
    if (rc) return rc;
    if (!is_device_ptr(state_t)) return fail(c, LD_EINVAL, "state_t must be a device state buffer");
    if (!opt_device(fields_t) || !opt_device(grad_params))
        return fail(c, LD_EINVAL, "fields_t and grad_params must be device pointers or NULL");
    cudaError_t e = ld::launch_adj_step(c, state_t, fields_t, grad_params);
    if (e != cudaSuccess) return cuda_fail(c, e, "ld_adjoint_step");
    c->adj_cur ^= 1;
    return LD_OK;
}

int ld_adjoint_init(ld_ctx* c, const double* phi0, const double* u0, double* grad_phi0, double* grad_params) {
    int rc = check_adj(c);
    if (rc) return rc;
    if (!is_device_ptr(phi0) || !is_device_ptr(grad_phi0))
        return fail(c, LD_EINVAL, "phi0 and grad_phi0 must be device pointers");
    if (!opt_device(u0) || !opt_device(grad_params))
        return fail(c, LD_EINVAL, "u0 and grad_params must be device pointers or NULL");
    cudaError_t e = ld::launch_adj_init(c, phi0, u0, grad_phi0, grad_params);
    if (e != cudaSuccess) return cuda_fail(c, e, "ld_adjoint_init");
    return LD_OK;
}

int ld_adjoint_get(ld_ctx* c, double* fbar, double* gbar) {
    int rc = check_adj(c);
    if (rc) return rc;
    if (!opt_device(fbar) || !opt_device(gbar)) return fail(c, LD_EINVAL, "outputs must be device pointers or NULL");
    cudaError_t e = ld::launch_adj_io(c, 1, fbar, gbar);
    if (e != cudaSuccess) return cuda_fail(c, e, "ld_adjoint_get");
    return LD_OK;
}

int ld_adjoint_set(ld_ctx* c, const double* fbar, const double* gbar) {
    int rc = check_adj(c);
    if (rc) return rc;
    if (!is_device_ptr(fbar) || !is_device_ptr(gbar)) return fail(c, LD_EINVAL, "fbar and gbar must be device pointers");
    cudaError_t e = ld::launch_adj_io(c, 0, const_cast<double*>(fbar), const_cast<double*>(gbar));
    if (e != cudaSuccess) return cuda_fail(c, e, "ld_adjoint_set");
    return LD_OK;
}

const char* ld_strerror(int code) {
    switch (code) {
        case LD_OK: return "success";
        case LD_EINVAL: return "invalid argument";
        case LD_ECUDA: return "CUDA error";
        case LD_ENONFINITE: return "non-finite value in the state";
        case LD_ESTATE: return "call out of order";
        default: return "unknown error code";
    }
}

const char* ld_last_error(const ld_ctx* c) { return c ? c->last_error : g_last_error; }

}  // extern "C"
