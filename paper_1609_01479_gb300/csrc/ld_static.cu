// ld_totals_static: the FP64 conservation totals of a set of distributions,
// computed without any allocation by the library or the caller.
//
// Some callers cannot call cudaMalloc or hand the library a workspace: a
// monitoring or checkpoint hook that inspects a running simulation must not
// change its device-memory footprint, and code that runs inside another
// library's memory-pool or allocator callback may not allocate at all. For
// them the per-block partial sums of this reduction live in one file-scope
// device array of fixed size (kStaticMaxBlocks x 5 doubles = 160 KiB), which
// every GPU that loads the library holds until the process exits.
//
// The first call on each device looks up that array's device address with
// cudaGetSymbolAddress (with the device current) and caches it; make that
// first call before any stream capture. The cached address belongs to the
// device's primary context, so after cudaDeviceReset the call is invalid
// for the rest of the process. All calls share the array: calls
// that overlap on the GPU (on different streams without ordering between
// them) race on it and their results are undefined. Each call writes every
// partial it later reads, so nothing has to start at zero.
#include <mutex>

#include "ld_common.cuh"
#include "ld_internal.h"

namespace {

constexpr int kStaticThreads = 256;
constexpr int kSitesPerThread = 64;
constexpr int kStaticMaxBlocks = 4096;
constexpr int kTotals = 5;
constexpr long long kSitesPerBlock = (long long)kStaticThreads * kSitesPerThread;
constexpr long long kStaticMaxSites = kStaticMaxBlocks * kSitesPerBlock;  // 67,108,864
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_totals_scratch[kStaticMaxBlocks * kTotals];

std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

// Block b sums sites [b*T*K, (b+1)*T*K): thread t takes b*T*K + t + j*T,
// j = 0..K-1, in that order; then a fixed shuffle tree and the warp partials
// in warp order. The partial of block b goes to partials[b*5 .. b*5+4].
__global__ void __launch_bounds__(kStaticThreads)
    k_totals_static_partial(long long n, const double* __restrict__ f, const double* __restrict__ g,
                            double* __restrict__ partials) {
    double v[kTotals] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const long long base = (long long)blockIdx.x * kSitesPerBlock + threadIdx.x;
    for (int j = 0; j < kSitesPerThread; ++j) {
        const long long s = base + (long long)j * kStaticThreads;
        if (s >= n) break;
#pragma unroll
        for (int i = 0; i < ld::Q; ++i) {
            const double fi = f[i * n + s];
            v[0] += fi;
            v[2] += ld::cx(i) * fi;
            v[3] += ld::cy(i) * fi;
            v[4] += ld::cz(i) * fi;
            v[1] += g[i * n + s];
        }
    }
    __shared__ double red[kStaticThreads / 32][kTotals];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kTotals; ++k) {
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
        if (lane == 0) red[warp][k] = v[k];
    }
    __syncthreads();
    if (threadIdx.x < kTotals) {
        double a = 0.0;
        for (int w = 0; w < kStaticThreads / 32; ++w) a += red[w][threadIdx.x];
        partials[(long long)blockIdx.x * kTotals + threadIdx.x] = a;
    }
}

// One block: thread t sums the partials of blocks t, t+T, ... in order, then
// a fixed tree over threads.
__global__ void __launch_bounds__(kStaticThreads)
    k_totals_static_final(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
    __shared__ double red[kStaticThreads / 32][kTotals];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double v[kTotals] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += kStaticThreads)
#pragma unroll
        for (int k = 0; k < kTotals; ++k) v[k] += partials[(long long)b * kTotals + k];
#pragma unroll
    for (int k = 0; k < kTotals; ++k) {
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
        if (lane == 0) red[warp][k] = v[k];
    }
    __syncthreads();
    if (threadIdx.x < kTotals) {
        double a = 0.0;
        for (int w = 0; w < kStaticThreads / 32; ++w) a += red[w][threadIdx.x];
        out[threadIdx.x] = a;
    }
}

// Device address of the static scratch on the current device (looked up once
// per device); nullptr on failure with the CUDA error in *err.
double* scratch_on_current_device(cudaError_t* err) {
    int dev = 0;
    *err = cudaGetDevice(&dev);
    if (*err != cudaSuccess) return nullptr;
    if (dev < 0 || dev >= kMaxDevices) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        *err = cudaGetSymbolAddress(&p, g_totals_scratch);
        if (*err != cudaSuccess) return nullptr;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    return g_scratch_ptr[dev];
}

}  // namespace

extern "C" int ld_totals_static(int nx, int ny, int nz, const double* f, const double* g, double* totals,
                                void* cuda_stream) {
    if (nx < 1 || ny < 1 || nz < 1) return ld::report_error(LD_EINVAL, "ld_totals_static: lattice dims must be >= 1");
    const long long n = (long long)nx * ny * nz;
    if (n > kStaticMaxSites)
        return ld::report_error(LD_EINVAL,
                                "ld_totals_static: %lld sites exceed the %lld its static scratch can reduce "
                                "(use ld_moments with a workspace)",
                                n, kStaticMaxSites);
    if (!ld::is_device_pointer(f) || !ld::is_device_pointer(g) || !ld::is_device_pointer(totals))
        return ld::report_error(LD_EINVAL, "ld_totals_static: f, g and totals must be device pointers");
    cudaError_t e = cudaSuccess;
    double* partials = scratch_on_current_device(&e);
    if (!partials) return ld::report_error(LD_ECUDA, "ld_totals_static: set-up failed: %s", cudaGetErrorString(e));
    const int nblocks = (int)((n + kSitesPerBlock - 1) / kSitesPerBlock);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    k_totals_static_partial<<<nblocks, kStaticThreads, 0, s>>>(n, f, g, partials);
    k_totals_static_final<<<1, kStaticThreads, 0, s>>>(partials, nblocks, totals);
    e = cudaGetLastError();
    if (e != cudaSuccess) return ld::report_error(LD_ECUDA, "ld_totals_static: %s", cudaGetErrorString(e));
    return LD_OK;
}
