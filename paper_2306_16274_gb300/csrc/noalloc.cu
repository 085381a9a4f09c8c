// lbm_field_totals_noalloc: FP64 totals of caller-held rho / u fields without any allocation.
//
// Who needs this: callers that cannot allocate device memory while they run -- host applications
// whose device memory is handed out up front by their own pool allocator (a cudaMalloc from inside
// them would go around their budget), and real-time loops that may not block on cudaMalloc /
// cudaFree, which can synchronise the whole device.  They bring their own input and output
// buffers; the only scratch this path needs (one partial sum per block) lives in a fixed device
// array declared below, which every GPU that loads the library holds until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_PER_THREAD = 8;                           // cells summed by one thread
constexpr int NA_CELLS_PER_BLOCK = NA_THREADS * NA_PER_THREAD;
constexpr int NA_MAX_BLOCKS = LBM_NOALLOC_MAX_CELLS / NA_CELLS_PER_BLOCK;   // 16384
static_assert(NA_MAX_BLOCKS * NA_CELLS_PER_BLOCK == LBM_NOALLOC_MAX_CELLS, "limit must be a block multiple");

// Scratch of this path: 4 doubles per block (sum rho, sum rho u_x, sum rho u_y, sum rho u_z),
// 512 KB.  Every call overwrites the partials of the blocks it launches before reading them, so
// nothing has to start at zero; calls that overlap on the GPU share this array and race.
static __device__ __align__(256) double g_partials[NA_MAX_BLOCKS * 4];

constexpr int NA_MAX_DEVICES = 64;
double* g_partials_addr[NA_MAX_DEVICES] = {};
std::mutex g_setup_mutex;

// Device address of g_partials on the current device.  In host code the symbol is only a
// host-side stand-in, so the address is looked up at set-up, once per device, with that device
// current, and kept for the life of the process.  A cudaDeviceReset destroys the context the
// address belongs to; the cached address is then stale, so this entry point does not support a
// device reset in the same process.
cudaError_t partials_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partials_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_partials);
        if (e != cudaSuccess) return e;
        g_partials_addr[dev] = static_cast<double*>(p);
    }
    *out = g_partials_addr[dev];
    return cudaSuccess;
}

// True when p is memory of the current device (device or managed allocation) aligned to `align`
// bytes.  cudaPointerGetAttributes allocates nothing; a plain host pointer reports
// cudaMemoryTypeUnregistered (or an error, which is cleared) and is refused.
bool on_current_device(const void* p, size_t align, int dev) {
    if (!p || (reinterpret_cast<uintptr_t>(p) % align) != 0) return false;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return false;
    return a.type == cudaMemoryTypeManaged || a.device == dev;
}

// Per-block partial sums in a fixed order: each thread adds its cells in index order, then a
// fixed shuffle tree and the warps in order.  Deterministic for a given ncell.
__global__ void __launch_bounds__(NA_THREADS) totals_partials_kernel(const float* __restrict__ rho,
                                                                    const float* __restrict__ u, long long n,
                                                                    double* __restrict__ partials) {
    __shared__ double red[4][NA_THREADS / 32];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const long long base = (long long)blockIdx.x * NA_CELLS_PER_BLOCK + threadIdx.x;
#pragma unroll
    for (int k = 0; k < NA_PER_THREAD; ++k) {
        const long long i = base + (long long)k * NA_THREADS;
        if (i < n) {
            const double r = rho[i];
            acc[0] += r;
            acc[1] += r * (double)u[i];
            acc[2] += r * (double)u[n + i];
            acc[3] += r * (double)u[2 * n + i];
        }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        double v = acc[c];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0) red[c][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int w = 0; w < NA_THREADS / 32; ++w) s += red[threadIdx.x][w];
        partials[4 * (long long)blockIdx.x + threadIdx.x] = s;
    }
}

__global__ void __launch_bounds__(NA_THREADS) totals_finish_kernel(const double* __restrict__ partials, int nblocks,
                                                                  double* __restrict__ totals) {
    __shared__ double red[4][NA_THREADS];
    const int t = threadIdx.x;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = t; b < nblocks; b += NA_THREADS)
        for (int c = 0; c < 4; ++c) acc[c] += partials[4 * b + c];
    for (int c = 0; c < 4; ++c) red[c][t] = acc[c];
    __syncthreads();
    for (int w = NA_THREADS / 2; w > 0; w >>= 1) {
        if (t < w)
            for (int c = 0; c < 4; ++c) red[c][t] += red[c][t + w];
        __syncthreads();
    }
    if (t < 4) totals[t] = red[t][0];
}

}  // namespace

extern "C" lbm_status lbm_field_totals_noalloc(const float* rho, const float* u, int64_t ncell, double* totals,
                                               void* cuda_stream) {
    if (!rho || !u || !totals) {
        lbm::set_thread_error("lbm_field_totals_noalloc: rho, u and totals must be device pointers");
        return LBM_ERR_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        lbm::set_thread_error("lbm_field_totals_noalloc: no current CUDA device");
        return LBM_ERR_CUDA;
    }
    if (!on_current_device(rho, alignof(float), dev) || !on_current_device(u, alignof(float), dev) ||
        !on_current_device(totals, alignof(double), dev)) {
        lbm::set_thread_error("lbm_field_totals_noalloc: rho and u must be float arrays and totals a double array "
                              "in memory of the current device (device or managed allocations), naturally aligned");
        return LBM_ERR_ARG;
    }
    if (ncell < 1 || ncell > (int64_t)LBM_NOALLOC_MAX_CELLS) {
        lbm::set_thread_error("lbm_field_totals_noalloc: ncell must lie in [1, LBM_NOALLOC_MAX_CELLS = 33554432]; "
                              "the fixed scratch array holds one partial sum per 2048 cells");
        return LBM_ERR_ARG;
    }
    double* partials = nullptr;
    const cudaError_t se = partials_address(&partials);
    if (se != cudaSuccess) {
        lbm::set_thread_error(cudaGetErrorString(se));
        return LBM_ERR_CUDA;
    }
    const cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int nblocks = (int)((ncell + NA_CELLS_PER_BLOCK - 1) / NA_CELLS_PER_BLOCK);
    totals_partials_kernel<<<nblocks, NA_THREADS, 0, st>>>(rho, u, (long long)ncell, partials);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        totals_finish_kernel<<<1, NA_THREADS, 0, st>>>(partials, nblocks, totals);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        lbm::set_thread_error(cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    return LBM_OK;
}
