// mm_noalloc.cu -- conserved totals for callers that must not allocate.
//
// mm_totals needs a context, and a context allocates device memory for its
// partial sums.  Some callers cannot allocate at all: code that runs while a
// CUDA stream is being captured into a graph (cudaMalloc is not allowed
// there), code that must not synchronise the device (cudaFree does), and
// hosts that hand all device memory to their own pool and forbid any other
// allocation.  mm_totals_noalloc serves them: its scratch is the file-scope
// array below, which the CUDA runtime places in device memory when this
// library is loaded on a device and which stays there until the process
// exits.
#include <cstdio>
#include <mutex>

#include "mm_internal.cuh"

namespace {

constexpr int NA_TILE = 4096;      // cells summed into one partial
constexpr int NA_MAX_TILES = 4096; // partials the scratch holds
static_assert((long long)NA_TILE * NA_MAX_TILES == MM_TOTALS_NOALLOC_MAX_CELLS, "limit in mm.h");

// (sum, compensation) of each of the 5 components for every tile: 320 KiB.
static __device__ __align__(256) double g_totals_scratch[2 * 5 * NA_MAX_TILES];

// In host code the name g_totals_scratch is only a host-side stand-in; the
// device address comes from cudaGetSymbolAddress, once per device.
constexpr int NA_MAX_DEVICES = 64;
std::mutex g_setup_mu;
double *g_scratch_dev[NA_MAX_DEVICES] = {nullptr};

__device__ __forceinline__ void nsum_add(double &s, double &c, double x)
{
    const double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
}

// One block per tile of NA_TILE cells: Neumaier sums per thread, then a
// fixed-order tree over the block.  Every partial of this call's tiles is
// written before the final kernel reads it.
__global__ void __launch_bounds__(256) k_totals_tiles(const double *__restrict__ U, int64_t n,
                                                      double *__restrict__ part, int ntiles)
{
    __shared__ double ss[256], sc[256];
    const int64_t lo = (int64_t)blockIdx.x * NA_TILE;
    const int64_t hi = min(n, lo + NA_TILE);
    for (int k = 0; k < 5; ++k) {
        double s = 0.0, c = 0.0;
        for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) nsum_add(s, c, U[k * n + i]);
        ss[threadIdx.x] = s;
        sc[threadIdx.x] = c;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) {
                double a = ss[threadIdx.x], ca = sc[threadIdx.x];
                nsum_add(a, ca, ss[threadIdx.x + o]);
                ss[threadIdx.x] = a;
                sc[threadIdx.x] = ca + sc[threadIdx.x + o];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            part[2 * (k * ntiles + blockIdx.x)] = ss[0];
            part[2 * (k * ntiles + blockIdx.x) + 1] = sc[0];
        }
        __syncthreads();
    }
}

__global__ void k_totals_tiles_final(const double *__restrict__ part, int ntiles, double *__restrict__ totals)
{
    const int k = threadIdx.x;
    if (k >= 5) return;
    double s = 0.0, c = 0.0;
    for (int b = 0; b < ntiles; ++b) {
        nsum_add(s, c, part[2 * (k * ntiles + b)]);
        c += part[2 * (k * ntiles + b) + 1];
    }
    totals[k] = s + c;
}

void put_err(char *err, int64_t len, const char *msg)
{
    if (err && len > 0) snprintf(err, (size_t)len, "%s", msg);
}

}  // namespace

extern "C" mm_status mm_totals_noalloc(const double *U, int64_t n, double *totals, void *cuda_stream, char *err,
                                       int64_t err_len)
{
    if (!U || !totals) {
        put_err(err, err_len, "mm_totals_noalloc: U and totals must be device pointers");
        return MM_EINVAL;
    }
    if (n < 1) {
        put_err(err, err_len, "mm_totals_noalloc: n must be at least 1");
        return MM_EINVAL;
    }
    if (n > MM_TOTALS_NOALLOC_MAX_CELLS) {
        char msg[160];
        snprintf(msg, sizeof(msg), "mm_totals_noalloc: n = %lld exceeds the static scratch limit of %lld cells",
                 (long long)n, (long long)MM_TOTALS_NOALLOC_MAX_CELLS);
        put_err(err, err_len, msg);
        return MM_ECAPACITY;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        put_err(err, err_len, "mm_totals_noalloc: no usable current device");
        return MM_ECUDA;
    }
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mu);
        if (!g_scratch_dev[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_totals_scratch);
            if (e != cudaSuccess || !p) {
                put_err(err, err_len, "mm_totals_noalloc: cudaGetSymbolAddress of the scratch array failed");
                return MM_ECUDA;
            }
            g_scratch_dev[dev] = static_cast<double *>(p);
        }
        scratch = g_scratch_dev[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int ntiles = (int)((n + NA_TILE - 1) / NA_TILE);
    // An earlier, unrelated call may have left a launch error pending; take
    // it off first so that the checks below report only this call's launches
    // (an error that persists, a sticky one, shows up again at the launch).
    (void)cudaGetLastError();
    k_totals_tiles<<<ntiles, 256, 0, s>>>(U, n, scratch, ntiles);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_totals_tiles_final<<<1, 32, 0, s>>>(scratch, ntiles, totals);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        char msg[200];
        snprintf(msg, sizeof(msg), "mm_totals_noalloc: kernel launch failed: %s", cudaGetErrorString(e));
        put_err(err, err_len, msg);
        return MM_ECUDA;
    }
    return MM_OK;
}
