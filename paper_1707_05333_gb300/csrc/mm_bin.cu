// mm_bin.cu -- generator binning (the neighbour search of Sec. 3) and the
// device-wide exclusive scan used to compact faces.
//
// Generators go into a uniform grid of bins about one generator wide; a
// counting sort places their positions contiguously per bin (double4_32a x,y,z,id)
// so that a clipping warp streams whole bins.  Order inside a bin is whatever
// the atomics give: the clipper sorts candidates by (distance, id, image), so
// results do not depend on it.
#include "mm_internal.cuh"

namespace mm {

__device__ __forceinline__ int bin_coord(double x, double ibs, int g)
{
    int c = (int)floor(x * ibs);
    return c < 0 ? 0 : (c >= g ? g - 1 : c);
}

// Box of every cell from the box offsets (binary search; cells of a box are contiguous).
__global__ void k_fill_cbox(const long long *__restrict__ box_off, int nbox, int64_t n, int *__restrict__ cbox)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = nbox - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (box_off[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    cbox[i] = lo;
}

void launch_fill_cbox(const long long *box_off, int nbox, int64_t n, int *cbox, cudaStream_t s)
{
    int nb = (int)((n + 255) / 256);
    k_fill_cbox<<<nb, 256, 0, s>>>(box_off, nbox, n, cbox);
}

__global__ void k_bin_count(const double *__restrict__ pos, int64_t n, const BoxDev *__restrict__ boxes,
                            const int *__restrict__ cbox, int *__restrict__ bin_of, int *__restrict__ count,
                            DevStatus *st)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const BoxDev g = boxes[cbox[i]];
    double x = pos[i], y = pos[n + i], z = pos[2 * n + i];
    bool ok = (x >= 0.0 && x < g.L[0]) && (y >= 0.0 && y < g.L[1]) && (z >= 0.0 && z < g.L[2]);
    if (!ok) {
        atomicOr(&st->flags, ST_EINVAL);
        atomicExch(&st->bad_cell, (int)i);
        x = y = z = 0.0;
    }
    int b = g.bin_off + bin_coord(x, g.ibs[0], g.g[0]) +
            g.g[0] * (bin_coord(y, g.ibs[1], g.g[1]) + g.g[1] * bin_coord(z, g.ibs[2], g.g[2]));
    bin_of[i] = b;
    atomicAdd(&count[b], 1);
}

__global__ void k_bin_scatter(const double *__restrict__ pos, int64_t n, const int *__restrict__ bin_of,
                              const int *__restrict__ start, int *__restrict__ cursor, double4_32a *__restrict__ sorted)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int b = bin_of[i];
    int slot = start[b] + atomicAdd(&cursor[b], 1);
    // the generator index rides in .w as a bit pattern (no FP64 conversion to read it back)
    sorted[slot] = make_double4_32a(pos[i], pos[n + i], pos[2 * n + i], __longlong_as_double((long long)i));
}

// Order each bin's generators by index, so that everything downstream (the
// candidate batches of the clipper, hence plane order and rounding) is
// independent of the atomics' order.  Bins hold a handful of generators.
__global__ void k_bin_sort(const int *__restrict__ start, int64_t nbins, double4_32a *__restrict__ sorted,
                           float4 *__restrict__ sortedf)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nbins) return;
    const int lo = start[b], hi = start[b + 1];
    for (int k = lo + 1; k < hi; ++k) {
        double4_32a v = sorted[k];
        int m = k - 1;
        while (m >= lo && __double_as_longlong(sorted[m].w) > __double_as_longlong(v.w)) {
            sorted[m + 1] = sorted[m];
            --m;
        }
        sorted[m + 1] = v;
    }
    // FP32 copies of the positions for the clipper's candidate filter
    for (int k = lo; k < hi; ++k) {
        const double4_32a v = sorted[k];
        sortedf[k] = make_float4((float)v.x, (float)v.y, (float)v.z, 0.0f);
    }
}

void launch_bin_sort(const int *start, int64_t nbins, double4_32a *sorted, float4 *sortedf, cudaStream_t s)
{
    int nb = (int)((nbins + 255) / 256);
    k_bin_sort<<<nb, 256, 0, s>>>(start, nbins, sorted, sortedf);
}

void launch_bin_count(const double *pos, int64_t n, const BoxDev *boxes, const int *cbox, int *bin_of, int *count,
                      DevStatus *st, cudaStream_t s)
{
    int nb = (int)((n + 255) / 256);
    k_bin_count<<<nb, 256, 0, s>>>(pos, n, boxes, cbox, bin_of, count, st);
}

void launch_bin_scatter(const double *pos, int64_t n, const int *bin_of, const int *start, int *cursor,
                        double4_32a *sorted, cudaStream_t s)
{
    int nb = (int)((n + 255) / 256);
    k_bin_scatter<<<nb, 256, 0, s>>>(pos, n, bin_of, start, cursor, sorted);
}

// ---------------------------------------------------------------------------
// Exclusive scan: blocks of 1024 threads scan 4096 ints each, one block scans
// the block totals, then each block adds its offset.  out[n] = total.
// ---------------------------------------------------------------------------
constexpr int SCAN_T = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_T * SCAN_ITEMS;

__device__ __forceinline__ int block_excl_scan(int v, int *sh_warp, int &total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = (lane < (blockDim.x >> 5)) ? sh_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        sh_warp[lane] = w;  // inclusive warp totals
    }
    __syncthreads();
    total = sh_warp[(blockDim.x >> 5) - 1];
    int before = wid > 0 ? sh_warp[wid - 1] : 0;
    __syncthreads();
    return before + x - v;
}

__global__ void k_scan_tiles(const int *__restrict__ in, int *__restrict__ out, int64_t n, int *__restrict__ tile_sum)
{
    __shared__ int sh[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int total;
    int ex = block_excl_scan(s, sh, total);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) out[base + k] = ex;
        ex += v[k];
    }
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

__global__ void k_scan_sums(int *__restrict__ tile_sum, int ntiles, int *__restrict__ out, int64_t n)
{
    __shared__ int sh[32];
    int carry = 0;
    for (int b0 = 0; b0 < ntiles; b0 += SCAN_T) {
        int b = b0 + threadIdx.x;
        int v = b < ntiles ? tile_sum[b] : 0;
        int total;
        int ex = block_excl_scan(v, sh, total);
        if (b < ntiles) tile_sum[b] = carry + ex;
        carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = carry;
}

__global__ void k_scan_add(int *__restrict__ out, int64_t n, const int *__restrict__ tile_sum)
{
    int add = tile_sum[blockIdx.x];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k)
        if (base + k < n) out[base + k] += add;
}

size_t scan_tmp_size(int64_t n) { return (size_t)((n + SCAN_TILE - 1) / SCAN_TILE + 1); }

void launch_scan(const int *in, int *out, int64_t n, int *tmp, cudaStream_t s)
{
    int ntiles = (int)((n + SCAN_TILE - 1) / SCAN_TILE);
    if (ntiles < 1) ntiles = 1;
    k_scan_tiles<<<ntiles, SCAN_T, 0, s>>>(in, out, n, tmp);
    k_scan_sums<<<1, SCAN_T, 0, s>>>(tmp, ntiles, out, n);
    k_scan_add<<<ntiles, SCAN_T, 0, s>>>(out, n, tmp);
}

}  // namespace mm
