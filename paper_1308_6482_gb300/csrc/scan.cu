// Device-wide exclusive prefix sum of int32 values, in place, in two
// launches: (1) per-tile sums; (2) each tile adds the sums of the tiles
// before it (read directly: there are few tiles) and scans itself; the last
// tile writes the total.  Used for the cell grid and the per-particle pair
// counts of the pair builder and for the incidence lists of the
// deterministic force sum.
#include "lub_internal.cuh"

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// exclusive block scan of one value per thread; returns the block total
__device__ __forceinline__ int block_exclusive(int v, int &total)
{
    __shared__ int warp_tot[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = (lane < SCAN_THREADS / 32) ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < SCAN_THREADS / 32) warp_tot[lane] = t;  // inclusive warp prefix
    }
    __syncthreads();
    const int warp_off = wid ? warp_tot[wid - 1] : 0;
    total = warp_tot[SCAN_THREADS / 32 - 1];
    __syncthreads();
    return warp_off + x - v;
}

__device__ __forceinline__ int block_sum(int v)
{
    int tot;
    block_exclusive(v, tot);
    return tot;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_tile_sums(const int32_t *__restrict__ a, int64_t n,
                                                            int32_t *__restrict__ sums)
{
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int s = 0;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        const int64_t idx = base + (int64_t)q * SCAN_THREADS + threadIdx.x;  // coalesced
        if (idx < n) s += a[idx];
    }
    const int tot = block_sum(s);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_tile_scan(int32_t *__restrict__ a, int64_t n,
                                                            const int32_t *__restrict__ sums,
                                                            int32_t *__restrict__ d_total)
{
    // prefix of this tile: sum of the tile sums before it
    int pre = 0;
    for (int t = threadIdx.x; t < (int)blockIdx.x; t += SCAN_THREADS) pre += sums[t];
    pre = block_sum(pre);
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int s = 0;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        v[q] = (base + q < n) ? a[base + q] : 0;
        s += v[q];
    }
    int tot;
    int off = block_exclusive(s, tot) + pre;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        if (base + q < n) a[base + q] = off;
        off += v[q];
    }
    if (d_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *d_total = pre + tot;
}

}  // namespace

size_t scan_tmp_bytes(int64_t n)
{
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb < 1) nb = 1;
    return (size_t)nb * sizeof(int32_t);
}

int scan_exclusive(lub_ctx *ctx, int32_t *data, int64_t n, int32_t *d_total, void *tmp, size_t tmp_bytes,
                   cudaStream_t st)
{
    if (tmp_bytes < scan_tmp_bytes(n)) return lub_set_error(ctx, LUB_ERR_ARG, "scan: temp too small");
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb < 1) nb = 1;
    int32_t *sums = (int32_t *)tmp;
    k_tile_sums<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(data, n, sums);
    k_tile_scan<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(data, n, sums, d_total);
    return lub_check_cuda(ctx, cudaGetLastError(), "scan launch");
}
