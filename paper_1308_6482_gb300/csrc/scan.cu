// Device-wide exclusive prefix sum of int32 values, in place, in one launch:
// a single pass with decoupled look-back (Merrill & Garland, "Single-pass
// parallel prefix scan with decoupled look-back", 2016).  Each block takes
// the next tile by an atomic ticket (so it only ever waits on tiles whose
// blocks are already running), scans it and publishes the tile total; one
// warp then looks back over the published totals of the 32 tiles before it
// at a time, down to the nearest tile that has published its inclusive
// prefix, and publishes its own.  Every wait is bounded: on timeout the block
// sets bit 2 of *err and carries on with what it has (the host reports
// LUB_ERR_TIMEOUT where it reads the flags).  Used for the cell grid and the
// per-particle pair counts of the pair builder and for the incidence lists of
// the deterministic force sum.
#include "lub_internal.cuh"
#include "scan_tile.cuh"

namespace {

using namespace scan_tile;

#ifdef LUB_TESTING
// a test build's hook: the tile that never publishes (-1: none)
__device__ int g_test_mute_tile = -1;
#endif

// state: [0] ticket counter, [1 ..] one word per tile (zeroed before the launch)
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_lookback(int32_t *__restrict__ a, int64_t n,
                                                                unsigned long long *__restrict__ state,
                                                                int32_t *__restrict__ d_total,
                                                                int32_t *__restrict__ err)
{
    pdl_wait();
    pdl_trigger();
    __shared__ int tile_s;
    if (threadIdx.x == 0) tile_s = (int)atomicAdd(state, 1ull);
    __syncthreads();
#ifdef LUB_TESTING
    scan_one_tile(a, n, state + 1, tile_s, d_total, err, g_test_mute_tile);
#else
    scan_one_tile(a, n, state + 1, tile_s, d_total, err);
#endif
}

// the aligned body in 16-byte words, the unaligned head and tail bytes by
// block 0
__global__ void __launch_bounds__(256) k_zero(uint4 *__restrict__ body, int64_t n16, unsigned char *__restrict__ head,
                                              int nhead, unsigned char *__restrict__ tail, int ntail)
{
    pdl_wait();
    pdl_trigger();
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n16; k += (int64_t)gridDim.x * blockDim.x)
        body[k] = make_uint4(0u, 0u, 0u, 0u);
    if (blockIdx.x == 0) {
        if ((int)threadIdx.x < nhead) head[threadIdx.x] = 0;
        if ((int)threadIdx.x < ntail) tail[threadIdx.x] = 0;
    }
}

}  // namespace

int zero_async(lub_ctx *ctx, int num_sms, void *ptr, size_t bytes, cudaStream_t st)
{
    if (bytes == 0) return LUB_OK;
    unsigned char *p = (unsigned char *)ptr;
    const size_t mis = (size_t)(((uintptr_t)p) & 15u);
    size_t nhead = mis ? 16 - mis : 0;
    if (nhead > bytes) nhead = bytes;
    const int64_t n16 = (int64_t)((bytes - nhead) / 16);
    const size_t ntail = bytes - nhead - (size_t)n16 * 16;
    const int grid = grid_for(n16 > 0 ? n16 : 1, 256, num_sms > 0 ? num_sms : 1, 4);
    return lub_check_cuda(ctx,
                          launch_pdl(k_zero, grid, 256, 0, st, (uint4 *)(p + nhead), n16, p, (int)nhead,
                                     p + nhead + (size_t)n16 * 16, (int)ntail),
                          "zero launch");
}

size_t scan_tmp_bytes(int64_t n) { return (size_t)(tiles_of(n) + 1) * sizeof(unsigned long long); }

int scan_exclusive(lub_ctx *ctx, int32_t *data, int64_t n, int32_t *d_total, void *tmp, size_t tmp_bytes,
                   cudaStream_t st, int32_t *err, bool state_zeroed)
{
    if (tmp_bytes < scan_tmp_bytes(n)) return lub_set_error(ctx, LUB_ERR_ARG, "scan: temp too small");
    const int64_t nt = tiles_of(n);
    if (!state_zeroed) {
        const int rc = zero_async(ctx, ctx ? ctx->num_sms : 1, tmp, scan_tmp_bytes(n), st);
        if (rc) return rc;
    }
    return lub_check_cuda(ctx,
                          launch_pdl(k_scan_lookback, (int)nt, SCAN_THREADS, 0, st, data, n,
                                     (unsigned long long *)tmp, d_total, err),
                          "scan launch");
}

#ifdef LUB_TESTING
// Test build only (no counterpart in the product library): one exclusive scan
// of n int32 values at data, in place, with tile mute_tile never publishing
// (-1: a plain scan); a timed-out look-back raises the context's timeout
// word, which lub_sync_status reports.
extern "C" int lub_test_scan(lub_ctx *ctx, int32_t *data, int64_t n, int32_t *d_total, int32_t mute_tile, void *stream)
{
    if (!ctx || !data || n < 1) return LUB_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = lub_ensure_scratch(ctx, scan_tmp_bytes(n));
    if (rc) return rc;
    rc = lub_check_cuda(ctx, cudaMemcpyToSymbolAsync(g_test_mute_tile, &mute_tile, sizeof(int), 0,
                                                     cudaMemcpyHostToDevice, st), "mute tile");
    if (!rc) rc = scan_exclusive(ctx, data, n, d_total, ctx->scratch, ctx->scratch_bytes, st, ctx->d_flags + 1);
    const int none = -1;
    if (!rc) rc = lub_check_cuda(ctx, cudaMemcpyToSymbolAsync(g_test_mute_tile, &none, sizeof(int), 0,
                                                              cudaMemcpyHostToDevice, st), "mute tile");
    if (!rc) rc = lub_check_cuda(ctx, cudaStreamSynchronize(st), "sync");
    return rc;
}
#endif
