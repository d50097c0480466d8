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

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;
constexpr unsigned long long ST_AGG = 1ull << 32;     // tile total published
constexpr unsigned long long ST_PREFIX = 2ull << 32;  // inclusive prefix published
constexpr long kSpinLimit = 1l << 22;                 // ~0.3 s of 64 ns naps

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
    return warp_off + x - v;
}

__device__ __forceinline__ unsigned long long load_state(const unsigned long long *p)
{
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

// state: [0] ticket counter, [1 ..] one word per tile (zeroed before the launch)
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_lookback(int32_t *__restrict__ a, int64_t n,
                                                                unsigned long long *__restrict__ state,
                                                                int32_t *__restrict__ d_total,
                                                                int32_t *__restrict__ err)
{
    pdl_wait();
    pdl_trigger();
    __shared__ int tile_s, prefix_s;
    if (threadIdx.x == 0) tile_s = (int)atomicAdd(state, 1ull);
    __syncthreads();
    const int tile = tile_s;
    unsigned long long *tstate = state + 1;
    const int64_t base = (int64_t)tile * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int s = 0;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        v[q] = (base + q < n) ? a[base + q] : 0;
        s += v[q];
    }
    int tot;
    const int off = block_exclusive(s, tot);
    if (threadIdx.x < 32) {
        // warp 0: publish the tile total, then look back 32 predecessors at a
        // time (lane l reads tile - 1 - l - 32 r) down to the nearest tile
        // that has published its inclusive prefix
        const int lane = threadIdx.x;
        int excl = 0;
        if (tile == 0) {
            if (lane == 0) {
                __threadfence();
                atomicExch(tstate, ST_PREFIX | (unsigned)tot);
            }
        } else {
            if (lane == 0) {
                __threadfence();
                atomicExch(tstate + tile, ST_AGG | (unsigned)tot);
            }
            long spins = 0;
            int top = tile - 1;
            while (true) {
                const int p = top - lane;
                const unsigned long long w = p >= 0 ? load_state(tstate + p) : ST_PREFIX;
                const unsigned long long flag = w & ~0xffffffffull;
                const unsigned pre = __ballot_sync(0xffffffffu, flag == ST_PREFIX);
                const unsigned none = __ballot_sync(0xffffffffu, flag == 0);
                const int stop = pre ? __ffs(pre) - 1 : 32;  // nearest inclusive prefix in the window
                const unsigned upto = stop == 32 ? 0xffffffffu : ((2u << stop) - 1u);
                if (none & upto) {
                    // a tile up to the stop has not published yet: wait (bounded)
                    if (++spins > kSpinLimit) {
                        if (lane == 0 && err) atomicOr(err, 4);
                        break;
                    }
                    __nanosleep(64);
                    continue;
                }
                int v = (lane <= stop) ? (int)(unsigned)(w & 0xffffffffull) : 0;
#pragma unroll
                for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                excl += v;
                if (stop < 32) break;
                top -= 32;
            }
            if (lane == 0) {
                __threadfence();
                atomicExch(tstate + tile, ST_PREFIX | (unsigned)(excl + tot));
            }
        }
        if (lane == 0) {
            prefix_s = excl;
            if (d_total && (int64_t)(tile + 1) * SCAN_TILE >= n) *d_total = excl + tot;
        }
    }
    __syncthreads();
    int run = prefix_s + off;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        if (base + q < n) a[base + q] = run;
        run += v[q];
    }
}

int64_t tiles_of(int64_t n)
{
    const int64_t t = (n + SCAN_TILE - 1) / SCAN_TILE;
    return t < 1 ? 1 : t;
}

}  // namespace

size_t scan_tmp_bytes(int64_t n) { return (size_t)(tiles_of(n) + 1) * sizeof(unsigned long long); }

int scan_exclusive(lub_ctx *ctx, int32_t *data, int64_t n, int32_t *d_total, void *tmp, size_t tmp_bytes,
                   cudaStream_t st, int32_t *err, bool state_zeroed)
{
    if (tmp_bytes < scan_tmp_bytes(n)) return lub_set_error(ctx, LUB_ERR_ARG, "scan: temp too small");
    const int64_t nt = tiles_of(n);
    if (!state_zeroed) {
        const int rc = lub_check_cuda(ctx, cudaMemsetAsync(tmp, 0, scan_tmp_bytes(n), st), "scan state");
        if (rc) return rc;
    }
    return lub_check_cuda(ctx,
                          launch_pdl(k_scan_lookback, (int)nt, SCAN_THREADS, 0, st, data, n,
                                     (unsigned long long *)tmp, d_total, err),
                          "scan launch");
}
