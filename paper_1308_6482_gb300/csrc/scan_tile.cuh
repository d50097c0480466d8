// One tile of the device-wide exclusive prefix sum with decoupled look-back
// (Merrill & Garland, "Single-pass parallel prefix scan with decoupled
// look-back", 2016), for a block of SCAN_THREADS threads: the block scans its
// tile, publishes the tile total, and one warp looks back over the published
// totals of the 32 tiles before it at a time, down to the nearest tile that
// has published its inclusive prefix, then publishes its own.  Tiles must be
// taken in order (an atomic ticket), so that a block only waits on tiles whose
// blocks are already running.  A published word carries its flag and value
// together (one 64-bit exchange), so no other memory needs ordering before
// it and no fence precedes it.  Every wait is bounded: on timeout the block
// sets bit 2 of *err and carries on with what it has.
#pragma once

#include <stdint.h>

namespace scan_tile {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;
constexpr unsigned long long ST_AGG = 1ull << 32;     // tile total published
constexpr unsigned long long ST_PREFIX = 2ull << 32;  // inclusive prefix published
// bound of every look-back wait, in polls (~2 s of L2 round trips); a test
// build compiles a short one in
#ifndef LUB_SCAN_SPIN_LIMIT
#define LUB_SCAN_SPIN_LIMIT (1l << 22)
#endif
constexpr long kSpinLimit = LUB_SCAN_SPIN_LIMIT;

__host__ __device__ inline int64_t tiles_of(int64_t n)
{
    const int64_t t = (n + SCAN_TILE - 1) / SCAN_TILE;
    return t < 1 ? 1 : t;
}

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
    __syncthreads();  // warp_tot is reused by the next call
    return warp_off + x - v;
}

__device__ __forceinline__ unsigned long long load_state(const unsigned long long *p)
{
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

// Scan tile `tile` of a[0, n) in place.  tstate: one word per tile, zero
// before the scan.  The tile holding the last element writes the total to
// *d_total.  All SCAN_THREADS threads of the block call it.  mute_tile (a
// test build's hook, -1 otherwise): that tile never publishes, as if its
// block never ran, so that the next tile's look-back runs out.
__device__ __forceinline__ void scan_one_tile(int32_t *__restrict__ a, int64_t n, unsigned long long *tstate, int tile,
                                              int32_t *__restrict__ d_total, int32_t *__restrict__ err,
                                              int mute_tile = -1)
{
    const bool mute = tile == mute_tile;
    __shared__ int prefix_s;
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
            if (lane == 0 && !mute) atomicExch(tstate, ST_PREFIX | (unsigned)tot);
        } else {
            if (lane == 0 && !mute) atomicExch(tstate + tile, ST_AGG | (unsigned)tot);
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
                    continue;
                }
                int x = (lane <= stop) ? (int)(unsigned)(w & 0xffffffffull) : 0;
#pragma unroll
                for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                excl += x;
                if (stop < 32) break;
                top -= 32;
            }
            if (lane == 0 && !mute) atomicExch(tstate + tile, ST_PREFIX | (unsigned)(excl + tot));
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
    __syncthreads();  // prefix_s is reused by the next tile of this block
}

}  // namespace scan_tile
