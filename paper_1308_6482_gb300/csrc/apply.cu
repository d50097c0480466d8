// K3: per-particle force and torque from the pair results (Sec. III B):
//   f_i += F_i,  t_i += T_i + (y*_i - r_i) x F_i,
//   f_j -= F_i,  t_j -= T_i + (y*_j - r_j) x F_i   (Eq. lub:resistance).
// Two variants:
//   atomic         one thread per pair, atomic adds (fast, order-dependent
//                  rounding); lanes of a warp that share particle i (pairs
//                  come sorted by i) are combined first with a segmented
//                  warp reduction, so i-side atomics drop to one per run.
//   deterministic  incidence lists (counting sort by particle, entries
//                  sorted by pair index and side), one thread per particle
//                  summing in that fixed order: bitwise reproducible.
#include "pair_force.cuh"

namespace {

template <typename T>
__device__ __forceinline__ void pair_contrib(const T *__restrict__ FT, const T *__restrict__ lever, size_t C,
                                             int k, int side, T out[6])
{
    const V3<T> F = mk<T>(FT[k], FT[C + k], FT[2 * C + k]);
    const V3<T> Tq = mk<T>(FT[3 * C + k], FT[4 * C + k], FT[5 * C + k]);
    const V3<T> l = side ? mk<T>(lever[3 * C + k], lever[4 * C + k], lever[5 * C + k])
                         : mk<T>(lever[k], lever[C + k], lever[2 * C + k]);
    const V3<T> t = add(Tq, cross(l, F));
    const T sg = side ? T(-1) : T(1);
    out[0] = sg * F.x; out[1] = sg * F.y; out[2] = sg * F.z;
    out[3] = sg * t.x; out[4] = sg * t.y; out[5] = sg * t.z;
}

template <typename T>
__global__ void __launch_bounds__(256) k_apply_atomic(const int32_t *__restrict__ pi, const int32_t *__restrict__ pj,
                                                      const int32_t *__restrict__ d_count, int32_t cap,
                                                      const T *__restrict__ FT, const T *__restrict__ lever, int n,
                                                      T *__restrict__ force, T *__restrict__ torque)
{
    pdl_wait();
    pdl_trigger();
    const int count = pair_count(d_count, cap);
    const size_t C = (size_t)cap;
    const size_t N = (size_t)n;
    // the loop bound is warp-uniform so the whole warp takes part in the shuffles
    for (int base = blockIdx.x * blockDim.x; base < count; base += gridDim.x * blockDim.x) {
        const int k = base + threadIdx.x;
        const bool active = k < count;
        int i = active ? pi[k] : -1;
        int j = active ? pj[k] : -1;
        if (i < 0 || i >= n) i = -1;
        T ci[6] = {0, 0, 0, 0, 0, 0}, cj[6] = {0, 0, 0, 0, 0, 0};
        if (i >= 0) {
            pair_contrib<T>(FT, lever, C, k, 0, ci);
            if (j >= 0 && j < n) pair_contrib<T>(FT, lever, C, k, 1, cj);
        }
        scatter_warp<T>(i, (j >= 0 && j < n) ? j : -1, N, ci, cj, force, torque);
    }
}

// deterministic variant ------------------------------------------------------
__global__ void k_inc_count(const int32_t *__restrict__ pi, const int32_t *__restrict__ pj,
                            const int32_t *__restrict__ d_count, int32_t cap, int n, int32_t *__restrict__ cnt)
{
    const int count = pair_count(d_count, cap);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
        const int i = pi[k], j = pj[k];
        if (i < 0 || i >= n) continue;
        atomicAdd(cnt + i, 1);
        if (j >= 0 && j < n) atomicAdd(cnt + j, 1);
    }
}

__global__ void k_inc_fill(const int32_t *__restrict__ pi, const int32_t *__restrict__ pj,
                           const int32_t *__restrict__ d_count, int32_t cap, int n,
                           const int32_t *__restrict__ start, int32_t *__restrict__ fill, int32_t *__restrict__ inc)
{
    const int count = pair_count(d_count, cap);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
        const int i = pi[k], j = pj[k];
        if (i < 0 || i >= n) continue;
        // the slots stay inside the 2 cap entries even if the scan's offsets were wrong (a timed-out wait)
        const int si = start[i] + atomicAdd(fill + i, 1);
        if (si >= 0 && si < 2 * cap) inc[si] = 2 * k;
        if (j >= 0 && j < n) {
            const int sj = start[j] + atomicAdd(fill + j, 1);
            if (sj >= 0 && sj < 2 * cap) inc[sj] = 2 * k + 1;
        }
    }
}

template <typename T>
__global__ void k_inc_sum(const int32_t *__restrict__ start, const int32_t *__restrict__ total,
                          int32_t *__restrict__ inc, int n, const T *__restrict__ FT, const T *__restrict__ lever,
                          int32_t cap, T *__restrict__ force, T *__restrict__ torque, int accumulate)
{
    const size_t C = (size_t)cap, N = (size_t)n;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int b = max(0, min(start[p], 2 * cap));
        const int e = max(b, min((p + 1 < n) ? start[p + 1] : *total, 2 * cap));
        // insertion sort of this particle's entries (pair index, side)
        for (int a = b + 1; a < e; ++a) {
            const int v = inc[a];
            int c = a - 1;
            while (c >= b && inc[c] > v) {
                inc[c + 1] = inc[c];
                --c;
            }
            inc[c + 1] = v;
        }
        T acc[6] = {0, 0, 0, 0, 0, 0};
        for (int a = b; a < e; ++a) {
            const int v = inc[a];
            T c6[6];
            pair_contrib<T>(FT, lever, C, v >> 1, v & 1, c6);
#pragma unroll
            for (int q = 0; q < 6; ++q) acc[q] += c6[q];
        }
        if (accumulate) {
            force[p] += acc[0]; force[N + p] += acc[1]; force[2 * N + p] += acc[2];
            torque[p] += acc[3]; torque[N + p] += acc[4]; torque[2 * N + p] += acc[5];
        } else {
            force[p] = acc[0]; force[N + p] = acc[1]; force[2 * N + p] = acc[2];
            torque[p] = acc[3]; torque[N + p] = acc[4]; torque[2 * N + p] = acc[5];
        }
    }
}

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

int launch_apply(lub_ctx *ctx, const int32_t *pi, const int32_t *pj, const int32_t *d_count, int32_t cap,
                 const void *FT, const void *lever, int32_t n, void *force, void *torque, int precision,
                 int accumulate, int deterministic, cudaStream_t st)
{
    const size_t esz = precision == LUB_MIXED ? sizeof(float) : sizeof(double);
    if (n == 0) return LUB_OK;
    if (!deterministic) {
        if (!accumulate) {
            const int rc = zero_force_torque(ctx, force, torque, 3 * (size_t)n * esz, st);
            if (rc) return rc;
        }
        if (cap == 0) return LUB_OK;
        const Shape2 sh = tuned_shape(ctx, LUB_TUNE_APPLY, cap);
        const int grid = sh.grid, block = sh.block;
        lub_trace_mark(ctx, LUB_TRACE_APPLY, st);
        if (precision == LUB_MIXED)
            (void)launch_pdl(k_apply_atomic<float>, grid, block, 0, st, pi, pj, d_count, cap, (const float *)FT,
                                                          (const float *)lever, n, (float *)force, (float *)torque);
        else
            (void)launch_pdl(k_apply_atomic<double>, grid, block, 0, st, pi, pj, d_count, cap, (const double *)FT,
                                                           (const double *)lever, n, (double *)force,
                                                           (double *)torque);
        lub_trace_mark(ctx, LUB_TRACE_APPLY, st);
        return lub_check_cuda(ctx, cudaGetLastError(), "k_apply_atomic launch");
    }
    // scratch: cnt/start [n], fill [n], inc [2 cap], total [1], scan temp
    const size_t b_cnt = align256((size_t)n * 4), b_fill = b_cnt, b_inc = align256(2 * (size_t)cap * 4 + 4);
    const size_t b_tot = 256, b_tmp = align256(scan_tmp_bytes(n));
    int rc = lub_ensure_scratch(ctx, b_cnt + b_fill + b_inc + b_tot + b_tmp);
    if (rc) return rc;
    char *s = (char *)ctx->scratch;
    int32_t *cnt = (int32_t *)s;
    int32_t *fill = (int32_t *)(s + b_cnt);
    int32_t *inc = (int32_t *)(s + b_cnt + b_fill);
    int32_t *tot = (int32_t *)(s + b_cnt + b_fill + b_inc);
    void *tmp = s + b_cnt + b_fill + b_inc + b_tot;
    rc = zero_async(ctx, ctx->num_sms, cnt, b_cnt + b_fill, st);
    if (rc) return rc;
    const int block = 256;
    const int gp = grid_for(cap > 0 ? cap : 1, block, ctx->num_sms, 8);
    k_inc_count<<<gp, block, 0, st>>>(pi, pj, d_count, cap, n, cnt);
    rc = scan_exclusive(ctx, cnt, n, tot, tmp, b_tmp, st, ctx->d_flags + 1);
    if (rc) return rc;
    k_inc_fill<<<gp, block, 0, st>>>(pi, pj, d_count, cap, n, cnt, fill, inc);
    const int gn = grid_for(n, block, ctx->num_sms, 8);
    if (precision == LUB_MIXED)
        k_inc_sum<float><<<gn, block, 0, st>>>(cnt, tot, inc, n, (const float *)FT, (const float *)lever, cap,
                                               (float *)force, (float *)torque, accumulate);
    else
        k_inc_sum<double><<<gn, block, 0, st>>>(cnt, tot, inc, n, (const double *)FT, (const double *)lever, cap,
                                                (double *)force, (double *)torque, accumulate);
    return lub_check_cuda(ctx, cudaGetLastError(), "deterministic apply launch");
}
