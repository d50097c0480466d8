// K0: candidate pairs by a cell list with the pre-filters of Sec. III A.
//
//   1. cell of every particle (cell edge >= 2 Rmax + Delta_L), counting sort
//      by cell (atomic slot + scan of the cell counts); particles are copied
//      into cell order as two float4 records: position relative to the cell
//      centre and Rmax, symmetry axis and e = R_par^2 - R_perp^2;
//   2. count pass: one thread per particle (in cell order, so neighbouring
//      threads read the same cells) sweeps the 27 neighbour cells and counts
//      partners j > i passing the tests; plane-wall candidates are counted
//      separately; both counts are scanned;
//   3. write pass: the same sweep writes the partners of i at its offset and
//      sorts them, giving the canonical (i, j) order without a global sort.
// The tests run in FP32 on cell-relative coordinates with a safety margin;
// a test that falls inside the margin is decided again in FP64 from the
// original double positions, so every decision is the double-precision one.
#include <string.h>

#include "lub_internal.cuh"

namespace {

struct Grid {
    int nc[3];
    float cs[3];
    double csd[3];
    int64_t ncell;
    float cutoff;  // Delta_L
    float margin;  // absolute FP32 error allowance of the tests
};

__device__ __forceinline__ double wrap_axis(double x, double L, int periodic)
{
    return periodic ? x - L * floor(x / L) : x;
}

__device__ __forceinline__ int cell_axis(double xw, double cs, int nc)
{
    double f = floor(xw / cs);
    if (!(f >= 0.0)) f = 0.0;  // also catches NaN
    if (f > (double)(nc - 1)) f = (double)(nc - 1);
    return (int)f;
}

__global__ void k_cells_count(PView P, DView D, Grid G, int32_t *__restrict__ cell_cnt, int32_t *__restrict__ cell_of,
                              int32_t *__restrict__ slot, float rmax_bound, int32_t *__restrict__ flags)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        const double xw = wrap_axis(P.x[i], D.L[0], D.periodic[0]);
        const double yw = wrap_axis(P.y[i], D.L[1], D.periodic[1]);
        const double zw = wrap_axis(P.z[i], D.L[2], D.periodic[2]);
        const int cx = cell_axis(xw, G.csd[0], G.nc[0]);
        const int cy = cell_axis(yw, G.csd[1], G.nc[1]);
        const int cz = cell_axis(zw, G.csd[2], G.nc[2]);
        const int c = (cz * G.nc[1] + cy) * G.nc[0] + cx;
        cell_of[i] = c;
        slot[i] = atomicAdd(cell_cnt + c, 1);
        const float rm = fmaxf(P.rpar[i], P.rperp[i]);
        if (!(rm <= rmax_bound)) atomicOr(flags, 1);  // bound violated or NaN shape
    }
}

__global__ void k_cells_fill(PView P, DView D, Grid G, const int32_t *__restrict__ cell_start,
                             const int32_t *__restrict__ cell_of, const int32_t *__restrict__ slot,
                             int32_t *__restrict__ sorted, float4 *__restrict__ rec0, float4 *__restrict__ rec1)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        const int c = cell_of[i];
        const int s = cell_start[c] + slot[i];
        const int cx = c % G.nc[0], cy = (c / G.nc[0]) % G.nc[1], cz = c / (G.nc[0] * G.nc[1]);
        const double xw = wrap_axis(P.x[i], D.L[0], D.periodic[0]);
        const double yw = wrap_axis(P.y[i], D.L[1], D.periodic[1]);
        const double zw = wrap_axis(P.z[i], D.L[2], D.periodic[2]);
        const float rpar = P.rpar[i], rperp = P.rperp[i];
        const V3<float> o = quat_axis<float>(P.qw[i], P.qx[i], P.qy[i], P.qz[i]);
        sorted[s] = i;
        rec0[s] = make_float4((float)(xw - (cx + 0.5) * G.csd[0]), (float)(yw - (cy + 0.5) * G.csd[1]),
                              (float)(zw - (cz + 0.5) * G.csd[2]), fmaxf(rpar, rperp));
        rec1[s] = make_float4(o.x, o.y, o.z, rpar * rpar - rperp * rperp);
    }
}

// exact (double) form of the three tests, as in the definition
__device__ bool pair_test_fp64(const PView &P, const DView &D, int i, int j, double cutoff)
{
    const V3<double> d = min_image(D, sub(load_pos(P, j), load_pos(P, i)));
    const double r = sqrt(dot(d, d));
    const double rmi = (double)fmaxf(P.rpar[i], P.rperp[i]), rmj = (double)fmaxf(P.rpar[j], P.rperp[j]);
    if (r > rmi + rmj + cutoff) return false;
    if (r > 0.0) {
        const V3<double> e = scl(-1.0 / r, d);
        const Shape<double> si = load_shape<double>(P, i), sj = load_shape<double>(P, j);
        if (r - support(si, e) > rmj + cutoff) return false;
        if (r - support(sj, e) > rmi + cutoff) return false;
    }
    return true;
}

// decision of one candidate from the cell-order records (FP32 with margin,
// FP64 when undecided)
__device__ __forceinline__ bool pair_test(const PView &P, const DView &D, const Grid &G, int i, int j,
                                          const float4 a0, const float4 a1, const float4 b0, const float4 b1,
                                          float ox, float oy, float oz, double cutoff_d)
{
    const float dx = b0.x - a0.x + ox, dy = b0.y - a0.y + oy, dz = b0.z - a0.z + oz;
    const float r2 = dx * dx + dy * dy + dz * dz;
    const float lim = a0.w + b0.w + G.cutoff;
    const float hi = lim + G.margin;
    if (r2 > hi * hi) return false;
    bool sure = true;
    const float lo = lim - G.margin;
    if (r2 >= lo * lo) sure = false;
    const float r = sqrtf(r2);
    if (r > 0.f) {
        const float ir = 1.0f / r;
        // half-widths along the line of centres: sigma^2 = R_perp^2 + e (o.e)^2,
        // with R_perp^2 = Rmax^2 - e for prolates (e > 0) and Rmax^2 for oblates
        const float ci = (a1.x * dx + a1.y * dy + a1.z * dz) * ir;
        const float cj = (b1.x * dx + b1.y * dy + b1.z * dz) * ir;
        const float api = a1.w > 0.f ? a0.w * a0.w - a1.w : a0.w * a0.w;
        const float apj = b1.w > 0.f ? b0.w * b0.w - b1.w : b0.w * b0.w;
        const float sgi = sqrtf(fmaxf(api + a1.w * ci * ci, 0.f));
        const float sgj = sqrtf(fmaxf(apj + b1.w * cj * cj, 0.f));
        const float t1 = r - sgi - (b0.w + G.cutoff);
        const float t2 = r - sgj - (a0.w + G.cutoff);
        if (t1 > G.margin || t2 > G.margin) return false;
        if (t1 >= -G.margin || t2 >= -G.margin) sure = false;
    } else {
        sure = false;
    }
    if (sure) return true;
    return pair_test_fp64(P, D, i, j, cutoff_d);
}

template <bool WRITE>
__global__ void __launch_bounds__(128) k_pairs_sweep(PView P, DView D, Grid G, const int32_t *__restrict__ cell_start,
                                                     const int32_t *__restrict__ sorted,
                                                     const float4 *__restrict__ rec0,
                                                     const float4 *__restrict__ rec1, const int32_t *__restrict__ cell_of,
                                                     int32_t *__restrict__ cnt_pp, int32_t *__restrict__ cnt_w,
                                                     const int32_t *__restrict__ totals, int32_t cap,
                                                     int32_t *__restrict__ pair_i, int32_t *__restrict__ pair_j,
                                                     double cutoff_d)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < P.n; s += gridDim.x * blockDim.x) {
        const int i = sorted[s];
        const float4 a0 = rec0[s], a1 = rec1[s];
        const int c = cell_of[i];
        const int cx = c % G.nc[0], cy = (c / G.nc[0]) % G.nc[1], cz = c / (G.nc[0] * G.nc[1]);
        int base = 0;
        bool do_write = false;
        if (WRITE) {
            // totals[0] = particle pairs, totals[1] = wall pairs
            do_write = (int64_t)totals[0] + totals[1] <= (int64_t)cap;
            base = cnt_pp[i];
        }
        int found = 0;
        for (int dz = -1; dz <= 1; ++dz) {
            int zc = cz + dz;
            if (zc < 0 || zc >= G.nc[2]) {
                if (!D.periodic[2]) continue;
                zc = (zc + G.nc[2]) % G.nc[2];
            }
            for (int dy = -1; dy <= 1; ++dy) {
                int yc = cy + dy;
                if (yc < 0 || yc >= G.nc[1]) {
                    if (!D.periodic[1]) continue;
                    yc = (yc + G.nc[1]) % G.nc[1];
                }
                for (int dx = -1; dx <= 1; ++dx) {
                    int xc = cx + dx;
                    if (xc < 0 || xc >= G.nc[0]) {
                        if (!D.periodic[0]) continue;
                        xc = (xc + G.nc[0]) % G.nc[0];
                    }
                    // skip repeated cells along non-periodic axes only; on periodic
                    // axes with fewer than three cells each image is distinct
                    const int c2 = (zc * G.nc[1] + yc) * G.nc[0] + xc;
                    const float ox = dx * G.cs[0], oy = dy * G.cs[1], oz = dz * G.cs[2];
                    const int e = cell_start[c2 + 1];
                    for (int t = cell_start[c2]; t < e; ++t) {
                        const int j = sorted[t];
                        if (j <= i) continue;
                        if (pair_test(P, D, G, i, j, a0, a1, rec0[t], rec1[t], ox, oy, oz, cutoff_d)) {
                            if (WRITE && do_write) pair_j[base + found] = j;
                            ++found;
                        }
                    }
                }
            }
        }
        if (!WRITE) {
            cnt_pp[i] = found;
        } else if (do_write) {
            // canonical order: sort the partners of i ascending
            int32_t *pjb = pair_j + base;
            for (int a = 1; a < found; ++a) {
                const int v = pjb[a];
                int b = a - 1;
                while (b >= 0 && pjb[b] > v) {
                    pjb[b + 1] = pjb[b];
                    --b;
                }
                pjb[b + 1] = v;
            }
            for (int a = 0; a < found; ++a) pair_i[base + a] = i;
        }
        // plane walls (exact double gap)
        int wf = 0;
        int wbase = WRITE ? totals[0] + cnt_w[i] : 0;
        for (int w = 0; w < D.n_walls; ++w) {
            const Shape<double> si = load_shape<double>(P, i);
            const double hw = (double)D.wall_dir[w] * (P.z[i] - D.wall_z[w]) - support(si, mk<double>(0.0, 0.0, 1.0));
            if (hw < cutoff_d) {
                if (WRITE && do_write) {
                    pair_i[wbase + wf] = i;
                    pair_j[wbase + wf] = -1 - w;
                }
                ++wf;
            }
        }
        if (!WRITE) cnt_w[i] = wf;
    }
}

__global__ void k_total(const int32_t *__restrict__ totals, int32_t *__restrict__ d_count)
{
    const int64_t t = (int64_t)totals[0] + totals[1];
    *d_count = t > 0x7fffffff ? 0x7fffffff : (int32_t)t;
}

__global__ void k_max_semi(PView P, unsigned int *__restrict__ out)
{
    float m = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        const float r = fmaxf(P.rpar[i], P.rperp[i]);
        if (r > m) m = r;
    }
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

int launch_max_semi_axis(lub_ctx *ctx, const PView &P, float *h_out, cudaStream_t st)
{
    int rc = lub_ensure_scratch(ctx, 256);
    if (rc) return rc;
    unsigned int *d = (unsigned int *)ctx->scratch;
    rc = lub_check_cuda(ctx, cudaMemsetAsync(d, 0, sizeof(unsigned int), st), "memset");
    if (rc) return rc;
    if (P.n > 0) k_max_semi<<<grid_for(P.n, 256, ctx->num_sms, 4), 256, 0, st>>>(P, d);
    unsigned int hv = 0;
    rc = lub_check_cuda(ctx, cudaMemcpyAsync(&hv, d, sizeof(hv), cudaMemcpyDeviceToHost, st), "copy max");
    if (rc) return rc;
    rc = lub_check_cuda(ctx, cudaStreamSynchronize(st), "sync");
    if (rc) return rc;
    float f;
    memcpy(&f, &hv, sizeof(f));
    *h_out = f;
    return LUB_OK;
}

int launch_pairs_build(lub_ctx *ctx, const PView &P, const DView &D, const lub_params &prm, float rmax, int32_t *pi,
                       int32_t *pj, int32_t cap, int32_t *d_count, cudaStream_t st)
{
    const double range = 2.0 * (double)rmax + prm.list_cutoff;
    Grid G;
    for (int a = 0; a < 3; ++a) {
        int nc = (int)floor(D.L[a] / range);
        if (nc < 1) nc = 1;
        if (nc > 1024) nc = 1024;
        G.nc[a] = nc;
        G.csd[a] = D.L[a] / nc;
        G.cs[a] = (float)G.csd[a];
    }
    // keep the grid at most a few cells per particle (huge, sparse boxes)
    const int64_t cell_limit = 8 * (int64_t)P.n + 4096;
    int64_t ncell = (int64_t)G.nc[0] * G.nc[1] * G.nc[2];
    if (ncell > cell_limit) {
        const double f = cbrt((double)ncell / (double)cell_limit);
        for (int a = 0; a < 3; ++a) {
            int nc = (int)floor(G.nc[a] / f);
            G.nc[a] = nc < 1 ? 1 : nc;
            G.csd[a] = D.L[a] / G.nc[a];
            G.cs[a] = (float)G.csd[a];
        }
    }
    G.ncell = (int64_t)G.nc[0] * G.nc[1] * G.nc[2];
    G.cutoff = (float)prm.list_cutoff;
    // FP32 error of cell-relative coordinates and of the test values, with headroom
    G.margin = (float)(1e-5 * (range + 1.0));
    const int64_t N = P.n;
    // scratch layout
    const size_t b_cell = align256((G.ncell + 1) * 4), b_n = align256((N + 1) * 4), b_rec = align256(N * 16);
    const size_t b_tot = 256, b_tmp = align256(scan_tmp_bytes(G.ncell + 1 > N + 1 ? G.ncell + 1 : N + 1));
    const size_t total = b_cell + 5 * b_n + 2 * b_rec + b_tot + b_tmp;
    int rc = lub_ensure_scratch(ctx, total);
    if (rc) return rc;
    char *s = (char *)ctx->scratch;
    int32_t *cell_cnt = (int32_t *)s;
    s += b_cell;
    int32_t *cell_of = (int32_t *)s;
    s += b_n;
    int32_t *slot = (int32_t *)s;
    s += b_n;
    int32_t *sorted = (int32_t *)s;
    s += b_n;
    int32_t *cnt_pp = (int32_t *)s;
    s += b_n;
    int32_t *cnt_w = (int32_t *)s;
    s += b_n;
    float4 *rec0 = (float4 *)s;
    s += b_rec;
    float4 *rec1 = (float4 *)s;
    s += b_rec;
    int32_t *totals = (int32_t *)s;  // [0] pp, [1] wall, [2] cells
    s += b_tot;
    void *tmp = s;

    rc = lub_check_cuda(ctx, cudaMemsetAsync(cell_cnt, 0, b_cell, st), "memset cells");
    if (rc) return rc;
    rc = lub_check_cuda(ctx, cudaMemsetAsync(ctx->d_flags, 0, sizeof(int32_t), st), "memset flags");
    if (rc) return rc;
    const int block = 256;
    const int gn = grid_for(N > 0 ? N : 1, block, ctx->num_sms, 8);
    if (N > 0) k_cells_count<<<gn, block, 0, st>>>(P, D, G, cell_cnt, cell_of, slot, rmax, ctx->d_flags);
    rc = scan_exclusive(ctx, cell_cnt, G.ncell + 1, totals + 2, tmp, b_tmp, st);
    if (rc) return rc;
    if (N > 0) {
        k_cells_fill<<<gn, block, 0, st>>>(P, D, G, cell_cnt, cell_of, slot, sorted, rec0, rec1);
        const int gs = grid_for(N, 128, ctx->num_sms, 16);
        k_pairs_sweep<false><<<gs, 128, 0, st>>>(P, D, G, cell_cnt, sorted, rec0, rec1, cell_of, cnt_pp, cnt_w,
                                                 totals, cap, pi, pj, prm.list_cutoff);
        rc = scan_exclusive(ctx, cnt_pp, N, totals + 0, tmp, b_tmp, st);
        if (rc) return rc;
        rc = scan_exclusive(ctx, cnt_w, N, totals + 1, tmp, b_tmp, st);
        if (rc) return rc;
        k_pairs_sweep<true><<<gs, 128, 0, st>>>(P, D, G, cell_cnt, sorted, rec0, rec1, cell_of, cnt_pp, cnt_w,
                                                totals, cap, pi, pj, prm.list_cutoff);
    } else {
        rc = lub_check_cuda(ctx, cudaMemsetAsync(totals, 0, 8, st), "memset totals");
        if (rc) return rc;
    }
    k_total<<<1, 1, 0, st>>>(totals, d_count);
    return lub_check_cuda(ctx, cudaGetLastError(), "pairs build launch");
}

// ---------------------------------------------------------------------------
// The same build on scratch the caller provides (used by the entry point that
// allocates nothing); max_cells bounds the cell grid to fit that scratch.
// ---------------------------------------------------------------------------
size_t pairs_scratch_bytes(int64_t n, int64_t max_cells)
{
    const size_t b_cell = align256((max_cells + 1) * 4), b_n = align256((n + 1) * 4), b_rec = align256(n * 16);
    const size_t b_tot = 256, b_tmp = align256(scan_tmp_bytes(max_cells + 1 > n + 1 ? max_cells + 1 : n + 1));
    return b_cell + 5 * b_n + 2 * b_rec + b_tot + b_tmp + 256;  // + 256: flags
}

int pairs_build_on_scratch(int num_sms, void *scratch, size_t scratch_bytes, int64_t max_cells, const PView &P,
                           const DView &D, const lub_params &prm, float rmax, int32_t *pi, int32_t *pj, int32_t cap,
                           int32_t *d_count, cudaStream_t st)
{
    const double range = 2.0 * (double)rmax + prm.list_cutoff;
    Grid G;
    for (int a = 0; a < 3; ++a) {
        int nc = (int)floor(D.L[a] / range);
        if (nc < 1) nc = 1;
        if (nc > 1024) nc = 1024;
        G.nc[a] = nc;
        G.csd[a] = D.L[a] / nc;
        G.cs[a] = (float)G.csd[a];
    }
    int64_t cell_limit = 8 * (int64_t)P.n + 4096;
    if (cell_limit > max_cells) cell_limit = max_cells;
    for (int pass = 0; pass < 4; ++pass) {
        const int64_t ncell = (int64_t)G.nc[0] * G.nc[1] * G.nc[2];
        if (ncell <= cell_limit) break;
        const double f = cbrt((double)ncell / (double)cell_limit) * (1.0 + 1e-9) + (pass ? 0.01 * pass : 0.0);
        for (int a = 0; a < 3; ++a) {
            int nc = (int)floor(G.nc[a] / f);
            G.nc[a] = nc < 1 ? 1 : nc;
            G.csd[a] = D.L[a] / G.nc[a];
            G.cs[a] = (float)G.csd[a];
        }
    }
    G.ncell = (int64_t)G.nc[0] * G.nc[1] * G.nc[2];
    if (G.ncell > max_cells) return LUB_ERR_ARG;
    G.cutoff = (float)prm.list_cutoff;
    G.margin = (float)(1e-5 * (range + 1.0));
    const int64_t N = P.n;
    const size_t b_cell = align256((G.ncell + 1) * 4), b_n = align256((N + 1) * 4), b_rec = align256(N * 16);
    const size_t b_tot = 256, b_tmp = align256(scan_tmp_bytes(G.ncell + 1 > N + 1 ? G.ncell + 1 : N + 1));
    if (b_cell + 5 * b_n + 2 * b_rec + b_tot + b_tmp + 256 > scratch_bytes) return LUB_ERR_ARG;
    char *s = (char *)scratch;
    int32_t *flags = (int32_t *)s;
    s += 256;
    int32_t *cell_cnt = (int32_t *)s;
    s += b_cell;
    int32_t *cell_of = (int32_t *)s;
    s += b_n;
    int32_t *slot = (int32_t *)s;
    s += b_n;
    int32_t *sorted = (int32_t *)s;
    s += b_n;
    int32_t *cnt_pp = (int32_t *)s;
    s += b_n;
    int32_t *cnt_w = (int32_t *)s;
    s += b_n;
    float4 *rec0 = (float4 *)s;
    s += b_rec;
    float4 *rec1 = (float4 *)s;
    s += b_rec;
    int32_t *totals = (int32_t *)s;
    s += b_tot;
    void *tmp = s;
    // the scratch keeps the previous call's contents: clear what must start at zero
    if (cudaMemsetAsync(cell_cnt, 0, b_cell, st) != cudaSuccess) return LUB_ERR_CUDA;
    if (cudaMemsetAsync(flags, 0, 256, st) != cudaSuccess) return LUB_ERR_CUDA;
    const int block = 256;
    const int gn = grid_for(N > 0 ? N : 1, block, num_sms, 8);
    if (N > 0) k_cells_count<<<gn, block, 0, st>>>(P, D, G, cell_cnt, cell_of, slot, rmax, flags);
    int rc = scan_exclusive(nullptr, cell_cnt, G.ncell + 1, totals + 2, tmp, b_tmp, st);
    if (rc) return rc;
    if (N > 0) {
        k_cells_fill<<<gn, block, 0, st>>>(P, D, G, cell_cnt, cell_of, slot, sorted, rec0, rec1);
        const int gs = grid_for(N, 128, num_sms, 16);
        k_pairs_sweep<false><<<gs, 128, 0, st>>>(P, D, G, cell_cnt, sorted, rec0, rec1, cell_of, cnt_pp, cnt_w,
                                                 totals, cap, pi, pj, prm.list_cutoff);
        rc = scan_exclusive(nullptr, cnt_pp, N, totals + 0, tmp, b_tmp, st);
        if (rc) return rc;
        rc = scan_exclusive(nullptr, cnt_w, N, totals + 1, tmp, b_tmp, st);
        if (rc) return rc;
        k_pairs_sweep<true><<<gs, 128, 0, st>>>(P, D, G, cell_cnt, sorted, rec0, rec1, cell_of, cnt_pp, cnt_w,
                                                totals, cap, pi, pj, prm.list_cutoff);
    } else {
        if (cudaMemsetAsync(totals, 0, 8, st) != cudaSuccess) return LUB_ERR_CUDA;
    }
    k_total<<<1, 1, 0, st>>>(totals, d_count);
    return cudaGetLastError() == cudaSuccess ? LUB_OK : LUB_ERR_CUDA;
}
