// K0: candidate pairs by a cell list with the pre-filters of Sec. III A.
//
//   1. cell of every particle (cell edge >= 2 Rmax + Delta_L in y and z, an
//      eighth of that in x; from the coordinates split into float-float) and
//      its slot in the cell (atomic), scan of the cell counts, copy of every
//      particle into cell order as two float4 records: position relative to
//      its cell centre with Rmax, and symmetry axis with e = R_par^2 -
//      R_perp^2;
//   2. sweep: one thread per slot, the slots in groups of 8 (a quarter warp);
//      the five rows of the half-shell stencil (y, z columns of cells: the
//      own column and the 4 forward neighbours) in turn; in each row the x
//      cells within reach of a group's particles form one run of slots,
//      staged 32 at a time in shared memory, and each lane tests its own
//      particle against every staged candidate; those that pass the
//      bounding-sphere test queue up for the full test, 32 at a time;
//      each unordered pair is visited once and stored for the smaller of its
//      two indices in one of that particle's KSLOT slots (atomic slot index); the
//      rare pairs beyond KSLOT go to an overflow list kept at the tail of the
//      caller's pair arrays; each thread also tests its particle's plane walls;
//   3. the test of the candidates the sweep's FP32 tests left inside their
//      margin, in float-float, then in FP64 inside the float-float margin
//      (k_pairs_undecided), stored as the sweep stores pairs;
//   4. one scan over [particle-pair counts | wall-pair counts] gives every
//      offset (wall pairs land after all particle pairs);
//   5. compaction: each particle sorts its partners (canonical (i, j) order)
//      and writes them, and its wall pairs, at its offsets.
// The pair arrays must hold the pairs plus the overflow entries; the count
// reports their sum when it does not fit (a capacity error, as for the pairs).
// The tests run in FP32 on cell-relative coordinates with a safety margin; a
// test inside the margin is decided again in FP64 from the original double
// positions, so every decision is the double-precision one.
//
// Ensemble mode: every suspension has its own cell grid (from its own box);
// the grids are laid out back to back in one global cell index space
// (cell_base of each suspension), so the same counting sort, sweep and scans
// run once over all suspensions, and no pair crosses two of them.
#include <string.h>

#include "ff.cuh"
#include "lub_internal.cuh"

namespace {

struct Grid {
    int nc[3];      // x: fine cells (xsub per coarse column); y, z: coarse
    float cs[3];
    double csd[3];
    double inv_cs[3];
    double invL[3];
    int64_t ncell;
    float cutoff;  // Delta_L
    float margin;  // absolute FP32 error allowance of the tests
    float rmax;    // bound of every particle's Rmax
    int xsub;      // fine x cells per cell edge of the interaction range
    float csff[3][2];  // cell edges as float-float (hi, lo)
    float inv_csf[3];
};

// Fine cells along x: a row of the stencil (one y, z column of cells) is cut
// into x cells a fraction of the interaction range wide, so each particle
// tests only the candidates in the x window its reach allows in that row
// (|dx| <= sqrt(reach^2 - dyz^2), dyz the distance to the row's y, z cells),
// a contiguous run of cells and so of slots, instead of three whole cells.
constexpr int kXSub = 8;

// partner slots per particle in the sweep; more go to the overflow list
constexpr int KSLOT = 16;

// one suspension's grid in ensemble mode
struct EnsGrid {
    Grid G;
    int32_t cell_base;
    int32_t pad;
};

// grid, domain and first global cell of suspension b (references: G0 and D0
// are __grid_constant__ kernel parameters, read in place)
template <bool ENS>
__device__ __forceinline__ const Grid &grid_ref(const Grid &G0, const EnsGrid *EG, int b)
{
    if (!ENS) return G0;
    return EG[b].G;
}
template <bool ENS>
__device__ __forceinline__ const DView &dom_ref(const DView &D0, const Ens &E, int b)
{
    if (!ENS) return D0;
    return E.dom[b].D;
}
template <bool ENS>
__device__ __forceinline__ int cell_base(const EnsGrid *EG, int b)
{
    return ENS ? __ldg(&EG[b].cell_base) : 0;
}

// Everything the pair build's kernels read and write, passed by value as one
// __grid_constant__ kernel parameter: the particles, the domain and grid (of
// the single suspension; the ensemble tables through E and EG), the
// workspace and the caller's outputs.
struct BuildView {
    PView P;
    DView D;
    Grid G;
    Ens E;
    const EnsGrid *EG;
    int32_t *flags, *cell_cnt, *cell_of, *slot, *sbat, *cnt, *totals, *slots;
    int2 *sc;  // per slot: its particle and its cell (x | y << 10 | z << 20)
    uint8_t *wbits;
    float4 *rel;  // each particle's position relative to its cell's centre (cells count -> cells fill)
    float4 *rec0, *rec1;
    unsigned long long *scan_state;
    int64_t z1, z2;  // state words of the cell scan and of the pair-count scan
    double cutoff_d;
    int32_t *pair_i, *pair_j, *d_count, *flags_out;
    float rmax_bound;
    int32_t cap;
    int64_t ncell_total;  // cells of all grids (the cell counts hold one more entry)
    int2 *und;            // candidates left to the FP64 test (in the cell index storage, free after the fill)
    int32_t und_cap;
};

// x < 0 in float-float
__device__ __forceinline__ bool ff_neg_(const ff x) { return x.hi < 0.f || (x.hi == 0.f && x.lo < 0.f); }

// Cell of one coordinate and the position relative to the cell's centre.  The
// double coordinate is split into float-float from its bits (46 significant
// bits: within 1.5e-11 at |x| = 1024, on the integer pipes; GB300 runs FP64
// at 1/74 of the FP32 rate) and the rest runs on the FP32 pipe: the wrap
// into [0, L) on a periodic axis, the cell floor(x / cs) in FP32, corrected
// by the exact sign of the float-float remainder x - c cs (so a cell holds
// its positions to within the split's error of its edges, far inside the
// 1e-9 allowance of the cell size), and the clamp to the edge cells of an
// open axis (a position outside the box then lies beyond its cell).  NaN
// goes to cell 0.
struct AxisCell {
    int c;
    float rel;
};

__device__ __forceinline__ AxisCell axis_cell(double x, const DView &D, const Grid &G, int a)
{
    ff p = ff_split_bits_nan(x);
    if (D.periodic[a]) {
        const ff L = {D.Lff[a][0], D.Lff[a][1]};
        const float k = floorf(p.hi * D.invLf[a]);
        if (k != 0.f && isfinite(k)) p = ff_sub(p, ff_mulf(L, k));
        if (ff_neg_(p))
            p = ff_add(p, L);
        else if (!ff_neg_(ff_sub(p, L)))
            p = ff_sub(p, L);
    }
    const int nc = G.nc[a];
    const ff cs = {G.csff[a][0], G.csff[a][1]};
    float f = floorf(p.hi * G.inv_csf[a]);
    if (!(f >= -1.f)) f = -1.f;  // also catches NaN
    if (f > (float)nc) f = (float)nc;
    int c = (int)f;
    ff r = ff_sub(p, ff_mulf(cs, (float)c));
    if (ff_neg_(r)) {
        --c;
        r = ff_add(r, cs);
    } else if (!ff_neg_(ff_sub(r, cs))) {
        ++c;
        r = ff_sub(r, cs);
    }
    if (c < 0 || c > nc - 1) {
        c = c < 0 ? 0 : nc - 1;
        r = ff_sub(p, ff_mulf(cs, (float)c));
    }
    const ff rel = ff_sub(r, ff_mulf(cs, 0.5f));
    return AxisCell{c, __fadd_rn(rel.hi, rel.lo)};
}

template <bool ENS>
__device__ __forceinline__ void cells_count(const BuildView &V)
{
    const PView &P = V.P;
    const Ens &E = V.E;
    int32_t *__restrict__ cell_cnt = V.cell_cnt;
    int32_t *__restrict__ cell_of = V.cell_of;
    int32_t *__restrict__ slot = V.slot;
    int32_t *__restrict__ flags = V.flags;
    unsigned long long *__restrict__ zero = V.scan_state;
    const int64_t nzero = V.z1;
    const float rmax_bound = V.rmax_bound;
    // state of the cell scan, which runs next
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nzero; k += (int64_t)gridDim.x * blockDim.x)
        zero[k] = 0ull;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        const int b = ENS ? batch_of(E, i) : 0;
        const Grid &G = grid_ref<ENS>(V.G, V.EG, b);
        const DView &D = dom_ref<ENS>(V.D, E, b);
        const int base = cell_base<ENS>(V.EG, b);
        const AxisCell ax = axis_cell(P.x[i], D, G, 0), ay = axis_cell(P.y[i], D, G, 1),
                       az = axis_cell(P.z[i], D, G, 2);
        const int c = base + (az.c * G.nc[1] + ay.c) * G.nc[0] + ax.c;
        cell_of[i] = c;
        V.rel[i] = make_float4(ax.rel, ay.rel, az.rel, 0.f);
        slot[i] = atomicAdd(cell_cnt + c, 1);
        const float rm = fmaxf(P.rpar[i], P.rperp[i]);
        if (!(rm <= rmax_bound)) atomicOr(flags, 1);  // bound violated or NaN shape
    }
}

template <bool ENS>
__global__ void k_cells_count(const __grid_constant__ BuildView V)
{
    pdl_wait();
    pdl_trigger();
    cells_count<ENS>(V);
}

template <bool ENS>
__device__ __forceinline__ void cells_fill(const BuildView &V)
{
    const PView &P = V.P;
    const Ens &E = V.E;
    const int32_t *__restrict__ cell_start = V.cell_cnt;
    const int32_t *__restrict__ cell_of = V.cell_of;
    const int32_t *__restrict__ slot = V.slot;
    int2 *__restrict__ sc = V.sc;
    float4 *__restrict__ rec0 = V.rec0;
    float4 *__restrict__ rec1 = V.rec1;
    int32_t *__restrict__ sbat = V.sbat;
    int32_t *__restrict__ cnt = V.cnt;
    unsigned long long *__restrict__ zero = V.scan_state;
    const int64_t nzero = V.z2;
    // the sweep's counts (2N + 1) and the state of the scan after it start at zero
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < 2 * (int64_t)P.n + 1; k += stride) cnt[k] = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nzero; k += stride) zero[k] = 0ull;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        const int b = ENS ? batch_of(E, i) : 0;
        const Grid &G = grid_ref<ENS>(V.G, V.EG, b);
        const int base = cell_base<ENS>(V.EG, b);
        const int cg = cell_of[i];
        const int s = cell_start[cg] + slot[i];
        const int c = cg - base;
        const int cx = c % G.nc[0], cy = (c / G.nc[0]) % G.nc[1], cz = c / (G.nc[0] * G.nc[1]);
        const float4 r = V.rel[i];
        const float rpar = P.rpar[i], rperp = P.rperp[i];
        const V3<float> o = quat_axis<float>(P.qw[i], P.qx[i], P.qy[i], P.qz[i]);
        sc[s] = make_int2(i, cx | (cy << 10) | (cz << 20));  // nc <= 1024 per axis
        if (ENS) sbat[s] = b;
        rec0[s] = make_float4(r.x, r.y, r.z, fmaxf(rpar, rperp));
        rec1[s] = make_float4(o.x, o.y, o.z, rpar * rpar - rperp * rperp);
    }
}

template <bool ENS>
__global__ void k_cells_fill(const __grid_constant__ BuildView V)
{
    pdl_wait();
    pdl_trigger();
    cells_fill<ENS>(V);
}

// exact (double) form of the three tests, as in the definition
__device__ __forceinline__ bool pair_test_fp64(const PView &P, const DView &D, int i, int j, double cutoff)
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

// decision of one candidate from the cell-order records in FP32 with a
// margin: kReject, kAccept, or kUndecided inside the margin (then the FP64
// test decides)
constexpr int kReject = 0, kAccept = 1, kUndecided = 2;

// support function sqrt(a2 + E (o.e)^2) of a spheroid along the unit e, in
// float-float (a2 = R_perp^2, E = R_par^2 - R_perp^2)
__device__ __forceinline__ ff ff_support(const ff o[3], float rpar, float rperp, const ff e[3])
{
    const ff a2 = two_prod(rperp, rperp), E = ff_sub(two_prod(rpar, rpar), a2);
    const ff c = ff_dot3(o, e);
    const ff s2 = ff_add(a2, ff_mul(E, ff_mul(c, c)));
    return ff_mul(s2, ff_rsqrt(s2));
}

// The three tests of pair_test_fp64 in float-float on the FP32 pipe, for the
// candidates the sweep's FP32 tests leave inside their margin: the positions
// split from their bits (within 2^-46 of each coordinate), the rest at about
// 44 bits, so each test value is within about 1e-12 of the pair's reach plus
// 1e-13 of the coordinates' magnitude of the exact one.  A test that clears
// its bound by more than 1e-10 of the reach plus 3e-14 of the coordinates'
// magnitude is decided here, as the FP64 test decides it; kUndecided
// otherwise (then the FP64 test: a dependent chain of FP64 operations, at
// 1/74 of the FP32 rate on this GPU, is the cost this saves).
__device__ __forceinline__ int pair_decide_ff(const PView &P, const DView &D, int i, int j, double cutoff)
{
    const double *pos[3] = {P.x, P.y, P.z};
    ff d[3];
    float mag = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const ff pi = ff_split_bits_nan(pos[a][i]), pj = ff_split_bits_nan(pos[a][j]);
        mag += fabsf(pi.hi) + fabsf(pj.hi);
        d[a] = ff_sub(pj, pi);
        if (D.periodic[a]) {
            const float k = rintf(d[a].hi * D.invLf[a]);
            if (k != 0.f) d[a] = ff_sub(d[a], ff_mulf(ff{D.Lff[a][0], D.Lff[a][1]}, k));
        }
    }
    const float rpi = P.rpar[i], rqi = P.rperp[i], rpj = P.rpar[j], rqj = P.rperp[j];
    const float rmi = fmaxf(rpi, rqi), rmj = fmaxf(rpj, rqj);
    const ff cut = ff_split_bits(cutoff);
    const ff r2 = ff_dot3(d, d);
    if (!(r2.hi > 0.f) || !isfinite(r2.hi) || !isfinite(mag)) return kUndecided;
    const ff ir = ff_rsqrt(r2);
    const ff r = ff_mul(r2, ir);
    const float margin = 1e-10f * (r.hi + rmi + rmj + cut.hi) + 3e-14f * mag;
    bool sure = true;
    // t > margin rejects; |t| <= margin leaves the pair undecided
    auto clears = [&](const ff t) {
        if (t.hi > margin) return false;
        if (t.hi >= -margin) sure = false;
        return true;
    };
    if (!clears(ff_sub(r, ff_add(ff_add(ff_make(rmi), ff_make(rmj)), cut)))) return kReject;
    // the support functions are even: along d / r as along -d / r
    ff e[3], oi[3], oj[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) e[a] = ff_mul(d[a], ir);
    ff_axis(P.qw[i], P.qx[i], P.qy[i], P.qz[i], oi);
    ff_axis(P.qw[j], P.qx[j], P.qy[j], P.qz[j], oj);
    if (!clears(ff_sub(ff_sub(r, ff_support(oi, rpi, rqi, e)), ff_add(ff_make(rmj), cut)))) return kReject;
    if (!clears(ff_sub(ff_sub(r, ff_support(oj, rpj, rqj, e)), ff_add(ff_make(rmi), cut)))) return kReject;
    return sure ? kAccept : kUndecided;
}

// the decision of a candidate that passed the bounding-sphere prefilter: aw
// and a1 the first particle's Rmax and record, bw and b1 the second's, d the
// vector between their centres; margin the absolute FP32 error allowance
__device__ __forceinline__ int pair_decide(float cutoff, float margin, float aw, const float4 a1, float bw,
                                           const float4 b1, float dx, float dy, float dz)
{
    const float r2 = dx * dx + dy * dy + dz * dz;
    const float lim = aw + bw + cutoff;
    bool sure = true;
    const float lo = lim - margin;
    if (r2 >= lo * lo) sure = false;
    // approximate square roots and reciprocal (relative error ~1e-7, far
    // inside the margin)
    const float r = sqrt_fast(r2);
    if (r > 0.f) {
        const float ir = rcp_fast(r);
        // half-widths along the line of centres: sigma^2 = R_perp^2 + e (o.e)^2,
        // with R_perp^2 = Rmax^2 - e for prolates (e > 0) and Rmax^2 for oblates
        const float ci = (a1.x * dx + a1.y * dy + a1.z * dz) * ir;
        const float cj = (b1.x * dx + b1.y * dy + b1.z * dz) * ir;
        const float api = a1.w > 0.f ? aw * aw - a1.w : aw * aw;
        const float apj = b1.w > 0.f ? bw * bw - b1.w : bw * bw;
        const float sgi = sqrt_fast(fmaxf(api + a1.w * ci * ci, 0.f));
        const float sgj = sqrt_fast(fmaxf(apj + b1.w * cj * cj, 0.f));
        const float t1 = r - sgi - (bw + cutoff);
        const float t2 = r - sgj - (aw + cutoff);
        if (t1 > margin || t2 > margin) return kReject;
        if (t1 >= -margin || t2 >= -margin) sure = false;
    } else {
        sure = false;
    }
    return sure ? kAccept : kUndecided;
}

// Half-shell stencil: the 14 coarse cells (the own cell and the 13 forward
// neighbours, offsets (dx, dy, dz) lexicographically above zero) as five rows
// of the y, z columns: row 0 = (dz, dy) = (0, 0), forward in x only; row 1 =
// (0, 1); rows 2..4 = (1, -1..1), the last four both ways in x.  Each
// unordered pair is seen from one side only: in another row from the particle
// whose forward rows hold the other; in row 0 from the one earlier in the
// column's slot order (the slots of a column run along x, cell by cell), the
// slots of the image at +L_x counting as later.  On a periodic axis the domain
// check (L > 2 range) leaves at most one image of a pair within range, so
// each pair passes exactly once.
constexpr int SWEEP_ROWS = 5;
constexpr int GL = 8;         // lanes (consecutive slots) per group
constexpr int NG = 32 / GL;   // groups per warp
constexpr int SC = 32;        // candidates a group stages per round
constexpr float kFar = 1e18f;  // x of an unused staging entry: fails every test
constexpr int kNone = 1 << 30;

template <bool B>
struct BoolTag {
    static constexpr bool value = B;
};

__device__ __forceinline__ void row_offsets(int row, int &dy, int &dz)
{
    dz = row >= 2 ? 1 : 0;
    dy = row == 0 ? 0 : (row == 1 ? 1 : row - 3);
}

// A particle's window in a row: the unwrapped fine x cells [lo, hi] within
// reach = Rmax_s + Rmax + Delta_L (+ margin) of it, given the distance from
// the particle to the row's y, z cells (lo > hi: none); cells below 0 and
// above nx - 1 belong to the images at -L_x and +L_x.  Row 0 starts at the
// particle's own cell.
__device__ __forceinline__ int2 row_window(const DView &D, const Grid &G, const float4 a0, int cx, int row)
{
    int dy, dz;
    row_offsets(row, dy, dz);
    const float oy = dy * G.cs[1], oz = dz * G.cs[2];
    const float reach = a0.w + G.rmax + G.cutoff + G.margin;
    const float hy = 0.5f * G.cs[1], hz = 0.5f * G.cs[2];
    const float ey = dy == 0 ? 0.f : fmaxf(fabsf(oy - a0.y) - hy, 0.f);
    const float ez = dz == 0 ? 0.f : fmaxf(fabsf(oz - a0.z) - hz, 0.f);
    const float r2yz = ey * ey + ez * ez;
    if (r2yz > reach * reach) return make_int2(kNone, -kNone);
    const float w = sqrt_fast(reach * reach - r2yz);  // the margin covers its rounding
    const float inv = G.inv_csf[0];
    const int nx = G.nc[0];
    int lo = row == 0 ? cx : cx + (int)floorf((a0.x - w) * inv + 0.5f);
    int hi = cx + (int)floorf((a0.x + w) * inv + 0.5f);
    if (row == 0 && hi < cx) hi = cx;
    if (!D.periodic[0]) {
        lo = min(max(lo, 0), nx - 1);
        hi = min(max(hi, 0), nx - 1);
    } else {
        lo = max(lo, -nx);
        hi = min(hi, 2 * nx - 1);
    }
    return make_int2(lo, hi);
}

// store of one accepted pair (i, j): in slot q of the smaller index (slot
// q of particle i at slots[q N + i]), or in the overflow list at the tail of
// the pair arrays
__device__ __forceinline__ void store_candidate(int i, int j, int N, int32_t *__restrict__ cnt,
                                                int32_t *__restrict__ slots, int32_t *__restrict__ ovf_n, int32_t cap,
                                                int32_t *__restrict__ pair_i, int32_t *__restrict__ pair_j)
{
    const int lo = min(i, j), hi = max(i, j);
    const int q = atomicAdd(cnt + lo, 1);
    if (q < KSLOT) {
        slots[(size_t)q * N + lo] = hi;
    } else {
        const int o = atomicAdd(ovf_n, 1);
        if (o < cap) {
            pair_i[cap - 1 - o] = lo;
            pair_j[cap - 1 - o] = hi;
        }
    }
}

// A candidate inside the FP32 margin, left to the tests of
// k_pairs_undecided: (smaller index, larger index) in the buffer und, and
// beyond its und_cap entries (at least one per particle: only inputs built to
// sit on the filters' edges fill it) tagged (smaller index | INT32_MIN) at
// the tail of the pair arrays, with the overflow list.
__device__ __forceinline__ void defer_candidate(int i, int j, const BuildView &V)
{
    const int lo = min(i, j), hi = max(i, j);
    const int u = atomicAdd(V.totals + 3, 1);
    if (u < V.und_cap) {
        V.und[u] = make_int2(lo, hi);
    } else {
        const int o = atomicAdd(V.totals + 2, 1);
        if (o < V.cap) {
            V.pair_i[V.cap - 1 - o] = (int32_t)((unsigned)lo | 0x80000000u);
            V.pair_j[V.cap - 1 - o] = hi;
        }
    }
}

// One warp's shared memory in the sweep (the block holds blockDim.x / 32 of
// them, dynamic): the groups' staging (rows padded by one entry, so that the
// groups' broadcast reads fall in different banks), each lane's particle,
// and the warp's queue of candidates for the full test (a ring of 64).
struct SweepWarp {
    float4 cand[NG * (SC + 1)];
    float4 own1[32];  // each lane's symmetry axis and e
    float4 qd[64];    // queued: d (x, y, z) and Rmax of the candidate
    float2 ownw[32];  // each lane's Rmax and its group's margin
    int cand_t[NG * (SC + 1)];
    int own_i[32];    // each lane's particle index
    int qt[64];       // queued: candidate slot t
    uint8_t qo[64];   // queued: lane of the particle
};
static_assert(sizeof(SweepWarp) % 16 == 0, "warp blocks stay 16-byte aligned");

// One thread per slot s (cell order); the thread also tests its particle's
// walls.  cnt: [0, N) pair counts per particle (of the smaller index of each
// pair), [N, 2N) wall-pair counts; slots [KSLOT][N] (slot-major, so that the
// compaction's reads of the first few slots of consecutive particles are
// coalesced and touch only the slots in use); wall bits per particle;
// overflow entry o at pair_i/pair_j[cap - 1 - o].
//
// Each quarter warp is a group of 8 consecutive slots.  The group's slots in
// one column (all of them, but for the few groups that straddle two columns,
// which take one pass per column) share their rows: per row, the union of
// their windows is one run of slots (up to three on a periodic x axis), which
// the group stages in shared memory 32 candidates at a time, x taken relative
// to the cell of the group's first slot; every lane then tests its own
// particle against the staged ones by broadcast reads (the bounding spheres,
// with the margin), a candidate outside its own window failing like any other
// distant one.  Staging a candidate once for 8 particles, instead of fetching
// it and its run bookkeeping per (particle, candidate), keeps the load/store
// pipe, the bound of a per-candidate share-out, mostly free.  (Groups of 16
// test more candidates outside their particles' windows; groups of 4 reading
// the runs straight from L1 spend more instructions per test.)  The few
// candidates that pass (about 12 per particle, a third of them pairs) queue up
// per warp, one per lane and round, and take the rest of the test and the
// store 32 at a time, every lane busy.
// The group-relative x of a particle or candidate within E of the group's
// cell carries an FP32 error of a few ulp(E); the group's margin adds
// E 2^-20 to the grid's, so that every decision inside it still goes to the
// FP64 test.
//
// Candidates inside the FP32 margin (about one in 10^4) are left to the
// next kernel (defer_candidate), which tests them in float-float and, inside
// that test's far smaller margin, in FP64: deciding them in the drain kept
// the FP64 test's registers in the sweep's loop, where they cost spills
// (the sweep ran 10 % faster without it).

template <bool ENS>
__device__ __forceinline__ void sweep_groups(const BuildView &V)
{
    const PView &P = V.P;
    const DView &D0 = V.D;
    const Grid &G0 = V.G;
    const Ens &E = V.E;
    const EnsGrid *__restrict__ EG = V.EG;
    const int32_t *__restrict__ cell_start = V.cell_cnt;
    const int2 *__restrict__ sc = V.sc;
    const float4 *__restrict__ rec0 = V.rec0;
    const float4 *__restrict__ rec1 = V.rec1;
    const int32_t *__restrict__ sbat = V.sbat;
    int32_t *__restrict__ cnt = V.cnt;
    int32_t *__restrict__ slots = V.slots;
    uint8_t *__restrict__ wbits = V.wbits;
    int32_t *__restrict__ ovf_n = V.totals + 2;
    const int32_t cap = V.cap;
    int32_t *__restrict__ pair_i = V.pair_i;
    int32_t *__restrict__ pair_j = V.pair_j;
    const double cutoff_d = V.cutoff_d;
    const int N = P.n;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5, g = lane / GL;
    // this warp's part of the block's dynamic shared memory
    extern __shared__ float4 sweep_smem[];
    SweepWarp &W = reinterpret_cast<SweepWarp *>(sweep_smem)[wq];
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int s0w = s - lane;
    const bool valid = s < N;
    // the full test and the store of queue entry e (the candidate's record
    // and index are fetched together, before the decision needs them)
    auto drain = [&](int e) {
        const float4 d = W.qd[e];
        const int t = W.qt[e];
        const int o = W.qo[e];
        const float4 b1 = rec1[t];
        const int jj = sc[t].x;
        const int ii = W.own_i[o];
        const float2 wm = W.ownw[o];
        const int bo = ENS ? sbat[s0w + o] : 0;
        const Grid &G = grid_ref<ENS>(G0, EG, bo);
        const int r = pair_decide(G.cutoff, wm.y, wm.x, W.own1[o], d.w, b1, d.x, d.y, d.z);
        // inside the margin the FP64 test decides, in the next kernel
        if (r == kAccept)
            store_candidate(ii, jj, N, cnt, slots, ovf_n, cap, pair_i, pair_j);
        else if (r == kUndecided)
            defer_candidate(ii, jj, V);
    };
    int b = 0, cc = 0, colkey = -1, pidx = -1;
    float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
    if (valid) {
        b = ENS ? sbat[s] : 0;
        const Grid &G = grid_ref<ENS>(G0, EG, b);
        const DView &D = dom_ref<ENS>(D0, E, b);
        a0 = rec0[s];
        a1 = rec1[s];
        const int2 own = sc[s];
        cc = own.y;
        const int cy = (cc >> 10) & 1023, cz = cc >> 20;
        colkey = cell_base<ENS>(EG, b) + (cz * G.nc[1] + cy) * G.nc[0];  // first cell of the column
        // plane walls: the gap dir (z - z_w) - sigma(e_z) in FP32 from the
        // records (z - z_w in float-float), decided in FP64 only within the
        // margin (the exact test costs some 60 FP64 operations)
        const int i = own.x;
        pidx = i;
        const float rm2 = a0.w * a0.w;
        const float sz = sqrt_fast(fmaxf((a1.w > 0.f ? rm2 - a1.w : rm2) + a1.w * a1.z * a1.z, 0.f));
        int wf = 0, bits = 0;
        // z - z_w in float-float from the bits of both (no FP64 pipe)
        const ff zf = ff_split_bits_nan(P.z[i]);
        for (int ww = 0; ww < D.n_walls; ++ww) {
            const ff dzw = ff_sub(zf, ff_split_bits_nan(D.wall_z[ww]));
            const float hw = (float)D.wall_dir[ww] * (dzw.hi + dzw.lo) - sz;
            bool in = hw < G.cutoff - G.margin;
            if (!in && hw <= G.cutoff + G.margin) {
                const Shape<double> si = load_shape<double>(P, i);
                in = (double)D.wall_dir[ww] * (P.z[i] - D.wall_z[ww]) - support(si, mk<double>(0.0, 0.0, 1.0)) <
                     cutoff_d;
            }
            if (in) {
                bits |= 1 << ww;
                ++wf;
            }
        }
        cnt[N + i] = wf;
        wbits[i] = (uint8_t)bits;
    }
    const int cx = cc & 1023;
    float4 *const cg = &W.cand[g * (SC + 1)];
    int *const ctg = &W.cand_t[g * (SC + 1)];
    int qn = 0, qh = 0;  // the warp's queue: qn entries from qh on (a ring of 64)
    bool done = !valid;
    // one pass per column among each group's slots (one for most groups)
    while (__any_sync(FULL, !done)) {
        const unsigned pend = __ballot_sync(FULL, !done);
        const unsigned gp = pend & (((1u << GL) - 1u) << (GL * g));
        const int leader = gp ? __ffs(gp) - 1 : lane;
        // every lane takes part in every shuffle (none inside a condition)
        const int lkey = __shfl_sync(FULL, colkey, leader);
        const bool act = gp != 0 && !done && colkey == lkey;
        // the group's column, suspension and reference cell: its leader's
        const int lcc = __shfl_sync(FULL, cc, leader);
        int lb = ENS ? __shfl_sync(FULL, b, leader) : 0;
        if (ENS && (lb < 0 || lb >= E.nb)) {  // range check: never taken by a correct sweep
            atomicOr(V.flags, 16);
            lb = 0;
        }
        const int lcx = lcc & 1023, lcy = (lcc >> 10) & 1023, lcz = (lcc >> 20) & 1023;
        const int s_lead = s0w + leader;
        const Grid &G = grid_ref<ENS>(G0, EG, lb);
        const DView &D = dom_ref<ENS>(D0, E, lb);
        const int nx = G.nc[0];
        const float cs0 = G.cs[0];
        int span = act ? cx - lcx : 0;
#pragma unroll
        for (int o = GL / 2; o; o >>= 1) span = max(span, __shfl_xor_sync(FULL, span, o));
        // every x of the pass lies within E of the group's cell
        const float Ex = (float)(span + 2) * cs0 + 2.f * G.rmax + G.cutoff + G.margin;
        const float marg = G.margin + Ex * 0x1p-20f;
        const float ax = a0.x + (float)(cx - lcx) * cs0;
        const float awc = a0.w + G.cutoff + marg;
        if (act) {
            W.own1[lane] = a1;
            W.ownw[lane] = make_float2(a0.w, marg);
            W.own_i[lane] = pidx;
        }
        for (int row = 0; row < SWEEP_ROWS; ++row) {
            int dy, dz;
            row_offsets(row, dy, dz);
            int yc = lcy + dy, zc = lcz + dz;
            bool exists = gp != 0;
            if (yc < 0 || yc >= G.nc[1]) {
                if (!D.periodic[1]) exists = false;
                yc += yc < 0 ? G.nc[1] : -G.nc[1];
            }
            if (zc < 0 || zc >= G.nc[2]) {
                if (!D.periodic[2]) exists = false;
                zc += zc < 0 ? G.nc[2] : -G.nc[2];
            }
            int2 w = make_int2(kNone, -kNone);
            if (act && exists) w = row_window(D, G, a0, cx, row);
#pragma unroll
            for (int o = GL / 2; o; o >>= 1) {
                w.x = min(w.x, __shfl_xor_sync(FULL, w.x, o));
                w.y = max(w.y, __shfl_xor_sync(FULL, w.y, o));
            }
            // the union's runs: run k holds the x cells of the image at (k - 1) L_x
            int beg[3] = {0, 0, 0}, num[3] = {0, 0, 0};
            const int rowbase = cell_base<ENS>(EG, lb) + (zc * G.nc[1] + yc) * nx;
            if (exists && (rowbase < 0 || (int64_t)rowbase + nx > V.ncell_total)) {  // range check, as above
                atomicOr(V.flags, 16);
                exists = false;
            }
            if (exists && w.x <= w.y) {
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const int lo = max(w.x, (k - 1) * nx), hi = min(w.y, k * nx - 1);
                    if (lo > hi) continue;
                    const int e = cell_start[rowbase + hi - (k - 1) * nx + 1];
                    const int st = (row == 0 && k == 1) ? s_lead + 1 : cell_start[rowbase + lo - (k - 1) * nx];
                    beg[k] = st;
                    num[k] = e > st ? e - st : 0;
                    if (st < 0 || (int64_t)st + num[k] > N) {  // range check, as above
                        atomicOr(V.flags, 16);
                        num[k] = 0;
                    }
                }
            }
            const int T = num[0] + num[1] + num[2];
            int Tw = T;
#pragma unroll
            for (int o = GL; o < 32; o <<= 1) Tw = max(Tw, __shfl_xor_sync(FULL, Tw, o));
            const float oy = dy * G.cs[1], oz = dz * G.cs[2];
            // ONE: every group of the warp has one run in this row, the image
            // at 0 (no periodic wrap): slot t = beg[1] + u, and in row 0 the
            // order test needs no stored slot
            auto rounds = [&](auto one) {
                constexpr bool ONE = decltype(one)::value;
                for (int c0 = 0; c0 < Tw; c0 += SC) {
                    __syncwarp();
#pragma unroll
                    for (int h = 0; h < SC / GL; ++h) {
                        const int q = (lane % GL) + GL * h, u = c0 + q;
                        float4 v = make_float4(kFar, 0.f, 0.f, 0.f);
                        int tk = 0;
                        if (u < T) {
                            int k = 1, t = beg[1] + u;
                            if (!ONE) {
                                k = u < num[0] ? 0 : (u < num[0] + num[1] ? 1 : 2);
                                t = k == 0 ? beg[0] + u : (k == 1 ? beg[1] + u - num[0] : beg[2] + u - num[0] - num[1]);
                            }
                            const float4 r0 = rec0[t];
                            const int dc = (sc[t].y & 1023) + (k - 1) * nx - lcx;
                            v = make_float4(r0.x + (float)dc * cs0, r0.y + oy, r0.z + oz, r0.w);
                            // row 0: the image at +L_x comes after every slot
                            tk = (row == 0 && k == 2) ? (int)((unsigned)t | 0x80000000u) : t;
                        }
                        cg[q] = v;
                        if (!ONE) ctg[q] = tk;
                    }
                    __syncwarp();
                    // the bounding spheres of the lane's particle and the staged
                    // candidates, in blocks of 8 up to the warp's longest run (the
                    // rest of a shorter group's staging holds far entries)
                    const int cn = min(SC, Tw - c0);
                    const int kb = beg[1] + c0 - s;  // ONE, row 0: candidate c comes after s iff c + kb > 0
                    unsigned m = 0;
                    if (act) {
                        for (int c8 = 0; c8 < cn; c8 += 8) {
                            unsigned mb = 0;
                            if (row == 0) {
#pragma unroll
                                for (int j = 0; j < 8; ++j) {
                                    const float4 q = cg[c8 + j];
                                    const float ex = q.x - ax, ey = q.y - a0.y, ez = q.z - a0.z;
                                    const float hi = awc + q.w;
                                    bool later;
                                    if (ONE) {
                                        later = c8 + j + kb > 0;
                                    } else {
                                        const int tk = ctg[c8 + j];
                                        later = tk < 0 || tk > s;
                                    }
                                    const bool p = ex * ex + ey * ey + ez * ez <= hi * hi && later;
                                    mb |= (unsigned)p << j;
                                }
                            } else {
#pragma unroll
                                for (int j = 0; j < 8; ++j) {
                                    const float4 q = cg[c8 + j];
                                    const float ex = q.x - ax, ey = q.y - a0.y, ez = q.z - a0.z;
                                    const float hi = awc + q.w;
                                    mb |= (unsigned)(ex * ex + ey * ey + ez * ez <= hi * hi) << j;
                                }
                            }
                            m |= mb << c8;
                        }
                    }
                    // the passes into the warp's queue, one per lane and round
                    while (__any_sync(FULL, m != 0)) {
                        const bool have = m != 0;
                        const unsigned bal = __ballot_sync(FULL, have);
                        if (have) {
                            const int c = __ffs(m) - 1;
                            m &= m - 1;
                            const int e = (qh + qn + __popc(bal & ((1u << lane) - 1u))) & 63;
                            const float4 q = cg[c];
                            W.qd[e] = make_float4(q.x - ax, q.y - a0.y, q.z - a0.z, q.w);
                            W.qt[e] = ONE ? beg[1] + c0 + c : (ctg[c] & 0x7fffffff);
                            W.qo[e] = (uint8_t)lane;
                        }
                        qn += __popc(bal);
                        if (qn >= 32) {
                            __syncwarp();
                            drain((qh + lane) & 63);
                            __syncwarp();
                            qh = (qh + 32) & 63;
                            qn -= 32;
                        }
                    }
                }
            };
            if (__all_sync(FULL, num[0] == 0 && num[2] == 0))
                rounds(BoolTag<true>{});
            else
                rounds(BoolTag<false>{});
        }
        done = done || act;
    }
    __syncwarp();
    if (lane < qn) drain((qh + lane) & 63);
}

// 64 registers: four blocks of 256 or eight of 128 per SM (the shared memory
// follows the block: blockDim.x / 32 SweepWarp)
template <bool ENS>
__global__ void __launch_bounds__(256, 4) k_pairs_sweep(const __grid_constant__ BuildView V)
{
    pdl_wait();
    pdl_trigger();
    sweep_groups<ENS>(V);
}

// The test of the candidates the sweep left inside its FP32 margin, in
// float-float (pair_decide_ff) and in FP64 where that leaves it open: those
// in und, then the tagged entries of the pair arrays' tail (entries untagged
// there are pairs beyond their particle's slots).  An accepted candidate
// takes the next slot of its smaller index as the sweep's pairs do; beyond
// the slots it stays where it is, as a pair the compaction collects (an und
// entry, or the tail entry untagged).  Every other entry becomes -1, which
// the compaction never matches.  Nothing is appended here, so the tail's
// length stays as the sweep left it.
template <bool ENS>
__global__ void __launch_bounds__(256) k_pairs_undecided(const __grid_constant__ BuildView V)
{
    pdl_wait();
    pdl_trigger();
    const int N = V.P.n;
    const int nu = min(V.totals[3], V.und_cap);
    const int nt = V.totals[3] > V.und_cap ? min(V.totals[2], V.cap) : 0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nu + nt; k += gridDim.x * blockDim.x) {
        int lo, hi;
        if (k < nu) {
            const int2 e = V.und[k];
            lo = e.x;
            hi = e.y;
        } else {
            const int32_t t = V.pair_i[V.cap - 1 - (k - nu)];
            if (t >= 0) continue;
            lo = t & 0x7fffffff;
            hi = V.pair_j[V.cap - 1 - (k - nu)];
        }
        const int b = ENS ? batch_of(V.E, lo) : 0;
        const DView &D = dom_ref<ENS>(V.D, V.E, b);
        const int dec = pair_decide_ff(V.P, D, lo, hi, V.cutoff_d);
        bool keep = false;  // accepted beyond the slots
        if (dec == kAccept || (dec == kUndecided && pair_test_fp64(V.P, D, lo, hi, V.cutoff_d))) {
            const int q = atomicAdd(V.cnt + lo, 1);
            if (q < KSLOT)
                V.slots[(size_t)q * N + lo] = hi;
            else
                keep = true;
        }
        if (k < nu)
            V.und[k].x = keep ? lo : -1;
        else
            V.pair_i[V.cap - 1 - (k - nu)] = keep ? lo : -1;
    }
}

// Canonical order: each particle's partners, sorted, then its wall pairs, at
// the offsets of the scan (off = the scanned counts, off[2N] = the total).
// The count is the total, or total + overflow entries when they do not fit.
__device__ __forceinline__ void pairs_compact(const BuildView &V)
{
    const int32_t n = V.P.n;
    const int32_t *__restrict__ off = V.cnt;
    const int32_t *__restrict__ slots = V.slots;
    const uint8_t *__restrict__ wbits = V.wbits;
    const int32_t *__restrict__ ovf_n = V.totals + 2;
    const int32_t cap = V.cap;
    int32_t *__restrict__ pair_i = V.pair_i;
    int32_t *__restrict__ pair_j = V.pair_j;
    int32_t *__restrict__ d_count = V.d_count;
    const int32_t *__restrict__ flags = V.flags;
    int32_t *__restrict__ flags_out = V.flags_out;
    const int total = off[2 * n];
    const int novf = *ovf_n;
    const int64_t need = (int64_t)total + novf;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *d_count = need > cap ? (int32_t)(need < (int64_t)INT32_MAX ? need : (int64_t)INT32_MAX) : total;
        if (flags_out) {
            *flags_out = *flags;  // this build's flags, for the host-count path
            if (*flags & 4) atomicOr(flags_out + 1, 4);  // a timed-out wait, for lub_sync_status
        }
    }
    if (need > cap) return;
    // each warp's pairs are one run of the output (its particles are
    // consecutive): staged in shared memory and stored as whole runs, unless
    // a particle of the warp has more pairs than slots (then every lane
    // stores its own)
    __shared__ int2 stage[8][32 * KSLOT];
    int2 *const sg = stage[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    // warp-uniform loop bound: every lane of a warp takes part in the
    // warp's reductions and its staged stores
    const int n_up = (n + 31) & ~31;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_up; i += gridDim.x * blockDim.x) {
        const bool live = i < n;
        const int b = live ? off[i] : 0, m = live ? off[i + 1] - b : 0;
        // the unrolled slot loads and pair stores stop at the warp's largest
        // count (mostly 4..8 of the 16), so the loads and stores beyond it
        // are skipped, not issued with every lane predicated off
        const int mw = __reduce_max_sync(0xffffffffu, m < KSLOT ? m : KSLOT);
        if (!__any_sync(0xffffffffu, m > KSLOT)) {
            // sort in registers: compare-exchange passes (m is small, mostly 0..4)
            int v[KSLOT];
#pragma unroll
            for (int q = 0; q < KSLOT; ++q) v[q] = INT32_MAX;
#pragma unroll
            for (int q = 0; q < KSLOT; ++q) {
                if (q >= mw) break;
                if (q < m) v[q] = slots[(size_t)q * n + i];
            }
            if (m > 1) {
#pragma unroll
                for (int q = 1; q < KSLOT; ++q) {
                    if (q >= m) break;
#pragma unroll
                    for (int r = q; r > 0; --r) {
                        const int x = v[r - 1], y = v[r];
                        v[r - 1] = min(x, y);
                        v[r] = max(x, y);
                    }
                }
            }
            // lane 0 is live whenever any lane is (i grows with the lane)
            const int b0 = __shfl_sync(0xffffffffu, b, 0);
            const int tw = (int)__reduce_max_sync(0xffffffffu, (unsigned)(live ? b + m - b0 : 0));
#pragma unroll
            for (int q = 0; q < KSLOT; ++q) {
                if (q >= mw) break;
                if (q < m) sg[b - b0 + q] = make_int2(i, v[q]);
            }
            __syncwarp();
            for (int t = lane; t < tw; t += 32) {
                const int2 e = sg[t];
                pair_i[b0 + t] = e.x;
                pair_j[b0 + t] = e.y;
            }
            __syncwarp();
        } else if (live) {
            // the slots, then (beyond them) this particle's entries at the
            // tail and among the candidates the FP64 test accepted, then
            // sort in place
            const int ms = m < KSLOT ? m : KSLOT;
            for (int q = 0; q < ms; ++q) {
                pair_i[b + q] = i;
                pair_j[b + q] = slots[(size_t)q * n + i];
            }
            int c = ms;
            for (int o = 0; o < novf && c < m; ++o)
                if (pair_i[cap - 1 - o] == i) {
                    pair_j[b + c] = pair_j[cap - 1 - o];
                    pair_i[b + c] = i;
                    ++c;
                }
            const int nu = min(V.totals[3], V.und_cap);
            for (int u = 0; u < nu && c < m; ++u)
                if (V.und[u].x == i) {
                    pair_j[b + c] = V.und[u].y;
                    pair_i[b + c] = i;
                    ++c;
                }
            for (int a = b + 1; a < b + m; ++a) {
                const int x = pair_j[a];
                int q = a - 1;
                while (q >= b && pair_j[q] > x) {
                    pair_j[q + 1] = pair_j[q];
                    --q;
                }
                pair_j[q + 1] = x;
            }
        }
        if (!live) continue;
        const int wb = off[n + i];
        const int bits = wbits[i];
        int c = 0;
        for (int w = 0; w < 2; ++w)
            if (bits & (1 << w)) {
                pair_i[wb + c] = i;
                pair_j[wb + c] = -1 - w;
                ++c;
            }
    }
}

__global__ void __launch_bounds__(256) k_pairs_compact(const __grid_constant__ BuildView V)
{
    pdl_wait();
    pdl_trigger();
    pairs_compact(V);
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

Grid make_grid(const DView &D, const lub_params &prm, float rmax, int64_t n, int64_t max_cells)
{
    // cells at least (1 + 1e-9) times the interaction range, so a particle
    // assigned to a cell by rounding at its border still finds every partner
    // in the 27 neighbour cells
    const double range = (2.0 * (double)rmax + prm.list_cutoff) * (1.0 + 1e-9);
    Grid G;
    memset(&G, 0, sizeof(G));  // padding too: grid tables are compared bytewise
    for (int a = 0; a < 3; ++a) {
        int nc = (int)floor(D.L[a] / range);
        if (nc < 1) nc = 1;
        if (nc > 1024) nc = 1024;
        G.nc[a] = nc;
    }
    // keep the grid at most a few cells per particle (huge, sparse boxes) and
    // within max_cells
    int64_t limit = 8 * n + 4096;
    if (limit > max_cells) limit = max_cells;
    for (int pass = 0; pass < 8; ++pass) {
        const int64_t ncell = (int64_t)G.nc[0] * G.nc[1] * G.nc[2];
        if (ncell <= limit) break;
        const double f = cbrt((double)ncell / (double)limit) * (1.0 + 0.02 * pass);
        for (int a = 0; a < 3; ++a) {
            int nc = (int)floor(G.nc[a] / f);
            G.nc[a] = nc < 1 ? 1 : nc;
        }
    }
    // fine x cells within the same limits (at most 1024 per axis: the packed
    // cell coordinates of the sweep hold 10 bits each)
    const int64_t ncoarse = (int64_t)G.nc[0] * G.nc[1] * G.nc[2];
    int xs = kXSub;
    while (xs > 1 && ((int64_t)G.nc[0] * xs > 1024 || ncoarse * xs > limit)) --xs;
    G.xsub = xs;
    G.nc[0] *= xs;
    for (int a = 0; a < 3; ++a) {
        G.csd[a] = D.L[a] / G.nc[a];
        G.cs[a] = (float)G.csd[a];
        G.inv_cs[a] = G.nc[a] / D.L[a];
        G.invL[a] = 1.0 / D.L[a];
        G.csff[a][0] = (float)G.csd[a];
        G.csff[a][1] = (float)(G.csd[a] - (double)G.csff[a][0]);
        G.inv_csf[a] = (float)G.inv_cs[a];
    }
    G.ncell = (int64_t)G.nc[0] * G.nc[1] * G.nc[2];
    G.cutoff = (float)prm.list_cutoff;
    // FP32 error of cell-relative coordinates and of the test values, with headroom
    G.margin = (float)(1e-5 * (range + 1.0));
    G.rmax = rmax;
    return G;
}

struct Layout {
    int32_t *flags, *cell_cnt, *cell_of, *slot, *sorted, *cellc, *sbat, *cnt, *totals, *slots;
    uint8_t *wbits;
    float4 *rel, *rec0, *rec1;
    void *tmp;
    size_t tmp_bytes, total;
};

Layout layout(void *base, int64_t N, int64_t ncell, bool ens = false)
{
    const size_t b_cell = align256((ncell + 1) * 4), b_n = align256((N + 1) * 4), b_n2 = align256((2 * N + 1) * 4);
    const size_t b_slots = align256((size_t)N * KSLOT * 4), b_bits = align256((size_t)N + 1);
    const size_t b_rec = align256(N * 16),
                 b_tmp = align256(scan_tmp_bytes(ncell + 1 > 2 * N + 1 ? ncell + 1 : 2 * N + 1));
    Layout L;
    char *s = (char *)base;
    L.flags = (int32_t *)s;
    s += 256;
    L.totals = (int32_t *)s;  // [0] all pairs, [1] cells, [2] tail entries, [3] candidates left to FP64
    s += 256;
    L.cell_cnt = (int32_t *)s;
    s += b_cell;
    L.cell_of = (int32_t *)s;
    s += b_n;
    L.slot = (int32_t *)s;
    s += b_n;
    L.sorted = (int32_t *)s;  // with the cellc storage after it: the int2 per slot (particle, cell)
    s += b_n;
    L.cellc = (int32_t *)s;
    s += b_n;
    L.sbat = (int32_t *)s;  // suspension of each slot (ensemble mode only)
    if (ens) s += b_n;
    L.cnt = (int32_t *)s;
    s += b_n2;
    L.slots = (int32_t *)s;
    L.rel = (float4 *)s;  // shares the slots' storage: read by the cells fill, before the sweep fills the slots
    s += b_slots;
    L.wbits = (uint8_t *)s;
    s += b_bits;
    L.rec0 = (float4 *)s;
    s += b_rec;
    L.rec1 = (float4 *)s;
    s += b_rec;
    L.tmp = s;
    L.tmp_bytes = b_tmp;
    s += b_tmp;
    L.total = (size_t)(s - (char *)base);
    return L;
}

// the build on a workspace; flags live in the workspace.  G.ncell is the
// total number of cells (all suspensions in ensemble mode).
template <bool ENS>
int build_core(lub_ctx *ctx, int num_sms, void *scratch, const Grid &G, const PView &P, const DView &D, const Ens &E,
               const EnsGrid *EG, const lub_params &prm, float rmax, int32_t *pi, int32_t *pj, int32_t cap,
               int32_t *d_count, cudaStream_t st, int32_t *flags_out = nullptr)
{
    const int64_t N = P.n;
    Layout L = layout(scratch, N, G.ncell, ENS);
    // the scratch keeps earlier contents: clear what must start at zero, the
    // flags, totals and cell counts in one (they are contiguous); the kernels
    // clear the sweep's counts and the scans' states for the launches after them
    int rc = zero_async(ctx, num_sms, L.flags, 512 + (G.ncell + 1) * 4, st);
    if (rc) return rc;
    if (N == 0) {
        rc = lub_check_cuda(ctx, cudaMemsetAsync(d_count, 0, 4, st), "memset count");
        if (!rc && flags_out) rc = lub_check_cuda(ctx, cudaMemsetAsync(flags_out, 0, 4, st), "memset flags");
        return rc;
    }
    BuildView V;
    memset(&V, 0, sizeof(V));
    V.P = P;
    V.D = D;
    V.G = G;
    V.E = E;
    V.EG = EG;
    V.flags = L.flags;
    V.cell_cnt = L.cell_cnt;
    V.cell_of = L.cell_of;
    V.slot = L.slot;
    V.sc = reinterpret_cast<int2 *>(L.sorted);  // the sorted and cellc storage, contiguous
    V.sbat = L.sbat;
    V.cnt = L.cnt;
    V.totals = L.totals;
    V.slots = L.slots;
    V.wbits = L.wbits;
    V.rel = L.rel;
    V.rec0 = L.rec0;
    V.rec1 = L.rec1;
    V.scan_state = (unsigned long long *)L.tmp;
    V.z1 = scan_state_words(G.ncell + 1);
    V.z2 = scan_state_words(2 * N + 1);
    V.cutoff_d = prm.list_cutoff;
    V.pair_i = pi;
    V.pair_j = pj;
    V.d_count = d_count;
    V.flags_out = flags_out;
    V.rmax_bound = rmax;
    V.cap = cap;
    V.ncell_total = G.ncell;
    // the buffer of candidates left to the FP64 test: the cell index and
    // slot arrays, contiguous and free once the cells are filled
    V.und = reinterpret_cast<int2 *>(L.cell_of);
    const int64_t und_cap = (int64_t)(L.slot - L.cell_of + (N + 1)) / 2;
    V.und_cap = (int32_t)(und_cap < INT32_MAX ? und_cap : INT32_MAX);
    cudaError_t e;
    const int block = 256;
    const int gn = grid_for(N, block, num_sms, 32);  // one particle per thread up to 1.2M
    e = launch_pdl(k_cells_count<ENS>, gn, block, 0, st, V);
    if ((rc = lub_check_cuda(ctx, e, "cells count launch"))) return rc;
    if ((rc = scan_exclusive(ctx, L.cell_cnt, G.ncell + 1, L.totals + 1, L.tmp, L.tmp_bytes, st, L.flags, true)))
        return rc;
    e = launch_pdl(k_cells_fill<ENS>, gn, block, 0, st, V);
    if ((rc = lub_check_cuda(ctx, e, "cells fill launch"))) return rc;
    // one slot per thread (no grid-stride loop)
    Shape2 sw = tuned_shape(ctx, LUB_TUNE_SWEEP, N);
    sw.grid = (int)((N + sw.block - 1) / sw.block);
    lub_trace_mark(ctx, LUB_TRACE_SWEEP, st);
    e = launch_pdl(k_pairs_sweep<ENS>, sw.grid, sw.block, (size_t)(sw.block / 32) * sizeof(SweepWarp), st, V);
    lub_trace_mark(ctx, LUB_TRACE_SWEEP, st);
    if ((rc = lub_check_cuda(ctx, e, "sweep launch"))) return rc;
    e = launch_pdl(k_pairs_undecided<ENS>, num_sms, 256, 0, st, V);
    if ((rc = lub_check_cuda(ctx, e, "undecided pairs launch"))) return rc;
    // one scan over [particle pairs | wall pairs] (+1 entry: the end of the last run)
    if ((rc = scan_exclusive(ctx, L.cnt, 2 * N + 1, L.totals + 0, L.tmp, L.tmp_bytes, st, L.flags, true))) return rc;
    e = launch_pdl(k_pairs_compact, grid_for(N, 256, num_sms, 32), 256, 0, st, V);
    return lub_check_cuda(ctx, e, "pairs compact launch");
}

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
    const Grid G = make_grid(D, prm, rmax, P.n, (int64_t)1 << 40);
    const size_t need = layout(nullptr, P.n, G.ncell).total;
    int rc = lub_ensure_scratch(ctx, need);
    if (rc) return rc;
    const Ens E = {nullptr, 0};
    // the build leaves its flags in ctx->d_flags for the host-count path
    return build_core<false>(ctx, ctx->num_sms, ctx->scratch, G, P, D, E, nullptr, prm, rmax, pi, pj, cap, d_count,
                             st, ctx->d_flags);
}

// ---------------------------------------------------------------------------
// The same build on scratch the caller provides (used by the entry point that
// allocates nothing); max_cells bounds the cell grid to fit that scratch.
// ---------------------------------------------------------------------------
size_t pairs_scratch_bytes(int64_t n, int64_t max_cells)
{
    return layout(nullptr, n, max_cells).total;
}

int pairs_build_on_scratch(int num_sms, void *scratch, size_t scratch_bytes, int64_t max_cells, const PView &P,
                           const DView &D, const lub_params &prm, float rmax, int32_t *pi, int32_t *pj, int32_t cap,
                           int32_t *d_count, cudaStream_t st)
{
    const Grid G = make_grid(D, prm, rmax, P.n, max_cells);
    if (G.ncell > max_cells) return LUB_ERR_ARG;
    if (layout(nullptr, P.n, G.ncell).total > scratch_bytes) return LUB_ERR_ARG;
    const Ens E = {nullptr, 0};
    return build_core<false>(nullptr, num_sms, scratch, G, P, D, E, nullptr, prm, rmax, pi, pj, cap, d_count, st);
}

// ---------------------------------------------------------------------------
// ensemble form: one grid per suspension, back to back in the cell index space
// ---------------------------------------------------------------------------
int launch_pairs_build_ens(lub_ctx *ctx, const PView &P, const Ens &E, const DView *hdom, const int32_t *hoff,
                           const lub_params &prm, float rmax, int32_t *pi, int32_t *pj, int32_t cap, int32_t *d_count,
                           cudaStream_t st)
{
    std::vector<EnsGrid> tab((size_t)E.nb);
    int64_t total = 0;
    for (int b = 0; b < E.nb; ++b) {
        memset(&tab[b], 0, sizeof(EnsGrid));
        tab[b].G = make_grid(hdom[b], prm, rmax, (int64_t)hoff[b + 1] - hoff[b], (int64_t)1 << 40);
        tab[b].cell_base = (int32_t)total;
        total += tab[b].G.ncell;
        if (total > ((int64_t)1 << 30))
            return lub_set_error(ctx, LUB_ERR_ARG, "the ensemble's cell grids exceed 2^30 cells");
    }
    const void *dev = nullptr;
    int rc = lub_upload_table(ctx, 1, tab.data(), tab.size() * sizeof(EnsGrid), st, &dev);
    if (rc) return rc;
    Grid G;
    memset(&G, 0, sizeof(G));
    G.ncell = total;
    DView D;
    memset(&D, 0, sizeof(D));
    const size_t need = layout(nullptr, P.n, total, true).total;
    if ((rc = lub_ensure_scratch(ctx, need))) return rc;
    return build_core<true>(ctx, ctx->num_sms, ctx->scratch, G, P, D, E, (const EnsGrid *)dev, prm, rmax, pi, pj, cap,
                            d_count, st, ctx->d_flags);
}
