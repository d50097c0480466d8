// Link-based lubrication of Ding and Aidun, as summarised in Sec. II
// (Eq. methods:dlub), for comparison with the contact-based corrections: for
// every D3Q19 link c_r that ends on a lattice site of particle i and stems
// from a site of particle j, or from a fluid site midway along 2 c_r from a
// site of j, a partial force
//   df = -3 qbar mu / (2 c_r^2 lambda*) c^ (c^ . (v_bi - v_bj)) (1/h*^2 - 1/c_r^2)
// on i where 0 < h* < c_r, and -df on j; h* is the distance along the link
// (or pair of links) between where it leaves j's surface and where it enters
// i's, v_b the rigid-body velocities there, lambda* the mean of the two
// surfaces' mean curvatures there.  Lattice sites are the integer points of
// the box coordinates (spacing 1); a site belongs to a particle when it lies
// in or on its spheroid, and a site in both is no stem; particle j is taken
// at its minimum image from i; a fluid site is in neither particle; the forces
// act at the two intersection points, torques about the centres; walls give
// nothing.
//
// One warp per pair; the lanes take the sites of the box where i's extent
// meets j's extent widened by 2 on every axis (a link, or two, moves a site by
// at most 2 per axis).  Sites are integer offsets from each centre's integer
// part, so membership is decided in FP32 from (float) offset - fraction
// (exact to about 1e-7) with a margin, and again in FP64 inside the margin:
// every decision is the FP64 one without an FP64 operation per test; the
// links that qualify are measured in FP64.
#include "lub_internal.cuh"

namespace {

constexpr float kMargin = 1e-4f;  // relative margin of the FP32 membership test

struct Body {
    double r[3], o[3];
    double ia2, ic2;    // 1 / R_perp^2, 1 / R_par^2
    double Rpar, Rperp;
    int nint[3];        // floor of the centre (the anchor of the site offsets)
    float f[3];         // centre - floor, in float
    float of[3], ia2f, dcf;  // axis, 1 / R_perp^2 and 1 / R_par^2 - 1 / R_perp^2 in float
};

__device__ __forceinline__ Body body_at(const PView &P, int k, const double r[3])
{
    Body b;
    const V3<double> o = quat_axis<double>(__ldg(P.qw + k), __ldg(P.qx + k), __ldg(P.qy + k), __ldg(P.qz + k));
    b.o[0] = o.x;
    b.o[1] = o.y;
    b.o[2] = o.z;
    b.Rpar = __ldg(P.rpar + k);
    b.Rperp = __ldg(P.rperp + k);
    b.ia2 = 1.0 / (b.Rperp * b.Rperp);
    b.ic2 = 1.0 / (b.Rpar * b.Rpar);
    for (int a = 0; a < 3; ++a) {
        b.r[a] = r[a];
        const double fl = floor(r[a]);
        b.nint[a] = (int)fl;
        b.f[a] = (float)(r[a] - fl);
        b.of[a] = (float)b.o[a];
    }
    b.ia2f = (float)b.ia2;
    b.dcf = (float)(b.ic2 - b.ia2);
    return b;
}

// (x - r)^T M^-1 (x - r) for the site x = floor(r) + m (m: integer offset
// from the body's anchor), in FP32 from (float) m - frac r, and in FP64
__device__ __forceinline__ float quad_f(const Body &b, const int m[3])
{
    float u[3];
    for (int a = 0; a < 3; ++a) u[a] = (float)m[a] - b.f[a];
    const float ou = b.of[0] * u[0] + b.of[1] * u[1] + b.of[2] * u[2];
    return (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) * b.ia2f + ou * ou * b.dcf;
}

__device__ __forceinline__ double quad_d(const Body &b, const int m[3])
{
    double u[3];
    for (int a = 0; a < 3; ++a) u[a] = (double)(b.nint[a] + m[a]) - b.r[a];
    const double ou = b.o[0] * u[0] + b.o[1] * u[1] + b.o[2] * u[2];
    return (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) * b.ia2 + ou * ou * (b.ic2 - b.ia2);
}

__device__ __forceinline__ bool inside(const Body &b, const int m[3])
{
    const float q = quad_f(b, m);
    if (q < 1.0f - kMargin) return true;
    if (q > 1.0f + kMargin) return false;
    return quad_d(b, m) <= 1.0;
}

// the line x0 + t e (|e| = 1) meets the surface at t_lo <= t_hi (false: misses)
__device__ __forceinline__ bool line_surface(const Body &b, const double x0[3], const double e[3], double &t_lo,
                                             double &t_hi)
{
    const double u[3] = {x0[0] - b.r[0], x0[1] - b.r[1], x0[2] - b.r[2]};
    const double ou = b.o[0] * u[0] + b.o[1] * u[1] + b.o[2] * u[2];
    const double oe = b.o[0] * e[0] + b.o[1] * e[1] + b.o[2] * e[2];
    const double dc = b.ic2 - b.ia2;
    const double A = b.ia2 + oe * oe * dc;  // |e| = 1
    const double B = 2.0 * ((u[0] * e[0] + u[1] * e[1] + u[2] * e[2]) * b.ia2 + ou * oe * dc);
    const double C = (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) * b.ia2 + ou * ou * dc - 1.0;
    const double disc = B * B - 4.0 * A * C;
    if (!(disc >= 0.0)) return false;
    const double sq = disc > 0.0 ? disc * rsqrt64(disc) : 0.0;
    const double i2a = rcp64(2.0 * A);
    t_lo = (-B - sq) * i2a;
    t_hi = (-B + sq) * i2a;
    return true;
}

// mean curvature (1/S1 + 1/S2) / 2 at the surface point y (radii of
// curvature of Eq. lub:curvature-radii, in the body coordinates of y)
__device__ __forceinline__ double mean_curvature(const Body &b, const double y[3])
{
    // with sin p ~ z_b / R_par and cos p ~ rho / R_perp (normalised),
    // s1^2 = R_perp^2 sin^2 p + R_par^2 cos^2 p; 1/S1 = R_par R_perp / s1^3,
    // 1/S2 = R_par / (R_perp s1)
    const double u[3] = {y[0] - b.r[0], y[1] - b.r[1], y[2] - b.r[2]};
    const double zb = b.o[0] * u[0] + b.o[1] * u[1] + b.o[2] * u[2];
    const double rho2 = fmax(u[0] * u[0] + u[1] * u[1] + u[2] * u[2] - zb * zb, 0.0);
    const double sp2 = zb * zb * b.ic2, cp2 = rho2 * b.ia2;
    const double s1sq = (b.Rperp * b.Rperp * sp2 + b.Rpar * b.Rpar * cp2) * rcp64(sp2 + cp2);
    const double is1 = rsqrt64(s1sq);
    return 0.5 * (b.Rpar * b.Rperp * is1 * is1 * is1 + b.Rpar * rcp64(b.Rperp) * is1);
}

// the 18 nonzero D3Q19 lattice vectors: (+-1,0,0), (0,+-1,0), (0,0,+-1), then
// the face diagonals (+-1,+-1,0), (+-1,0,+-1), (0,+-1,+-1)
__constant__ int8_t kD3Q19[18][3] = {{1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},  {0, 0, 1},  {0, 0, -1},
                                     {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},  {1, 0, 1},  {-1, 0, -1},
                                     {1, 0, -1}, {-1, 0, 1},  {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

__device__ __forceinline__ int d3q19(int r, int a) { return kD3Q19[r][a]; }

// a qualifying link: the site of i (offset from i's anchor), the direction,
// one link (1) or two through a fluid site (2)
struct LinkEntry {
    int m[3];
    int r, kind;
};
constexpr int kQueue = 64;  // entries per warp: at most 31 waiting plus 32 new

template <bool ENS>
__global__ void __launch_bounds__(128) k_links(PView P, const __grid_constant__ DView D0, Ens E,
                                               const int32_t *__restrict__ pi, const int32_t *__restrict__ pj,
                                               const int32_t *__restrict__ d_count, int32_t cap, double mu,
                                               double qbar, double *__restrict__ force, double *__restrict__ torque,
                                               int32_t *__restrict__ nlinks)
{
    pdl_wait();
    pdl_trigger();
    __shared__ LinkEntry link_queue[4 * kQueue];
    const int count = pair_count(d_count, cap);
    const size_t C = (size_t)cap;
    const int lane = threadIdx.x & 31;
    const int nwarp = (gridDim.x * blockDim.x) >> 5;
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < count; k += nwarp) {
        const int i = __ldg(pi + k), j = __ldg(pj + k);
        double F[3] = {0, 0, 0}, Ti[3] = {0, 0, 0}, Tj[3] = {0, 0, 0};
        int nl = 0;
        bool alien = false;
        const DView &D = pair_domain<ENS>(D0, E, i, j, &alien);
        const bool ok = !alien && i >= 0 && i < P.n && j >= 0 && j < P.n && i != j &&
                        shape_ok(__ldg(P.rpar + i), __ldg(P.rperp + i)) &&
                        shape_ok(__ldg(P.rpar + j), __ldg(P.rperp + j));
        if (ok) {
            const V3<double> ri = load_pos(P, i);
            const V3<double> d = min_image(D, sub(load_pos(P, j), ri));
            const double rir[3] = {ri.x, ri.y, ri.z}, rjr[3] = {ri.x + d.x, ri.y + d.y, ri.z + d.z};
            const Body bi = body_at(P, i, rir), bj = body_at(P, j, rjr);
            const double vi[3] = {__ldg(P.vx + i), __ldg(P.vy + i), __ldg(P.vz + i)};
            const double wi[3] = {__ldg(P.wx + i), __ldg(P.wy + i), __ldg(P.wz + i)};
            const double vj[3] = {__ldg(P.vx + j), __ldg(P.vy + j), __ldg(P.vz + j)};
            const double wj[3] = {__ldg(P.wx + j), __ldg(P.wy + j), __ldg(P.wz + j)};
            // sites of i's box within 2 (per axis) of j's box, as offsets m from
            // i's anchor (the same site is m + dij from j's)
            int lo[3], n[3], dij[3];
            int nsites = 1;
            for (int a = 0; a < 3; ++a) {
                const double wa = sqrt(bi.Rperp * bi.Rperp + (bi.Rpar * bi.Rpar - bi.Rperp * bi.Rperp) * bi.o[a] * bi.o[a]);
                const double wb = sqrt(bj.Rperp * bj.Rperp + (bj.Rpar * bj.Rpar - bj.Rperp * bj.Rperp) * bj.o[a] * bj.o[a]);
                const double l = fmax(ceil(rir[a] - wa), ceil(rjr[a] - wb - 2.0 - 1e-9));
                const double h = fmin(floor(rir[a] + wa), floor(rjr[a] + wb + 2.0 + 1e-9));
                lo[a] = (int)l - bi.nint[a];
                n[a] = h >= l ? (int)(h - l) + 1 : 0;
                nsites *= n[a];
                dij[a] = bi.nint[a] - bj.nint[a];
            }
            // Qualifying links go to a per-warp queue and are measured 32 at a
            // time, one per lane: they cluster on a few sites, and measuring
            // them where they are found would run the FP64 code with most
            // lanes idle.
            auto measure = [&](const LinkEntry &en) {
                const int c0 = d3q19(en.r, 0), c1 = d3q19(en.r, 1), c2 = d3q19(en.r, 2);
                const double cr = en.r < 6 ? 1.0 : 1.4142135623730951, icr = en.r < 6 ? 1.0 : 0.7071067811865476;
                const double e[3] = {c0 * icr, c1 * icr, c2 * icr};
                const double x0[3] = {(double)(bi.nint[0] + en.m[0] - en.kind * c0),
                                      (double)(bi.nint[1] + en.m[1] - en.kind * c1),
                                      (double)(bi.nint[2] + en.m[2] - en.kind * c2)};
                double tjl, tjh, til, tih;
                if (!line_surface(bj, x0, e, tjl, tjh) || !line_surface(bi, x0, e, til, tih)) return;
                const double hs = til - tjh;
                if (!(hs > 0.0 && hs < cr)) return;
                double pI[3], pJ[3], aI[3], aJ[3];
                for (int a = 0; a < 3; ++a) {
                    pI[a] = x0[a] + til * e[a];
                    pJ[a] = x0[a] + tjh * e[a];
                    aI[a] = pI[a] - rir[a];
                    aJ[a] = pJ[a] - rjr[a];
                }
                double dv[3];
                dv[0] = (vi[0] + wi[1] * aI[2] - wi[2] * aI[1]) - (vj[0] + wj[1] * aJ[2] - wj[2] * aJ[1]);
                dv[1] = (vi[1] + wi[2] * aI[0] - wi[0] * aI[2]) - (vj[1] + wj[2] * aJ[0] - wj[0] * aJ[2]);
                dv[2] = (vi[2] + wi[0] * aI[1] - wi[1] * aI[0]) - (vj[2] + wj[0] * aJ[1] - wj[1] * aJ[0]);
                const double lam = 0.5 * (mean_curvature(bi, pI) + mean_curvature(bj, pJ));
                const double icr2 = en.r < 6 ? 1.0 : 0.5;
                const double coef = -1.5 * qbar * mu * icr2 * rcp64(lam) * (rcp64(hs * hs) - icr2) *
                                    (e[0] * dv[0] + e[1] * dv[1] + e[2] * dv[2]);
                const double df[3] = {coef * e[0], coef * e[1], coef * e[2]};
                F[0] += df[0];
                F[1] += df[1];
                F[2] += df[2];
                Ti[0] += aI[1] * df[2] - aI[2] * df[1];
                Ti[1] += aI[2] * df[0] - aI[0] * df[2];
                Ti[2] += aI[0] * df[1] - aI[1] * df[0];
                Tj[0] -= aJ[1] * df[2] - aJ[2] * df[1];
                Tj[1] -= aJ[2] * df[0] - aJ[0] * df[2];
                Tj[2] -= aJ[0] * df[1] - aJ[1] * df[0];
                ++nl;
            };
            LinkEntry *queue = link_queue + (threadIdx.x >> 5) * kQueue;
            int queued = 0;  // warp-uniform
            auto drain = [&]() {  // measure the first 32 entries, move the rest to the front
                __syncwarp();
                const LinkEntry en = queue[lane];
                __syncwarp();
                if (lane < queued - 32) queue[lane] = queue[32 + lane];
                __syncwarp();
                measure(en);
                queued -= 32;
            };
            for (int q0 = 0; q0 < nsites; q0 += 32) {
                const int q = q0 + lane;
                int mi[3] = {0, 0, 0};
                bool site = false;
                if (q < nsites) {
                    mi[0] = lo[0] + q % n[0];
                    mi[1] = lo[1] + (q / n[0]) % n[1];
                    mi[2] = lo[2] + q / (n[0] * n[1]);
                    site = inside(bi, mi);
                }
                for (int r = 0; r < 18; ++r) {
                    int kind = 0;
                    if (site) {
                        const int c0 = d3q19(r, 0), c1 = d3q19(r, 1), c2 = d3q19(r, 2);
                        const int y1[3] = {mi[0] - c0, mi[1] - c1, mi[2] - c2};
                        const int y1b[3] = {y1[0] + dij[0], y1[1] + dij[1], y1[2] + dij[2]};
                        const bool y1i = inside(bi, y1), y1j = inside(bj, y1b);
                        if (y1j && !y1i) {
                            kind = 1;
                        } else if (!y1j && !y1i) {
                            const int y2[3] = {mi[0] - 2 * c0, mi[1] - 2 * c1, mi[2] - 2 * c2};
                            const int y2b[3] = {y2[0] + dij[0], y2[1] + dij[1], y2[2] + dij[2]};
                            if (inside(bj, y2b) && !inside(bi, y2)) kind = 2;
                        }
                    }
                    const unsigned hit = __ballot_sync(0xffffffffu, kind != 0);
                    if (!hit) continue;
                    if (kind) {
                        LinkEntry &en = queue[queued + __popc(hit & ((1u << lane) - 1u))];
                        en.m[0] = mi[0];
                        en.m[1] = mi[1];
                        en.m[2] = mi[2];
                        en.r = r;
                        en.kind = kind;
                    }
                    queued += __popc(hit);
                    if (queued >= 32) drain();
                }
            }
            // the rest: one per lane
            __syncwarp();
            if (lane < queued) measure(queue[lane]);
            __syncwarp();
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            for (int a = 0; a < 3; ++a) {
                F[a] += __shfl_xor_sync(0xffffffffu, F[a], o);
                Ti[a] += __shfl_xor_sync(0xffffffffu, Ti[a], o);
                Tj[a] += __shfl_xor_sync(0xffffffffu, Tj[a], o);
            }
            nl += __shfl_xor_sync(0xffffffffu, nl, o);
        }
        if (lane == 0) {
            for (int a = 0; a < 3; ++a) {
                force[a * C + k] = F[a];
                torque[a * C + k] = Ti[a];
                torque[(3 + a) * C + k] = Tj[a];
            }
            if (nlinks) nlinks[k] = nl;
        }
    }
}

}  // namespace

int launch_links(lub_ctx *ctx, const PView &P, const DView &D, const Ens &E, const int32_t *pi, const int32_t *pj,
                 const int32_t *d_count, int32_t cap, double mu, double qbar, double *force, double *torque,
                 int32_t *nlinks, cudaStream_t st)
{
    if (cap == 0) return LUB_OK;
    const int block = 128;
    const int64_t warps = cap;
    int64_t grid = (warps * 32 + block - 1) / block;
    if (grid > 64 * (int64_t)ctx->num_sms) grid = 64 * (int64_t)ctx->num_sms;
    cudaError_t e;
    if (E.nb)
        e = launch_pdl(k_links<true>, (int)grid, block, 0, st, P, D, E, pi, pj, d_count, cap, mu, qbar, force, torque,
                       nlinks);
    else
        e = launch_pdl(k_links<false>, (int)grid, block, 0, st, P, D, E, pi, pj, d_count, cap, mu, qbar, force,
                       torque, nlinks);
    return lub_check_cuda(ctx, e, "k_links launch");
}
