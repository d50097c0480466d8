// K1: closest points and signed gap of every candidate pair (Sec. III A).
//
// The common-normal points of two convex bodies are the stationary point of
//   g(n) = n.d - sigma_i(n) - sigma_j(n),  |n| = 1,  d = r_j - r_i,
// (max g = minimum surface distance; minus the penetration depth on overlap),
// with y*_i = r_i + M_i n / sigma_i and y*_j = r_j - M_j n / sigma_j.  The
// paper's tangent-sphere iteration converges linearly (about 40 iterations
// from the line of centres); here Newton's method runs on the sphere in a
// tangent chart (t1, t2) at n, using the closed-form tangent Hessian of the
// spheroid support function
//   sigma = sqrt(a2 + e c^2),  c = o.n,  u_a = o.t_a,
//   grad_t sigma = e c u / sigma,
//   Hess_t sigma = (a2 / sigma) (I + (e / sigma^2) u u^T),
// so that the chart Hessian of g is -(Hess_t sigma_i + Hess_t sigma_j) - g I.
//
// LUB_MIXED, one thread per pair:
//   * Newton iterations in FP32 from the line of centres (or the normal
//     passed in, for a warm start);
//   * then, for every pair, the gap and one more Newton step with the
//     gradient in float-float arithmetic (about 48 bits, on the FP32 pipe).
//     h is stationary in n, so the FP32 normal costs the gap only O(dn^2),
//     while n.d - sigma_i - sigma_j cancels far beyond FP32 for small gaps.
//     The normal itself must be better than FP32 at every gap: the normal
//     relative surface velocity n.(V_j - V_i) is a difference of terms of the
//     size of the velocities, so an error dn of the normal is an error of
//     dn |V_j - V_i| in it, and where it nearly cancels a 1e-5 force bound
//     relative to it needs dn near 1e-9 rad; the float-float step lands
//     near 1e-13;
//   * pairs whose FP32 Newton did not converge are appended to a compacted
//     work list (one atomic per warp) and solved again in FP64 by a second
//     kernel, so only full warps of such pairs use the slow FP64 pipe.
// LUB_FP64: the whole solve and gap in double.
#include "ff.cuh"
#include "lub_mlp.cuh"
#include "mlp_infer.cuh"
#include "pair_force.cuh"

namespace {

struct NewtonOut {
    int iters;
    bool converged;
};

// FP64 stopping rule: Newton converges quadratically, so after a step of
// length s the remaining error is about K s^2 (K of order one to ten for
// these shapes); stopping once a step is below 1e-7 rad leaves an error of
// order 1e-14 rad in n, so the contact points sit within 1e-12 R of the
// converged ones (the gap, stationary in n, within R 1e-26), without
// spending an iteration to confirm it
constexpr double kTolFp64 = 1e-7;

template <typename T>
__device__ __forceinline__ V3<T> perp_unit(const V3<T> &n)
{
    V3<T> e = (fabs((double)n.x) < 0.6) ? mk<T>(1, 0, 0) : mk<T>(0, 1, 0);
    return normalized(axpy(-dot(e, n), n, e));
}

// Newton ascent of g on the unit sphere from n (in/out), in precision T.
// Step-size convergence: |s| < tol (radians), after which the last step is
// applied.  Steps are clamped to 0.5 rad; a step that lowers g by more than
// the rounding noise is halved (at most 12 times per solve).
template <typename T>
__device__ NewtonOut newton_sphere(const Shape<T> &si, const Shape<T> &sj, const V3<T> &d, V3<T> &n, int maxit,
                                   T tol, T noise)
{
    n = normalized(n);  // g below assumes |n| = 1: a start off by 1e-7 would corrupt the first g
    V3<T> t1 = perp_unit(n);
    V3<T> n_acc = n, t1_acc = t1, t2_acc = cross(n, t1);
    T g_acc = -T(1e30), s1_acc = 0, s2_acc = 0;
    int halvings = 0;
    NewtonOut out{0, false};
    for (int it = 0; it < maxit; ++it) {
        V3<T> t2 = cross(n, t1);
        T ci = dot(si.o, n), u1i = dot(si.o, t1), u2i = dot(si.o, t2);
        T cj = dot(sj.o, n), u1j = dot(sj.o, t1), u2j = dot(sj.o, t2);
        T qi = si.a2 + si.e * ci * ci, qj = sj.a2 + sj.e * cj * cj;
        T ri = rsqrt_t(qi), rj = rsqrt_t(qj);
        T g = dot(n, d) - qi * ri - qj * rj;
        out.iters = it + 1;
        if (g < g_acc - noise && halvings < 12) {
            // the last step lowered g: retry from the accepted point with half the step
            ++halvings;
            s1_acc *= T(0.5);
            s2_acc *= T(0.5);
            n = normalized(axpy(s1_acc, t1_acc, axpy(s2_acc, t2_acc, n_acc)));
            t1 = normalized(axpy(-dot(t1_acc, n), n, t1_acc));
            continue;
        }
        n_acc = n;
        t1_acc = t1;
        t2_acc = t2;
        g_acc = g;
        T ki = si.e * ci * ri, kj = sj.e * cj * rj;
        T g1 = dot(t1, d) - ki * u1i - kj * u1j;
        T g2 = dot(t2, d) - ki * u2i - kj * u2j;
        // P = -Hess_t g = A_i (I + E_i u_i u_i^T) + A_j (I + E_j u_j u_j^T) + g I
        T Ai = si.a2 * ri, Aj = sj.a2 * rj;
        T Ei = si.e * ri * ri, Ej = sj.e * rj * rj;
        T P11 = Ai * (T(1) + Ei * u1i * u1i) + Aj * (T(1) + Ej * u1j * u1j) + g;
        T P22 = Ai * (T(1) + Ei * u2i * u2i) + Aj * (T(1) + Ej * u2j * u2j) + g;
        T P12 = Ai * Ei * u1i * u2i + Aj * Ej * u1j * u2j;
        T det = P11 * P22 - P12 * P12;
        T s1, s2;
        if (P11 > T(0) && det > T(0)) {
            T idet = rcp_t(det);
            s1 = (P22 * g1 - P12 * g2) * idet;
            s2 = (P11 * g2 - P12 * g1) * idet;
        } else {
            T sc = rcp_t(fabs(P11) + fabs(P22) + fabs(P12) + Ai + Aj);
            s1 = g1 * sc;
            s2 = g2 * sc;
        }
        T sn2 = s1 * s1 + s2 * s2;
        if (sn2 > T(0.25)) {
            T f = T(0.5) * rsqrt_t(sn2);
            s1 *= f;
            s2 *= f;
        }
        s1_acc = s1;
        s2_acc = s2;
        n = normalized(axpy(s1, t1, axpy(s2, t2, n)));
        t1 = normalized(axpy(-dot(t1, n), n, t1));
        if (sn2 < tol * tol) {
            out.converged = true;
            break;
        }
    }
    return out;
}

// Minimum-image separation r_j - r_i in float-float from the particles'
// records (rec_ld 0 and 1: the float-float centres); the image shift is
// taken from the float part (listed pairs are far from the ambiguous half
// box).  The centres carry 46 bits (split from their bits): an absolute
// error below 2^-46 |r| each (1.5e-11 at |r| = 1000), against the FP64
// subtraction and splitting it replaces (some 24 FP64 operations per pair,
// at 1/74 of the FP32 rate).
__device__ __forceinline__ void ff_separation(const float4 &ri0, const float4 &ri1, const float4 &rj0,
                                              const float4 &rj1, const DView &D, ff d[3])
{
    const ff pi[3] = {{ri0.x, ri0.y}, {ri0.z, ri0.w}, {ri1.x, ri1.y}};
    const ff pj[3] = {{rj0.x, rj0.y}, {rj0.z, rj0.w}, {rj1.x, rj1.y}};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        ff da = ff_sub(pj[a], pi[a]);
        if (D.periodic[a]) {
            const float k = rintf(da.hi * D.invLf[a]);
            if (k != 0.f) da = ff_sub(da, ff{k * D.Lff[a][0], k * D.Lff[a][1]});
        }
        d[a] = da;
    }
}

__device__ __forceinline__ bool pair_bad(const PView &P, const DView &D, int i, int j)
{
    bool bad = (i < 0 || i >= P.n || j >= P.n || j < -D.n_walls || j == i);
    if (!bad) bad = !shape_ok(__ldg(P.rpar + i), __ldg(P.rperp + i));
    if (!bad && j >= 0) bad = !shape_ok(__ldg(P.rpar + j), __ldg(P.rperp + j));
    return bad;
}

__device__ __forceinline__ double wall_gap(const PView &P, const DView &D, int i, int w, V3<double> &n)
{
    // plane wall w: n = -dir e_z, h = dir (z_i - wall_z) - sigma_i(e_z)
    const double dir = (double)D.wall_dir[w];
    const Shape<double> si = load_shape<double>(P, i);
    n = mk<double>(0.0, 0.0, -dir);
    return dir * (__ldg(P.z + i) - D.wall_z[w]) - support(si, mk<double>(0.0, 0.0, 1.0));
}

// ---------------------------------------------------------------------------
// per-pair solves, shared by the separate kernels and the fused pass
// ---------------------------------------------------------------------------
constexpr int kNoEntry = 0x7fffffff;

// The FP32 stage's finish for a particle pair, in float-float on the FP32
// pipe (GB300 runs FP64 at 1/74 of the FP32 rate): the gap at the FP32 Newton
// normal n and one Newton step from n with the gradient in float-float.  n
// is an exact float vector with |n|^2 = 1 + eps, eps of order 1e-7.  With
// sigma(m) = sqrt(a2 |m|^2 + e (o.m)^2) and M m = a2 m + e (o.m) o, the
// homogeneous g(m) = m.d - sigma_i(m) - sigma_j(m) has
//   grad g = R = R' - al n,  R' = d - b_i o_i - b_j o_j  (y_j - y_i at n),
//   b = e (o.n) / sigma,  al = a2_i / sigma_i + a2_j / sigma_j,
//   g(n) = n.R = n.R' - al (1 + eps)  (Euler: n.M n / sigma = sigma),
// so the gap at the unit normal is g(n) (1 - eps/2 + ...), and the gradient
// on the sphere is the part of R normal to n, which is that of R' (al n
// lies along n): R_t = R' - (n.R' / |n|^2) n.  R' and n.R' are formed in
// float-float by compensated sums (the products of the high parts exact,
// every rounding error gathered in one FP32 term); R_t, exactly normal to n
// and small, is rounded to FP32 once formed, so its components along the
// FP32 tangents t1, t2 (orthogonal to n to ~1e-7 only) give the tangential
// gradient to ~1e-14 |d|.  The tangent Hessian and the 2x2 solve run in
// FP32; their relative error e makes the step contract the error by e as
// well, so from the FP32 normal's ~1e-7 rad one step lands near 1e-13 rad.
// The stepped normal m = n + s is normalised by 1 - (|m|^2 - 1)/2, |m|^2 - 1
// of order 1e-7 (the next term is below 1e-14).  Out: nf the unit refined
// normal, hf the gap (float-float).  Returns the squared step length
// (radians^2), or infinity when the refined normal does not point from i
// towards j.
__device__ __forceinline__ float polish_gap_ff(const ff d[3], const ff oi[3], const ff oj[3], float api, float cpi,
                                               float apj, float cpj, const V3<float> n, ff nf[3], ff &hf)
{
    const ff a2i = two_prod(api, api), ei = ff_sub(two_prod(cpi, cpi), a2i);
    const ff a2j = two_prod(apj, apj), ej = ff_sub(two_prod(cpj, cpj), a2j);
    const float nv[3] = {n.x, n.y, n.z};
    const ff nn = ff_dot3_exact(nv, nv);
    const float eps = __fadd_rn(__fsub_rn(nn.hi, 1.0f), nn.lo);  // |n|^2 - 1 (nn.hi - 1 is exact)
    const ff ci = ff_dot3f_c(oi, nv), cj = ff_dot3f_c(oj, nv);
    // sigma^2 = a2 + e c^2 + a2 eps
    ff si2 = ff_add(a2i, ff_mul(ei, ff_mul(ci, ci))), sj2 = ff_add(a2j, ff_mul(ej, ff_mul(cj, cj)));
    si2 = fast_two_sum(si2.hi, __fmaf_rn(a2i.hi, eps, si2.lo));
    sj2 = fast_two_sum(sj2.hi, __fmaf_rn(a2j.hi, eps, sj2.lo));
    const ff ri = ff_rsqrt(si2), rj = ff_rsqrt(sj2);  // 1 / sigma
    const ff al = ff_add(ff_mul(a2i, ri), ff_mul(a2j, rj));
    const ff bi = ff_mul(ff_mul(ei, ci), ri), bj = ff_mul(ff_mul(ej, cj), rj);
    ff Rp[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        // d - b_i o_i - b_j o_j: the high products exact, the rest gathered in e
        const ff p = two_prod(bi.hi, oi[a].hi), q = two_prod(bj.hi, oj[a].hi);
        const ff t = two_sum(d[a].hi, -p.hi);
        const ff u = two_sum(t.hi, -q.hi);
        float e = __fadd_rn(__fadd_rn(d[a].lo, t.lo), __fsub_rn(u.lo, __fadd_rn(p.lo, q.lo)));
        e = __fsub_rn(e, __fmaf_rn(bi.hi, oi[a].lo, __fmul_rn(bi.lo, oi[a].hi)));
        e = __fsub_rn(e, __fmaf_rn(bj.hi, oj[a].lo, __fmul_rn(bj.lo, oj[a].hi)));
        Rp[a] = fast_two_sum(u.hi, e);
    }
    const ff nRp = ff_dot3f_c(Rp, nv);
    // g(n) = n.R' - al - al eps (n.R'.hi - al.hi cancels exactly)
    const ff tg = two_sum(nRp.hi, -al.hi);
    const ff g = fast_two_sum(tg.hi, __fsub_rn(__fadd_rn(tg.lo, __fsub_rn(nRp.lo, al.lo)), __fmul_rn(al.hi, eps)));
    hf = fast_two_sum(g.hi, __fmaf_rn(__fmul_rn(-0.5f, eps), g.hi, g.lo));
    // n.R' / |n|^2 to ~eps^2 relative; R_t = R' - that n, rounded to FP32
    // once formed (R'.hi - p.hi is exact or its rounding is that of R_t)
    const ff lam = fast_two_sum(nRp.hi, __fmaf_rn(-eps, nRp.hi, nRp.lo));
    float Rt[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const ff p = two_prod(lam.hi, nv[a]);
        Rt[a] = __fadd_rn(__fsub_rn(Rp[a].hi, p.hi), __fsub_rn(__fsub_rn(Rp[a].lo, p.lo), __fmul_rn(lam.lo, nv[a])));
    }
    const V3<float> t1 = perp_unit(n), t2 = cross(n, t1);
    const float G1 = t1.x * Rt[0] + t1.y * Rt[1] + t1.z * Rt[2];
    const float G2 = t2.x * Rt[0] + t2.y * Rt[1] + t2.z * Rt[2];
    // P = -Hess_t g in FP32 (as in newton_sphere)
    const V3<float> ofi = mk<float>(oi[0].hi, oi[1].hi, oi[2].hi), ofj = mk<float>(oj[0].hi, oj[1].hi, oj[2].hi);
    const float u1i = dot(ofi, t1), u2i = dot(ofi, t2), u1j = dot(ofj, t1), u2j = dot(ofj, t2);
    const float rif = ri.hi, rjf = rj.hi, gf = g.hi;
    const float Ai = a2i.hi * rif, Aj = a2j.hi * rjf;
    const float Ei = ei.hi * rif * rif, Ej = ej.hi * rjf * rjf;
    const float P11 = Ai * (1.f + Ei * u1i * u1i) + Aj * (1.f + Ej * u1j * u1j) + gf;
    const float P22 = Ai * (1.f + Ei * u2i * u2i) + Aj * (1.f + Ej * u2j * u2j) + gf;
    const float P12 = Ai * Ei * u1i * u2i + Aj * Ej * u1j * u2j;
    const float det = P11 * P22 - P12 * P12;
    float s1, s2;
    if (P11 > 0.f && det > 0.f) {
        const float idet = rcp_fast(det);
        s1 = (P22 * G1 - P12 * G2) * idet;
        s2 = (P11 * G2 - P12 * G1) * idet;
    } else {
        const float sc = rcp_fast(fabsf(P11) + fabsf(P22) + fabsf(P12) + Ai + Aj);
        s1 = G1 * sc;
        s2 = G2 * sc;
    }
    // m = n + s1 t1 + s2 t2 in float-float (the step is of order 1e-7), then
    // m (1 - em/2) with em = |m|^2 - 1 = eps + 2 n.s + |s|^2
    const float tv1[3] = {t1.x, t1.y, t1.z}, tv2[3] = {t2.x, t2.y, t2.z};
    float sv[3];
    ff m[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        sv[a] = __fmaf_rn(s1, tv1[a], __fmul_rn(s2, tv2[a]));
        m[a] = two_sum(nv[a], sv[a]);
    }
    const float ns = nv[0] * sv[0] + nv[1] * sv[1] + nv[2] * sv[2];
    const float ss = sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2];
    const float hem = -0.5f * (eps + (2.0f * ns + ss));
#pragma unroll
    for (int a = 0; a < 3; ++a) nf[a] = fast_two_sum(m[a].hi, __fmaf_rn(hem, m[a].hi, m[a].lo));
    const float step2 = s1 * s1 + s2 * s2;
    const float nd = m[0].hi * d[0].hi + m[1].hi * d[1].hi + m[2].hi * d[2].hi;
    return (nd > 0.f && isfinite(step2)) ? step2 : INFINITY;
}

// LUB_MIXED, FP32 stage of pair k = (i, j): FP32 Newton, then the
// float-float gap and Newton step (spheres: the float-float line of centres).
// The normal and gap in double (n64, h) and in float-float (nf, hf: what the
// fused pass hands to the force kernel).  Returns the FP64 work-list entry
// -1-k (a full FP64 solve from the line of centres, for a pair whose FP32
// Newton did not converge) or kNoEntry.
template <bool ENS>
__device__ __forceinline__ int closest_mixed_one(const PView &P, const DView &D0, const Ens &E,
                                                 const float2 *__restrict__ pff, int i, int j, int k,
                                                 const double *__restrict__ nin, size_t C, int warm, int maxit,
                                                 float tol32, V3<double> &n64, double &h, ff nf[3], ff &hf,
                                                 int &st, int &nit)
{
    int entry = kNoEntry;
    st = 0;
    nit = 0;
    n64 = mk<double>(0, 0, 0);
    h = 0.0;
    nf[0] = nf[1] = nf[2] = hf = ff_make(0.0f);
    bool alien;
    const DView &D = pair_domain<ENS>(D0, E, i, j, &alien);
    // the indices first; the shapes from the records (the same floats as P's)
    bool bad = alien || i < 0 || i >= P.n || j >= P.n || j < -D.n_walls || j == i;
    float4 ri1 = make_float4(0.f, 0.f, 0.f, 0.f), rj1 = ri1;
    if (!bad) {
        ri1 = rec_ld(pff, i, 1);
        bad = !shape_ok(ri1.z, ri1.w);
        if (!bad && j >= 0) {
            rj1 = rec_ld(pff, j, 1);
            bad = !shape_ok(rj1.z, rj1.w);
        }
    }
    if (bad) {
        st = LUB_ST_DEGENERATE;
    } else if (j < 0) {
        h = wall_gap(P, D, i, -1 - j, n64);
        nf[2] = ff_make((float)n64.z);  // +-1
        hf = ff_split_bits(h);
    } else {
        const float4 ri0 = rec_ld(pff, i, 0), rj0 = rec_ld(pff, j, 0);
        ff dff[3];
        ff_separation(ri0, ri1, rj0, rj1, D, dff);
        const V3<float> df = mk<float>(dff[0].hi, dff[1].hi, dff[2].hi);
        const float rpi = ri1.z, rqi = ri1.w, rpj = rj1.z, rqj = rj1.w;
        const float dd2 = dot(df, df);  // |d|^2 in FP32 (float-float for spheres only)
        if (!(dd2 > 0.f) || !isfinite(dd2)) {
            st = LUB_ST_DEGENERATE;
        } else if (rpi == rqi && rpj == rqj) {
            // two spheres: n = d/|d|, h = |d| - R_i - R_j, in float-float
            const ff dd = ff_dot3(dff, dff);
            const ff rs = ff_rsqrt(dd);
#pragma unroll
            for (int a = 0; a < 3; ++a) nf[a] = ff_mul(dff[a], rs);
            hf = ff_sub(ff_sub(ff_mul(dd, rs), ff_make(rpi)), ff_make(rpj));
            n64 = mk<double>(ff_to_double(nf[0]), ff_to_double(nf[1]), ff_to_double(nf[2]));
            h = ff_to_double(hf);
        } else {
            ff oi[3], oj[3];
            ff_axis_rec(rec_ld(pff, i, 2), rec_ld(pff, i, 3), oi);
            ff_axis_rec(rec_ld(pff, j, 2), rec_ld(pff, j, 3), oj);
            const Shape<float> si = shape_ff(oi, rpi, rqi), sj = shape_ff(oj, rpj, rqj);
            const float idl = rsqrtf(dd2), dl = dd2 * idl;  // Newton renormalises its start
            V3<float> n = scl(idl, df);
            if (warm) {
                const V3<float> w0 = mk<float>((float)nin[k], (float)nin[C + k], (float)nin[2 * C + k]);
                const float wl2 = dot(w0, w0);
                // a start on the far hemisphere falls back to the line of centres
                if (wl2 > 0.25f && wl2 < 4.0f && isfinite(wl2) && dot(w0, df) > 0.f) n = scl(rsqrtf(wl2), w0);
            }
            const float scale = dl + fmaxf(rpi, rqi) + fmaxf(rpj, rqj);
            const NewtonOut o = newton_sphere<float>(si, sj, df, n, maxit, tol32, 4e-7f * scale);
            nit = o.iters;
            const float step2 = polish_gap_ff(dff, oi, oj, rqi, rpi, rqj, rpj, n, nf, hf);
            n64 = mk<double>(ff_to_double(nf[0]), ff_to_double(nf[1]), ff_to_double(nf[2]));
            h = ff_to_double(hf);
            if (!o.converged || !(step2 < 1e-10f) || !isfinite(h)) {
                entry = -1 - k;
                st |= LUB_ST_FP64;  // on the work list (solved again in FP64 next)
            }
        }
    }
    if (!(st & LUB_ST_DEGENERATE) && h <= 0.0) st |= LUB_ST_OVERLAP;
    return entry;
}

// LUB_MIXED, a work-list pair (its FP32 Newton did not converge): a
// complete FP64 solve and gap from the line of centres, or, with w0 (the
// network's start), from w0 unless it lies on the far hemisphere
template <bool ENS>
__device__ __forceinline__ void refine_one(const PView &P, const DView &D0, const Ens &E, int i, int j, int maxit,
                                           V3<double> &n64, double &h, int &st, int &nit,
                                           const V3<double> *w0 = nullptr)
{
    bool alien;
    const DView &D = pair_domain<ENS>(D0, E, i, j, &alien);
    const V3<double> d = min_image(D, sub(load_pos(P, j), load_pos(P, i)));
    const double dl = sqrt(dot(d, d));
    const Shape<double> si = load_shape<double>(P, i), sj = load_shape<double>(P, j);
    V3<double> nn = scl(1.0 / dl, d);
    if (w0) {
        const double wl2 = dot(*w0, *w0);
        if (wl2 > 0.25 && wl2 < 4.0 && isfinite(wl2) && dot(*w0, d) > 0.0) nn = *w0;
    }
    const double scale = dl + (double)fmaxf(P.rpar[i], P.rperp[i]) + (double)fmaxf(P.rpar[j], P.rperp[j]);
    const NewtonOut o = newton_sphere<double>(si, sj, d, nn, maxit, kTolFp64, 1e-14 * scale);
    nit = o.iters;
    n64 = normalized(nn);
    h = dot(n64, d) - support(si, n64) - support(sj, n64);
    st = LUB_ST_FP64;
    if (!o.converged || !(dot(n64, d) > 0.0) || !isfinite(h)) st |= LUB_ST_NOCONV;
    if (h <= 0.0) st |= LUB_ST_OVERLAP;
}

// LUB_FP64: the whole solve and gap of pair k in double
template <bool ENS>
__device__ __forceinline__ void closest_fp64_one(const PView &P, const DView &D0, const Ens &E, int i, int j, int k,
                                                 const double *__restrict__ nin, size_t C, int warm, int maxit,
                                                 V3<double> &n64, double &h, int &st, int &nit)
{
    st = 0;
    nit = 0;
    n64 = mk<double>(0, 0, 0);
    h = 0.0;
    bool alien;
    const DView &D = pair_domain<ENS>(D0, E, i, j, &alien);
    if (alien || pair_bad(P, D, i, j)) {
        st = LUB_ST_DEGENERATE;
    } else if (j < 0) {
        h = wall_gap(P, D, i, -1 - j, n64);
    } else {
        const V3<double> d = min_image(D, sub(load_pos(P, j), load_pos(P, i)));
        const double dl = sqrt(dot(d, d));
        if (!(dl > 0.0) || !isfinite(dl)) {
            st = LUB_ST_DEGENERATE;
        } else {
            const float rpi = __ldg(P.rpar + i), rqi = __ldg(P.rperp + i);
            const float rpj = __ldg(P.rpar + j), rqj = __ldg(P.rperp + j);
            if (rpi == rqi && rpj == rqj) {
                n64 = scl(1.0 / dl, d);
                h = dl - (double)rpi - (double)rpj;
            } else {
                const Shape<double> si = load_shape<double>(P, i), sj = load_shape<double>(P, j);
                V3<double> nn = scl(1.0 / dl, d);
                if (warm) {
                    const V3<double> w0 = mk<double>(nin[k], nin[C + k], nin[2 * C + k]);
                    const double wl2 = dot(w0, w0);
                    // a start on the far hemisphere falls back to the line of centres
                    if (wl2 > 0.25 && wl2 < 4.0 && isfinite(wl2) && dot(w0, d) > 0.0) nn = w0;
                }
                const double scale = dl + (double)fmaxf(rpi, rqi) + (double)fmaxf(rpj, rqj);
                const NewtonOut o = newton_sphere<double>(si, sj, d, nn, maxit, kTolFp64, 1e-14 * scale);
                nit = o.iters;
                n64 = normalized(nn);
                h = dot(n64, d) - support(si, n64) - support(sj, n64);
                if (!o.converged || !(dot(n64, d) > 0.0) || !isfinite(h)) st |= LUB_ST_NOCONV;
            }
        }
    }
    if (!(st & LUB_ST_DEGENERATE) && h <= 0.0) st |= LUB_ST_OVERLAP;
}

// The fused pass's hand-over of pair k's unit normal and gap to the force
// kernel in float-float (no conversion from double there): nh[k] = (n_x,
// n_y), nh[C + k] = (n_z, h), each value as (hi, lo).
__device__ __forceinline__ void store_nh(float4 *__restrict__ nh, size_t C, int k, const ff nf[3], ff hf)
{
    nh[k] = make_float4(nf[0].hi, nf[0].lo, nf[1].hi, nf[1].lo);
    nh[C + k] = make_float4(nf[2].hi, nf[2].lo, hf.hi, hf.lo);
}

// the same from a double normal and gap (the FP64 solves of the work list),
// split with integer operations
__device__ __forceinline__ void store_nh(float4 *__restrict__ nh, size_t C, int k, const V3<double> &n64, double h)
{
    const ff nf[3] = {ff_split_bits(n64.x), ff_split_bits(n64.y), ff_split_bits(n64.z)};
    store_nh(nh, C, k, nf, ff_split_bits(h));
}

__device__ __forceinline__ void store_pair(double *__restrict__ nout, double *__restrict__ gap,
                                           uint8_t *__restrict__ status, uint8_t *__restrict__ iters, size_t C, int k,
                                           const V3<double> &n64, double h, int st, int nit)
{
    nout[k] = n64.x;
    nout[C + k] = n64.y;
    nout[2 * C + k] = n64.z;
    if (gap) gap[k] = h;
    if (status) status[k] = (uint8_t)st;
    if (iters) iters[k] = (uint8_t)(nit > 255 ? 255 : nit);
}

// Compacted append to the work list (warp-collective): entries -1-k (full
// FP64 solves), one atomic per warp.  wl_count[0]: entries; the list holds
// cap entries.
__device__ __forceinline__ void worklist_append(int entry, int32_t *__restrict__ wl_count, int32_t *__restrict__ wl,
                                                int cap)
{
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const bool full = entry != kNoEntry;
    const unsigned mf = __ballot_sync(0xffffffffu, full);
    if (mf) {
        int wbase = 0;
        const int leader = __ffs(mf) - 1;
        if (lane == leader) wbase = atomicAdd(wl_count, __popc(mf));
        wbase = __shfl_sync(0xffffffffu, wbase, leader);
        if (full) wl[wbase + __popc(mf & below)] = entry;
    }
}

__device__ __forceinline__ int wl_total(const int32_t *__restrict__ wl_count, int cap)
{
    return min(wl_count[0], cap);
}

// ---------------------------------------------------------------------------
// lub_closest_points kernels
// ---------------------------------------------------------------------------
// The per-call particle records of the FP32 stage and the FP32 resistance
// (rec_ld): float-float centre and symmetry axis, semi-axes and velocities,
// five float4 per particle (one float-float axis per particle instead of one
// per pair and side; four 16-byte loads fetch what a kernel needs)
// With zero16, zf, zt: also clears four counter words and the force and
// torque sums [3][n] of the pass that follows (one launch instead of three).
__global__ void __launch_bounds__(256) k_particles_ff(PView P, float4 *__restrict__ out, int32_t *__restrict__ zero16,
                                                      float *__restrict__ zf, float *__restrict__ zt)
{
    pdl_wait();
    pdl_trigger();
    // each warp's 32 records (2,560 contiguous bytes of out) pass through
    // shared memory, so that their stores are whole 512-byte runs instead of
    // 16-byte pieces at an 80-byte stride
    __shared__ float4 stage[8][32 * kRec];
    if (zero16 && blockIdx.x == 0 && threadIdx.x < 4) zero16[threadIdx.x] = 0;
    const size_t n = (size_t)P.n;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float4 *const sw = stage[w];
    // the loop bound is the same for every lane of a warp (the warp copies its records out together)
    for (int base = blockIdx.x * blockDim.x; base < P.n; base += gridDim.x * blockDim.x) {
        const int i = base + threadIdx.x;
        if (i < P.n) {
            if (zf) {
                zf[i] = 0.f;
                zf[n + i] = 0.f;
                zf[2 * n + i] = 0.f;
            }
            if (zt) {
                zt[i] = 0.f;
                zt[n + i] = 0.f;
                zt[2 * n + i] = 0.f;
            }
            // the centre split from its bits (46 bits: 1.5e-11 at |r| = 1024; no FP64 pipe)
            const ff x = ff_split_bits_nan(P.x[i]), y = ff_split_bits_nan(P.y[i]), z = ff_split_bits_nan(P.z[i]);
            ff o[3];
            ff_axis(P.qw[i], P.qx[i], P.qy[i], P.qz[i], o);
            float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (P.vx) {
                v[0] = P.vx[i];
                v[1] = P.vy[i];
                v[2] = P.vz[i];
                v[3] = P.wx[i];
                v[4] = P.wy[i];
                v[5] = P.wz[i];
            }
            float4 *r = sw + lane * kRec;
            r[0] = make_float4(x.hi, x.lo, y.hi, y.lo);
            r[1] = make_float4(z.hi, z.lo, P.rpar[i], P.rperp[i]);
            r[2] = make_float4(o[0].hi, o[0].lo, o[1].hi, o[1].lo);
            r[3] = make_float4(o[2].hi, o[2].lo, v[0], v[1]);
            r[4] = make_float4(v[2], v[3], v[4], v[5]);
        }
        __syncwarp();
        const int i0 = base + 32 * w;
        const int cnt = P.n - i0 < 32 ? (P.n - i0 > 0 ? P.n - i0 : 0) : 32;
        float4 *dst = out + (size_t)i0 * kRec;
        for (int q = lane; q < cnt * kRec; q += 32) dst[q] = sw[q];
        __syncwarp();
    }
}

template <bool ENS>
__global__ void __launch_bounds__(128, 8) k_closest_mixed(PView P, const __grid_constant__ DView D0, Ens E,
                                                       const int32_t *__restrict__ pi, const int32_t *__restrict__ pj,
                                                       const int32_t *__restrict__ d_count, int32_t cap,
                                                       double *__restrict__ nout, double *__restrict__ gap,
                                                       uint8_t *__restrict__ status, uint8_t *__restrict__ iters,
                                                       int maxit, float tol32, int warm,
                                                       int32_t *__restrict__ wl_count, int32_t *__restrict__ wl,
                                                       const float2 *__restrict__ pff, float4 *__restrict__ nh)
{
    pdl_wait();
    pdl_trigger();
    const int count = pair_count(d_count, cap);
    const size_t C = (size_t)cap;
    // warp-uniform loop bound: the whole warp takes part in the work-list ballot
    for (int base = blockIdx.x * blockDim.x; base < count; base += gridDim.x * blockDim.x) {
        const int k = base + threadIdx.x;
        int entry = kNoEntry;
        if (k < count) {
            const int i = __ldg(pi + k), j = __ldg(pj + k);
            V3<double> n64;
            double h;
            ff nf[3], hf;
            int st, nit;
            entry = closest_mixed_one<ENS>(P, D0, E, pff, i, j, k, nout, C, warm, maxit, tol32, n64, h, nf, hf, st,
                                           nit);
            store_pair(nout, gap, status, iters, C, k, n64, h, st, nit);
            if (nh) store_nh(nh, C, k, nf, hf);
        }
        worklist_append(entry, wl_count, wl, cap);
    }
}

template <bool ENS>
__global__ void __launch_bounds__(32) k_closest_refine(PView P, const __grid_constant__ DView D0, Ens E,
                                                        const int32_t *__restrict__ pi,
                                                        const int32_t *__restrict__ pj, int32_t cap,
                                                        double *__restrict__ nout, double *__restrict__ gap,
                                                        uint8_t *__restrict__ status, uint8_t *__restrict__ iters,
                                                        int maxit, const int32_t *__restrict__ wl_count,
                                                        const int32_t *__restrict__ wl, float4 *__restrict__ nh)
{
    pdl_wait();
    pdl_trigger();
    const int count = wl_total(wl_count, cap);
    const size_t C = (size_t)cap;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < count; q += gridDim.x * blockDim.x) {
        const int k = -1 - wl[q];
        V3<double> n64;
        double h;
        int st, nit;
        refine_one<ENS>(P, D0, E, pi[k], pj[k], maxit, n64, h, st, nit);
        store_pair(nout, gap, status, iters, C, k, n64, h, st, nit);
        if (nh) store_nh(nh, C, k, n64, h);
    }
}

template <bool ENS>
__global__ void __launch_bounds__(128) k_closest_fp64(PView P, const __grid_constant__ DView D0, Ens E,
                                                      const int32_t *__restrict__ pi, const int32_t *__restrict__ pj,
                                                      const int32_t *__restrict__ d_count, int32_t cap,
                                                      double *__restrict__ nout, double *__restrict__ gap,
                                                      uint8_t *__restrict__ status, uint8_t *__restrict__ iters,
                                                      int maxit, int warm)
{
    pdl_wait();
    pdl_trigger();
    const int count = pair_count(d_count, cap);
    const size_t C = (size_t)cap;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
        V3<double> n64;
        double h;
        int st, nit;
        closest_fp64_one<ENS>(P, D0, E, __ldg(pi + k), __ldg(pj + k), k, nout, C, warm, maxit, n64, h, st, nit);
        store_pair(nout, gap, status, iters, C, k, n64, h, st, nit);
    }
}

// ---------------------------------------------------------------------------
// the learned warm start inside the closest-point kernels (the mma.sync
// engine): every warp runs the network for its 32 pairs on the tensor cores,
// forms Newton's start normals from the outputs, writes them to n (the solve
// reads them back from there: the same thread, cached) and solves; one launch
// instead of the network's own, no start normals through HBM in between.
// ---------------------------------------------------------------------------
template <bool ENS>
__global__ void __launch_bounds__(32 * INF_WARPS, 2) k_closest_mixed_learned(
    PView P, const __grid_constant__ DView D0, Ens E, const int32_t *__restrict__ pi, const int32_t *__restrict__ pj,
    const int32_t *__restrict__ d_count, int32_t cap, double *__restrict__ nout, double *__restrict__ gap,
    uint8_t *__restrict__ status, uint8_t *__restrict__ iters, int maxit, float tol32, int32_t *__restrict__ wl_count,
    int32_t *__restrict__ wl, const float2 *__restrict__ pff, float4 *__restrict__ nh, MlpDevice M)
{
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    InfSmem &S = *reinterpret_cast<InfSmem *>(smem_raw);
    stage_weights(S, M);
    __syncthreads();
    const int count = pair_count(d_count, cap);
    const size_t C = (size_t)cap;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = (blockIdx.x * INF_WARPS + w) * 32; base < count; base += gridDim.x * INF_WARPS * 32) {
        const int k = base + lane;
        float f[NI];
        const PairIn in = pair_inputs<ENS>(P, D0, E, pi, pj, k, count, S.mean, S.istd, f);
        const float4 y = warp_mlp(S, S.x[w], S.y[w], f, lane);
        pair_outputs(P, in, y, k, count, C, nout, nullptr);
        int entry = kNoEntry;
        if (k < count) {
            V3<double> n64;
            double h;
            ff nf[3], hf;
            int st, nit;
            entry = closest_mixed_one<ENS>(P, D0, E, pff, __ldg(pi + k), __ldg(pj + k), k, nout, C, 1, maxit, tol32,
                                           n64, h, nf, hf, st, nit);
            store_pair(nout, gap, status, iters, C, k, n64, h, st, nit);
            if (nh) store_nh(nh, C, k, nf, hf);
        }
        worklist_append(entry, wl_count, wl, cap);
    }
}

template <bool ENS>
__global__ void __launch_bounds__(32 * INF_WARPS, 2) k_closest_fp64_learned(
    PView P, const __grid_constant__ DView D0, Ens E, const int32_t *__restrict__ pi, const int32_t *__restrict__ pj,
    const int32_t *__restrict__ d_count, int32_t cap, double *__restrict__ nout, double *__restrict__ gap,
    uint8_t *__restrict__ status, uint8_t *__restrict__ iters, int maxit, MlpDevice M)
{
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    InfSmem &S = *reinterpret_cast<InfSmem *>(smem_raw);
    stage_weights(S, M);
    __syncthreads();
    const int count = pair_count(d_count, cap);
    const size_t C = (size_t)cap;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = (blockIdx.x * INF_WARPS + w) * 32; base < count; base += gridDim.x * INF_WARPS * 32) {
        const int k = base + lane;
        float f[NI];
        const PairIn in = pair_inputs<ENS>(P, D0, E, pi, pj, k, count, S.mean, S.istd, f);
        const float4 y = warp_mlp(S, S.x[w], S.y[w], f, lane);
        pair_outputs(P, in, y, k, count, C, nout, nullptr);
        if (k < count) {
            V3<double> n64;
            double h;
            int st, nit;
            closest_fp64_one<ENS>(P, D0, E, __ldg(pi + k), __ldg(pj + k), k, nout, C, 1, maxit, n64, h, st, nit);
            store_pair(nout, gap, status, iters, C, k, n64, h, st, nit);
        }
    }
}

// LUB_WARM_MLP in mixed precision: the FP64 solves of the work list start
// from the network's prediction (mma.sync engine; every warp runs the
// network for 32 entries, writes the start normals to n and solves them)
template <bool ENS>
__global__ void __launch_bounds__(32 * INF_WARPS) k_closest_refine_learned(
    PView P, const __grid_constant__ DView D0, Ens E, const int32_t *__restrict__ pi, const int32_t *__restrict__ pj,
    int32_t cap, double *__restrict__ nout, double *__restrict__ gap, uint8_t *__restrict__ status,
    uint8_t *__restrict__ iters, int maxit, const int32_t *__restrict__ wl_count, const int32_t *__restrict__ wl,
    float4 *__restrict__ nh, MlpDevice M)
{
    pdl_wait();
    pdl_trigger();
    const int nwl = wl_total(wl_count, cap);
    if (nwl == 0) return;  // the usual case: no weights to stage
    extern __shared__ __align__(16) unsigned char smem_raw[];
    InfSmem &S = *reinterpret_cast<InfSmem *>(smem_raw);
    stage_weights(S, M);
    __syncthreads();
    const size_t C = (size_t)cap;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = (blockIdx.x * INF_WARPS + w) * 32; base < nwl; base += gridDim.x * INF_WARPS * 32) {
        const int q = base + lane;
        const bool act = q < nwl;
        const int k = act ? -1 - wl[q] : 0;
        const int cnt = act ? k + 1 : 0;  // pair k is valid for the helpers iff act
        float f[NI];
        const PairIn in = pair_inputs<ENS>(P, D0, E, pi, pj, k, cnt, S.mean, S.istd, f);
        const float4 y = warp_mlp(S, S.x[w], S.y[w], f, lane);
        pair_outputs(P, in, y, k, cnt, C, nout, nullptr);
        if (act) {
            const V3<double> w0 = mk<double>(nout[k], nout[C + k], nout[2 * C + k]);
            V3<double> n64;
            double h;
            int st, nit;
            refine_one<ENS>(P, D0, E, pi[k], pj[k], maxit, n64, h, st, nit, &w0);
            store_pair(nout, gap, status, iters, C, k, n64, h, st, nit);
            if (nh) store_nh(nh, C, k, n64, h);
        }
    }
}

// the shared-memory size of the learned kernels, set once per kernel (bits 16..)
template <typename K>
int learned_smem(lub_ctx *ctx, K kernel, int bit)
{
    if (ctx->mlp_smem_set & bit) return LUB_OK;
    const int rc = lub_check_cuda(
        ctx, cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(InfSmem)),
        "shared memory attribute");
    if (!rc) ctx->mlp_smem_set |= bit;
    return rc;
}

// ---------------------------------------------------------------------------
// fused pass (lub_correct): closest points, resistance and the atomic scatter
// of each pair without leaving registers.  nout is required (it holds the
// start normals and carries the FP32 normals to the refinement); gap,
// status, iters, FT and lever are written where given.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void store_force(T *__restrict__ FT, T *__restrict__ lever, size_t C, int k,
                                            const T out[12])
{
    if (FT)
#pragma unroll
        for (int a = 0; a < 6; ++a) FT[a * C + k] = out[a];
    if (lever)
#pragma unroll
        for (int a = 0; a < 6; ++a) lever[a * C + k] = out[6 + a];
}

// forces of a finished pair and its share of the warp's scatter
template <typename T>
__device__ __forceinline__ void force_and_scatter(const PView &P, const RParams &R, bool done, int i, int j,
                                                  const V3<double> &n64, double h, int &st, T *__restrict__ FT,
                                                  T *__restrict__ lever, size_t C, int k, T *__restrict__ force,
                                                  T *__restrict__ torque, const float2 *__restrict__ pff)
{
    T out[12];
    T ci[6] = {0, 0, 0, 0, 0, 0}, cj[6] = {0, 0, 0, 0, 0, 0};
    if (done) {
        pair_force<T>(P, R, i, j, n64, h, st, out, pff);
        store_force(FT, lever, C, k, out);
        side_contrib(out, 0, ci);
        if (j >= 0) side_contrib(out, 1, cj);
    }
    // the closest-point solve validated the indices of every pair without DEGENERATE
    const bool ok = done && !(st & LUB_ST_DEGENERATE);
    scatter_warp<T>(ok ? i : -1, ok ? j : -1, (size_t)P.n, ci, cj, force, torque);
}

template <bool ENS>
__global__ void __launch_bounds__(128) k_fused_fp64(PView P, const __grid_constant__ DView D0, Ens E, RParams R,
                                                    const int32_t *__restrict__ pi, const int32_t *__restrict__ pj,
                                                    const int32_t *__restrict__ d_count, int32_t cap,
                                                    double *__restrict__ nout, double *__restrict__ gap,
                                                    uint8_t *__restrict__ status, uint8_t *__restrict__ iters,
                                                    double *__restrict__ FT, double *__restrict__ lever, int maxit,
                                                    int warm, double *__restrict__ force, double *__restrict__ torque)
{
    pdl_wait();
    pdl_trigger();
    const int count = pair_count(d_count, cap);
    const size_t C = (size_t)cap;
    for (int base = blockIdx.x * blockDim.x; base < count; base += gridDim.x * blockDim.x) {
        const int k = base + threadIdx.x;
        int i = -1, j = -1, st = 0, nit = 0;
        V3<double> n64 = mk<double>(0, 0, 0);
        double h = 0.0;
        if (k < count) {
            i = __ldg(pi + k);
            j = __ldg(pj + k);
            closest_fp64_one<ENS>(P, D0, E, i, j, k, nout, C, warm, maxit, n64, h, st, nit);
        }
        force_and_scatter<double>(P, R, k < count, i, j, n64, h, st, FT, lever, C, k, force, torque, nullptr);
        if (k < count) store_pair(nout, gap, status, iters, C, k, n64, h, st, nit);
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// whether the network starts every pair's Newton solve (LUB_WARM_MLP_ALL,
// or LUB_WARM_MLP in FP64) or only the FP64 solves of the mixed work list
inline bool net_every_pair(const lub_params &prm)
{
    return prm.warm_start == LUB_WARM_MLP_ALL || (prm.warm_start == LUB_WARM_MLP && prm.precision == LUB_FP64);
}

// the network's start normals for every pair (learned warm start), then
// whether Newton starts from n
int start_normals(lub_ctx *ctx, const PView &P, const DView &D, const Ens &E, const lub_params &prm,
                  const int32_t *pi, const int32_t *pj, const int32_t *d_count, int32_t cap, double *n,
                  cudaStream_t st, int *warm)
{
    *warm = prm.warm_start == LUB_WARM_PREVIOUS;
    if (net_every_pair(prm)) {
        int rc = launch_mlp_start(ctx, P, D, E, pi, pj, d_count, cap, n, nullptr, st);
        if (rc) return rc;
        *warm = 1;
    }
    return LUB_OK;
}

}  // namespace

int launch_particles_ff(lub_ctx *ctx, const PView &P, float2 *out, cudaStream_t st, int32_t *zero16, float *zf,
                        float *zt)
{
    if (P.n == 0) {
        if (!zero16) return LUB_OK;
        return zero_async(ctx, ctx->num_sms, zero16, 16, st);
    }
    return lub_check_cuda(ctx,
                          launch_pdl(k_particles_ff, grid_for(P.n, 256, ctx->num_sms, 32), 256, 0, st, P,
                                     reinterpret_cast<float4 *>(out), zero16, zf, zt),
                          "particle table launch");
}

namespace {

// The work list of the mixed mode in the context scratch: counters [entries,
// unused, queue 0, queue 1] and cap entries; with nh and status_in (the
// fused pass), also the hand-over of normals and gaps in float-float (32
// bytes a pair, store_nh) and a status array for callers that pass none;
// with P, the per-call particle table (pff: 80 bytes per particle).
int work_list(lub_ctx *ctx, int32_t cap, cudaStream_t st, int32_t **wl_count, int32_t **wl,
              float4 **nh = nullptr, uint8_t **status_in = nullptr, const PView *P = nullptr,
              float2 **pff = nullptr, float *zf = nullptr, float *zt = nullptr)
{
    const size_t b_wl = ((4 * (size_t)cap + 255) / 256) * 256, b_nh = nh ? ((32 * (size_t)cap + 255) / 256) * 256 : 0,
                 b_st = (((size_t)cap + 255) / 256) * 256, b_pos = P ? particles_ff_bytes(P->n) : 0;
    int rc = lub_ensure_scratch(ctx, 256 + b_wl + b_nh + b_st + b_pos);
    if (rc) return rc;
    char *base = (char *)ctx->scratch;
    *wl_count = (int32_t *)base;
    *wl = (int32_t *)(base + 256);
    if (nh) *nh = (float4 *)(base + 256 + b_wl);
    if (status_in && !*status_in) *status_in = (uint8_t *)(base + 256 + b_wl + b_nh);
    if (!P) return zero_async(ctx, ctx->num_sms, *wl_count, 16, st);
    // the particle table's kernel also clears the counters (and the sums zf, zt)
    *pff = (float2 *)(base + 256 + b_wl + b_nh + b_st);
    return launch_particles_ff(ctx, *P, *pff, st, *wl_count, zf, zt);
}

// What lub_correct hands from the closest-point kernels of the mixed mode to
// the force pass: the status array (the caller's, or the context scratch's
// where it passes none), the per-call particle records and the normals and
// gaps in float-float.
struct ClosestKeep {
    uint8_t *status;
    const float2 *pff;
    const float4 *nh;
};

template <bool ENS>
int launch_closest_t(lub_ctx *ctx, const PView &P, const DView &D, const Ens &E, const lub_params &prm,
                     const int32_t *pi, const int32_t *pj, const int32_t *d_count, int32_t cap, double *n, double *gap,
                     uint8_t *status, uint8_t *iters, cudaStream_t st, ClosestKeep *keep = nullptr,
                     float *zero_force = nullptr, float *zero_torque = nullptr)
{
    int warm = 0, rc;
    const bool net_all = net_every_pair(prm);
    const bool net_wl = prm.warm_start == LUB_WARM_MLP && prm.precision == LUB_MIXED;
    if ((net_all || net_wl) && !ctx->mlp_ready)
        return lub_set_error(ctx, LUB_ERR_ARG, "the learned warm start needs lub_mlp_set first");
    // the learned start of every pair on the mma.sync engine runs inside the solve's kernel
    const bool fused_mlp = net_all && ctx->mlp_engine == LUB_MLP_MMA_SYNC;
    if (!fused_mlp && (rc = start_normals(ctx, P, D, E, prm, pi, pj, d_count, cap, n, st, &warm))) return rc;
    const int learned_grid = 2 * ctx->num_sms;
    if (prm.precision == LUB_MIXED) {
        int32_t *wl_count, *wl;
        float2 *pff = nullptr;
        float4 *nh = nullptr;
        if ((rc = work_list(ctx, cap, st, &wl_count, &wl, keep ? &nh : nullptr, keep ? &status : nullptr, &P, &pff,
                            zero_force, zero_torque)))
            return rc;
        if (keep) *keep = ClosestKeep{status, pff, nh};
        lub_trace_mark(ctx, LUB_TRACE_CLOSEST, st);
        if (fused_mlp) {
            if ((rc = learned_smem(ctx, k_closest_mixed_learned<ENS>, 16 << ENS))) return rc;
            (void)launch_pdl(k_closest_mixed_learned<ENS>, learned_grid, 32 * INF_WARPS, sizeof(InfSmem), st, P, D, E,
                             pi, pj, d_count, cap, n, gap, status, iters, prm.max_newton, (float)prm.newton_tol,
                             wl_count, wl, (const float2 *)pff, nh, *(const MlpDevice *)ctx->mlp);
        } else {
            const Shape2 sh = tuned_shape(ctx, LUB_TUNE_CLOSEST_MIXED, cap);
            (void)launch_pdl(k_closest_mixed<ENS>, sh.grid, sh.block, 0, st, P, D, E, pi, pj, d_count, cap, n, gap,
                             status, iters, prm.max_newton, (float)prm.newton_tol, warm, wl_count, wl,
                             (const float2 *)pff, nh);
        }
        lub_trace_mark(ctx, LUB_TRACE_CLOSEST, st);
        if (net_wl) {
            // the work list's FP64 solves from the network's start (returns at once when it is empty)
            if ((rc = learned_smem(ctx, k_closest_refine_learned<ENS>, 256 << ENS))) return rc;
            (void)launch_pdl(k_closest_refine_learned<ENS>, ctx->num_sms, 32 * INF_WARPS, sizeof(InfSmem), st, P, D,
                             E, pi, pj, cap, n, gap, status, iters, prm.max_newton, (const int32_t *)wl_count,
                             (const int32_t *)wl, nh, *(const MlpDevice *)ctx->mlp);
        } else {
            // small blocks so the (short) work list spreads over every SM
            const Shape2 sr = tuned_shape(ctx, LUB_TUNE_CLOSEST_REFINE, cap);
            (void)launch_pdl(k_closest_refine<ENS>, sr.grid, sr.block, 0, st, P, D, E, pi, pj, cap, n, gap, status,
                             iters, prm.max_newton, (const int32_t *)wl_count, (const int32_t *)wl, nh);
        }
    } else if (fused_mlp) {
        if ((rc = learned_smem(ctx, k_closest_fp64_learned<ENS>, 64 << ENS))) return rc;
        lub_trace_mark(ctx, LUB_TRACE_CLOSEST, st);
        (void)launch_pdl(k_closest_fp64_learned<ENS>, learned_grid, 32 * INF_WARPS, sizeof(InfSmem), st, P, D, E, pi,
                         pj, d_count, cap, n, gap, status, iters, prm.max_newton, *(const MlpDevice *)ctx->mlp);
        lub_trace_mark(ctx, LUB_TRACE_CLOSEST, st);
    } else {
        const Shape2 sh = tuned_shape(ctx, LUB_TUNE_CLOSEST_FP64, cap);
        lub_trace_mark(ctx, LUB_TRACE_CLOSEST, st);
        (void)launch_pdl(k_closest_fp64<ENS>, sh.grid, sh.block, 0, st, P, D, E, pi, pj, d_count, cap, n, gap, status,
                         iters, prm.max_newton, warm);
        lub_trace_mark(ctx, LUB_TRACE_CLOSEST, st);
    }
    return lub_check_cuda(ctx, cudaGetLastError(), "k_closest launch");
}

template <bool ENS>
int launch_correct_t(lub_ctx *ctx, const PView &P, const DView &D, const Ens &E, const lub_params &prm,
                     const int32_t *pi, const int32_t *pj, const int32_t *d_count, int32_t cap, double *n, double *gap,
                     uint8_t *status, uint8_t *iters, void *FT, void *lever, void *force, void *torque,
                     int accumulate, cudaStream_t st)
{
    const size_t esz = prm.precision == LUB_MIXED ? sizeof(float) : sizeof(double);
    int rc;
    if (!accumulate && (prm.precision != LUB_MIXED || cap == 0)) {
        if ((rc = zero_force_torque(ctx, force, torque, 3 * (size_t)P.n * esz, st))) return rc;
    }
    if (cap == 0) return LUB_OK;
    if (prm.precision == LUB_MIXED) {
        // the kernels of lub_closest_points, then those of lub_resistance_apply
        // on the same per-call particle records (built once; their kernel also
        // clears the sums unless accumulate is set)
        ClosestKeep keep;
        if ((rc = launch_closest_t<ENS>(ctx, P, D, E, prm, pi, pj, d_count, cap, n, gap, status, iters, st, &keep,
                                        accumulate ? nullptr : (float *)force,
                                        accumulate ? nullptr : (float *)torque)))
            return rc;
        return launch_resistance_apply(ctx, P, D, E, prm, pi, pj, d_count, cap, n, gap, keep.status, FT, lever,
                                       force, torque, 1, st, keep.pff, keep.nh);
    }
    int warm = 0;
    if ((rc = start_normals(ctx, P, D, E, prm, pi, pj, d_count, cap, n, st, &warm))) return rc;
    const RParams R = make_rparams(prm);
    const Shape2 sh = tuned_shape(ctx, LUB_TUNE_CLOSEST_FP64, cap);
    (void)launch_pdl(k_fused_fp64<ENS>, sh.grid, sh.block, 0, st, P, D, E, R, pi, pj, d_count, cap, n, gap, status,
                     iters, (double *)FT, (double *)lever, prm.max_newton, warm, (double *)force, (double *)torque);
    return lub_check_cuda(ctx, cudaGetLastError(), "fused pass launch");
}

// Temporal warm start: the previous list's normal of the same pair.  Both
// lists are canonical (particle pairs by (i, j), then wall pairs by (i, w)).
// First pass: the range of every particle's pairs in the previous list's
// particle segment (rng[i] = (begin, end), zero = none); second pass: each
// pair searches its particle's range (a few entries), wall pairs the wall
// segment by binary search.

// index of the previous list's first wall pair (pj < 0 from there on)
__device__ __forceinline__ int wall_segment(const int32_t *__restrict__ qj, int mq)
{
    int lo = 0, hi = mq;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(qj + mid) >= 0)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(256) k_carry_ranges(const int32_t *__restrict__ qi, const int32_t *__restrict__ qj,
                                                      const int32_t *__restrict__ q_count, int32_t qcap, int32_t n,
                                                      int2 *__restrict__ rng)
{
    __shared__ int seg_s;
    const int mq = pair_count(q_count, qcap);
    if (threadIdx.x == 0) seg_s = wall_segment(qj, mq);
    __syncthreads();
    const int seg = seg_s;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < seg; k += gridDim.x * blockDim.x) {
        const int i = qi[k];
        if (i < 0 || i >= n) continue;
        if (k == 0 || qi[k - 1] != i) rng[i].x = k;
        if (k == seg - 1 || qi[k + 1] != i) rng[i].y = k + 1;
    }
}

__global__ void __launch_bounds__(256) k_carry_normals(const int32_t *__restrict__ qi, const int32_t *__restrict__ qj,
                                                       const double *__restrict__ qn,
                                                       const int32_t *__restrict__ q_count, int32_t qcap,
                                                       const int2 *__restrict__ rng, int32_t n_particles,
                                                       const int32_t *__restrict__ pi, const int32_t *__restrict__ pj,
                                                       const int32_t *__restrict__ d_count, int32_t cap,
                                                       double *__restrict__ n)
{
    __shared__ int seg_s;
    const int mq = pair_count(q_count, qcap);
    if (threadIdx.x == 0) seg_s = wall_segment(qj, mq);
    __syncthreads();
    const int seg = seg_s;
    const int count = pair_count(d_count, cap);
    const size_t C = (size_t)cap, QC = (size_t)qcap;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
        const int i = pi[k], j = pj[k];
        int hit = -1;
        if (i >= 0 && i < n_particles) {
            if (j >= 0) {
                const int2 r = rng[i];
                for (int q = r.x; q < r.y; ++q)
                    if (__ldg(qj + q) == j) {
                        hit = q;
                        break;
                    }
            } else {
                // wall pairs by (i, w): key i * 4 + w
                const int64_t key = (int64_t)i * 4 + (-1 - j);
                int lo = seg, hi = mq;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    const int64_t km = (int64_t)__ldg(qi + mid) * 4 + (-1 - __ldg(qj + mid));
                    if (km < key)
                        lo = mid + 1;
                    else
                        hi = mid;
                }
                if (lo < mq && __ldg(qi + lo) == i && __ldg(qj + lo) == j) hit = lo;
            }
        }
        double x = 0.0, y = 0.0, z = 0.0;
        if (hit >= 0) {
            x = qn[hit];
            y = qn[QC + hit];
            z = qn[2 * QC + hit];
        }
        n[k] = x;
        n[C + k] = y;
        n[2 * C + k] = z;
    }
}

}  // namespace

int launch_carry_normals(lub_ctx *ctx, int32_t n_particles, const int32_t *qi, const int32_t *qj, const double *qn,
                         const int32_t *q_count, int32_t qcap, const int32_t *pi, const int32_t *pj,
                         const int32_t *d_count, int32_t cap, double *n, cudaStream_t st)
{
    if (cap == 0) return LUB_OK;
    const size_t bytes = (size_t)(n_particles > 0 ? n_particles : 1) * sizeof(int2);
    int rc = lub_ensure_scratch(ctx, bytes);
    if (rc) return rc;
    int2 *rng = (int2 *)ctx->scratch;
    if ((rc = lub_check_cuda(ctx, cudaMemsetAsync(rng, 0, bytes, st), "memset ranges"))) return rc;
    if (qcap > 0)
        k_carry_ranges<<<grid_for(qcap, 256, ctx->num_sms, 16), 256, 0, st>>>(qi, qj, q_count, qcap, n_particles, rng);
    k_carry_normals<<<grid_for(cap, 256, ctx->num_sms, 16), 256, 0, st>>>(qi, qj, qn, q_count, qcap, rng, n_particles,
                                                                          pi, pj, d_count, cap, n);
    return lub_check_cuda(ctx, cudaGetLastError(), "carry launch");
}

int launch_correct(lub_ctx *ctx, const PView &P, const DView &D, const Ens &E, const lub_params &prm,
                   const int32_t *pi, const int32_t *pj, const int32_t *d_count, int32_t cap, double *n, double *gap,
                   uint8_t *status, uint8_t *iters, void *FT, void *lever, void *force, void *torque, int accumulate,
                   cudaStream_t st)
{
    return E.nb ? launch_correct_t<true>(ctx, P, D, E, prm, pi, pj, d_count, cap, n, gap, status, iters, FT, lever,
                                         force, torque, accumulate, st)
                : launch_correct_t<false>(ctx, P, D, E, prm, pi, pj, d_count, cap, n, gap, status, iters, FT, lever,
                                          force, torque, accumulate, st);
}

int launch_closest(lub_ctx *ctx, const PView &P, const DView &D, const Ens &E, const lub_params &prm,
                   const int32_t *pi, const int32_t *pj, const int32_t *d_count, int32_t cap, double *n, double *gap,
                   uint8_t *status, uint8_t *iters, cudaStream_t st)
{
    if (cap == 0) return LUB_OK;
    return E.nb ? launch_closest_t<true>(ctx, P, D, E, prm, pi, pj, d_count, cap, n, gap, status, iters, st)
                : launch_closest_t<false>(ctx, P, D, E, prm, pi, pj, d_count, cap, n, gap, status, iters, st);
}
