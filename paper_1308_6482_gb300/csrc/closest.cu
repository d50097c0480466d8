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
//   * the gap of every pair in float-float arithmetic (about 48 bits, on the
//     FP32 pipe): h is stationary in n, so the FP32 normal costs only
//     O(dn^2), while the subtraction n.d - sigma_i - sigma_j cancels far
//     beyond FP32 for small gaps;
//   * pairs with h/a below fp64_switch (and pairs whose FP32 Newton did not
//     converge) are appended to a compacted work list (one atomic per warp)
//     and refined by FP64 Newton in a second kernel, so only full warps of
//     such pairs use the slow FP64 pipe.
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

// symmetry axis of q/|q| in float-float (quaternion components exact)
__device__ __forceinline__ void ff_axis(float w, float x, float y, float z, ff o[3])
{
    const ff q2 = ff_add(ff_add(two_prod(w, w), two_prod(x, x)), ff_add(two_prod(y, y), two_prod(z, z)));
    // s = 2 / |q|^2: float reciprocal plus one correction with the exact residual
    const float r0 = __fdiv_rn(2.0f, q2.hi);
    const ff res = ff_sub(ff_make(2.0f), ff_mulf(q2, r0));
    const ff s = fast_two_sum(r0, __fmul_rn(res.hi, __fmul_rn(r0, 0.5f)));
    o[0] = ff_mul(s, ff_add(two_prod(x, z), two_prod(w, y)));
    o[1] = ff_mul(s, ff_sub(two_prod(y, z), two_prod(w, x)));
    o[2] = ff_sub(ff_make(1.0f), ff_mul(s, ff_add(two_prod(x, x), two_prod(y, y))));
}

// sigma(n) = sqrt(R_perp^2 |n|^2 + (R_par^2 - R_perp^2) (o.n)^2) in float-float,
// for an exactly represented (not necessarily unit) float n with |n|^2 = nn
__device__ __forceinline__ ff ff_support(const PView &P, int k, const float n[3], ff nn)
{
    ff o[3];
    ff_axis(__ldg(P.qw + k), __ldg(P.qx + k), __ldg(P.qy + k), __ldg(P.qz + k), o);
    const float a = __ldg(P.rperp + k), c = __ldg(P.rpar + k);
    const ff on = ff_add(ff_add(ff_mulf(o[0], n[0]), ff_mulf(o[1], n[1])), ff_mulf(o[2], n[2]));
    const ff a2 = two_prod(a, a);
    const ff e = ff_sub(two_prod(c, c), a2);
    return ff_sqrt(ff_add(ff_mul(a2, nn), ff_mul(e, ff_mul(on, on))));
}

// g at the unit vector n/|n|, in float-float: g is homogeneous of degree one,
// so g(n/|n|) = g(n) / |n| = g(n) (1 - (|n|^2 - 1)/2 + ...), |n|^2 - 1 ~ 1e-7
__device__ __forceinline__ ff ff_gap(const PView &P, int i, int j, const ff d[3], const float n[3])
{
    const ff nn = ff_add(ff_add(two_prod(n[0], n[0]), two_prod(n[1], n[1])), two_prod(n[2], n[2]));
    const ff nd = ff_add(ff_add(ff_mulf(d[0], n[0]), ff_mulf(d[1], n[1])), ff_mulf(d[2], n[2]));
    const ff G = ff_sub(ff_sub(nd, ff_support(P, i, n, nn)), ff_support(P, j, n, nn));
    const float eps = __fadd_rn(__fsub_rn(nn.hi, 1.0f), nn.lo);
    return ff_sub(G, ff_make(__fmul_rn(G.hi, __fmul_rn(0.5f, eps))));
}

// Minimum-image separation r_j - r_i in float-float from the particles'
// float-float positions (pff: [3][N] (hi, lo)); the image shift is taken from
// the float part (listed pairs are far from the ambiguous half box).  About
// 48 bits: an absolute error near 2^-48 |r| (4e-12 at |r| = 1000), against
// the FP64 subtraction and splitting it replaces (some 24 FP64 operations per
// pair, at 1/64 of the FP32 rate).
__device__ __forceinline__ void ff_separation(const float2 *__restrict__ pff, size_t N, int i, int j,
                                              const DView &D, ff d[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float2 pi = __ldg(pff + a * N + i), pj = __ldg(pff + a * N + j);
        ff da = ff_sub(ff{pj.x, pj.y}, ff{pi.x, pi.y});
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

// LUB_MIXED, FP32 stage of pair k = (i, j): FP32 Newton + float-float gap.
// Returns the FP64 work-list entry: k (refine from the FP32 normal), -1-k
// (full FP64 solve from the line of centres) or kNoEntry.
template <bool ENS>
__device__ __forceinline__ int closest_mixed_one(const PView &P, const DView &D0, const Ens &E,
                                                 const float2 *__restrict__ pff, int i, int j, int k,
                                                 const double *__restrict__ nin, size_t C, int warm, int maxit,
                                                 float tol32, float fp64_switch, V3<double> &n64, double &h, int &st,
                                                 int &nit)
{
    int entry = kNoEntry;
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
        ff dff[3];
        ff_separation(pff, (size_t)P.n, i, j, D, dff);
        const V3<float> df = mk<float>(dff[0].hi, dff[1].hi, dff[2].hi);
        const float rpi = __ldg(P.rpar + i), rqi = __ldg(P.rperp + i);
        const float rpj = __ldg(P.rpar + j), rqj = __ldg(P.rperp + j);
        const ff dd = ff_add(ff_add(ff_mul(dff[0], dff[0]), ff_mul(dff[1], dff[1])), ff_mul(dff[2], dff[2]));
        if (!(dd.hi > 0.f) || !isfinite(dd.hi)) {
            st = LUB_ST_DEGENERATE;
        } else if (rpi == rqi && rpj == rqj) {
            // two spheres: n = d/|d|, h = |d| - R_i - R_j
            const ff dl = ff_sqrt(dd);
            const float inv = 1.0f / dl.hi;
            n64 = mk<double>(df.x * inv, df.y * inv, df.z * inv);
            h = ff_to_double(ff_sub(ff_sub(dl, ff_make(rpi)), ff_make(rpj)));
        } else {
            const Shape<float> si = load_shape<float>(P, i), sj = load_shape<float>(P, j);
            const float dl = sqrtf(dd.hi);
            V3<float> n = scl(1.0f / dl, df);
            if (warm) {
                const V3<float> w0 = mk<float>((float)nin[k], (float)nin[C + k], (float)nin[2 * C + k]);
                const float wl2 = dot(w0, w0);
                // a start on the far hemisphere falls back to the line of centres
                if (wl2 > 0.25f && wl2 < 4.0f && isfinite(wl2) && dot(w0, df) > 0.f) n = scl(rsqrtf(wl2), w0);
            }
            const float scale = dl + fmaxf(rpi, rqi) + fmaxf(rpj, rqj);
            const NewtonOut o = newton_sphere<float>(si, sj, df, n, maxit, tol32, 4e-7f * scale);
            nit = o.iters;
            const float nv[3] = {n.x, n.y, n.z};
            const ff hff = ff_gap(P, i, j, dff, nv);
            h = ff_to_double(hff);
            // unit normal for the output (|n|^2 - 1 ~ 1e-7)
            const float nn = dot(n, n);
            const float f = 1.5f - 0.5f * nn;
            n64 = mk<double>(n.x * f, n.y * f, n.z * f);
            const float amin = fminf(fminf(rpi, rqi), fminf(rpj, rqj));
            // (the switch compared in FP32: a heuristic threshold, no FP64 pipe)
            if (!o.converged || !isfinite(hff.hi))
                entry = -1 - k;
            else if (hff.hi < fp64_switch * amin)
                entry = k;
            if (entry != kNoEntry) st |= LUB_ST_FP64;  // on the work list (refined next)
            // consistency check of Sec. III A: the normals point to the other centre
            if (entry == kNoEntry && !(dot(n, df) > 0.f)) st |= LUB_ST_NOCONV;
        }
    }
    if (!(st & LUB_ST_DEGENERATE) && h <= 0.0) st |= LUB_ST_OVERLAP;
    return entry;
}

// One Newton step of g from the FP32 normal n of a work-list pair, in
// float-float on the FP32 pipe (about 48 bits; GB300 runs FP64 at 1/64 of
// the FP32 rate).  It works on the homogeneous g(m) = m.d - sigma_i(m) -
// sigma_j(m), sigma(m) = sqrt(a2 |m|^2 + e (o.m)^2), at m = n itself (an exact
// float vector, |n|^2 = 1 + O(1e-7)), with
//   t.grad sigma = (a2 (t.n) + e (o.n)(o.t)) / sigma.
// The tangents t1, t2 (FP32) are orthogonal to n to about 1e-7 only, so the
// gradient is projected: G_a = t_a.grad g - (t_a.n) g / |n|^2 (n.grad g = g by
// Euler's theorem), which vanishes exactly at the stationary point.  G to
// about 1e-14 absolute; the tangent Hessian and the 2x2 solve in FP32, whose
// relative error e makes the step contract the error by e as well, so from
// 1e-7 one step lands near 1e-14.  The refined unit normal goes to n64.
// Returns the step length (radians), or infinity when the normal does not
// point from i towards j.
__device__ __forceinline__ float polish_ff(const PView &P, const float2 *__restrict__ pff, const DView &D, int i,
                                           int j, const V3<float> n, V3<double> &n64)
{
    ff d[3], oi[3], oj[3];
    ff_separation(pff, (size_t)P.n, i, j, D, d);
    ff_axis(__ldg(P.qw + i), __ldg(P.qx + i), __ldg(P.qy + i), __ldg(P.qz + i), oi);
    ff_axis(__ldg(P.qw + j), __ldg(P.qx + j), __ldg(P.qy + j), __ldg(P.qz + j), oj);
    const float api = __ldg(P.rperp + i), cpi = __ldg(P.rpar + i);
    const float apj = __ldg(P.rperp + j), cpj = __ldg(P.rpar + j);
    const ff a2i = two_prod(api, api), ei = ff_sub(two_prod(cpi, cpi), a2i);
    const ff a2j = two_prod(apj, apj), ej = ff_sub(two_prod(cpj, cpj), a2j);
    const float nv[3] = {n.x, n.y, n.z};
    const ff nn = ff_dot3_exact(nv, nv);
    const ff ci = ff_dot3f(oi, nv), cj = ff_dot3f(oj, nv);
    const ff si = ff_sqrt(ff_add(ff_mul(a2i, nn), ff_mul(ei, ff_mul(ci, ci))));
    const ff sj = ff_sqrt(ff_add(ff_mul(a2j, nn), ff_mul(ej, ff_mul(cj, cj))));
    const ff ri = ff_rcp(si), rj = ff_rcp(sj);
    const ff g = ff_sub(ff_sub(ff_dot3f(d, nv), si), sj);
    const float lam = __fdiv_rn(g.hi, nn.hi);
    const V3<float> t1 = perp_unit(n), t2 = cross(n, t1);
    const float tv1[3] = {t1.x, t1.y, t1.z}, tv2[3] = {t2.x, t2.y, t2.z};
    // projected tangential gradient along t, and o_i.t, o_j.t in FP32 for the Hessian
    auto grad_t = [&](const float tv[3], float &uti, float &utj) -> float {
        const ff tn = ff_dot3_exact(tv, nv);
        const ff toi = ff_dot3f(oi, tv), toj = ff_dot3f(oj, tv);
        uti = toi.hi;
        utj = toj.hi;
        const ff gi = ff_mul(ff_add(ff_mul(a2i, tn), ff_mul(ei, ff_mul(ci, toi))), ri);
        const ff gj = ff_mul(ff_add(ff_mul(a2j, tn), ff_mul(ej, ff_mul(cj, toj))), rj);
        const ff G = ff_sub(ff_sub(ff_dot3f(d, tv), gi), gj);
        return __fadd_rn(__fsub_rn(G.hi, __fmul_rn(tn.hi, lam)), G.lo);
    };
    float u1i, u1j, u2i, u2j;
    const float G1 = grad_t(tv1, u1i, u1j), G2 = grad_t(tv2, u2i, u2j);
    // P = -Hess_t g in FP32 (as in newton_sphere)
    const float rif = ri.hi, rjf = rj.hi;
    const float Ai = a2i.hi * rif, Aj = a2j.hi * rjf;
    const float Ei = ei.hi * rif * rif, Ej = ej.hi * rjf * rjf;
    const float P11 = Ai * (1.f + Ei * u1i * u1i) + Aj * (1.f + Ej * u1j * u1j) + g.hi;
    const float P22 = Ai * (1.f + Ei * u2i * u2i) + Aj * (1.f + Ej * u2j * u2j) + g.hi;
    const float P12 = Ai * Ei * u1i * u2i + Aj * Ej * u1j * u2j;
    const float det = P11 * P22 - P12 * P12;
    float s1, s2;
    if (P11 > 0.f && det > 0.f) {
        const float idet = 1.0f / det;
        s1 = (P22 * G1 - P12 * G2) * idet;
        s2 = (P11 * G2 - P12 * G1) * idet;
    } else {
        const float sc = 1.0f / (fabsf(P11) + fabsf(P22) + fabsf(P12) + Ai + Aj);
        s1 = G1 * sc;
        s2 = G2 * sc;
    }
    // n + s1 t1 + s2 t2 in float-float (the step is of order 1e-7), normalised
    ff m[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) m[a] = two_sum(nv[a], __fmaf_rn(s1, tv1[a], __fmul_rn(s2, tv2[a])));
    const ff m2 = ff_add(ff_add(ff_mul(m[0], m[0]), ff_mul(m[1], m[1])), ff_mul(m[2], m[2]));
    const ff im = ff_rcp(ff_sqrt(m2));
    n64 = mk<double>(ff_to_double(ff_mul(m[0], im)), ff_to_double(ff_mul(m[1], im)), ff_to_double(ff_mul(m[2], im)));
    const float step = sqrtf(s1 * s1 + s2 * s2);
    const float nd = m[0].hi * d[0].hi + m[1].hi * d[1].hi + m[2].hi * d[2].hi;
    return (nd > 0.f && isfinite(step)) ? step : INFINITY;
}

// LUB_MIXED, refinement of a work-list pair: one float-float Newton step from
// the FP32 normal nn (the gap h_in of the FP32 stage stands: g is stationary
// in n, so the FP32 normal's error of ~1e-7 rad changes it by ~1e-14 of the
// sizes), or, if full, a complete FP64 solve and gap from the line of centres
template <bool ENS>
__device__ __forceinline__ void refine_one(const PView &P, const DView &D0, const Ens &E,
                                           const float2 *__restrict__ pff, int i, int j, bool full, V3<double> nn,
                                           double h_in, int st_in, int maxit, V3<double> &n64, double &h, int &st,
                                           int &nit)
{
    bool alien;
    const DView &D = pair_domain<ENS>(D0, E, i, j, &alien);
    if (!full) {
        const V3<float> n32 = mk<float>((float)nn.x, (float)nn.y, (float)nn.z);
        const bool converged = polish_ff(P, pff, D, i, j, n32, n64) < 1e-5f;
        nit = 1;
        h = h_in;
        st = st_in | LUB_ST_FP64;
        if (!converged) st |= LUB_ST_NOCONV;
        return;
    }
    const V3<double> d = min_image(D, sub(load_pos(P, j), load_pos(P, i)));
    const double dl = sqrt(dot(d, d));
    const Shape<double> si = load_shape<double>(P, i), sj = load_shape<double>(P, j);
    nn = scl(1.0 / dl, d);
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

// Compacted append to the work list (warp-collective).  One-step
// polishes (entry k) fill the list from the front, full solves (entry -1-k,
// several iterations each) from the back, so each kind runs in warps of its
// own instead of every warp waiting for one full solve.  wl_count[0]: front
// entries, wl_count[1]: back entries; the list holds cap entries.
__device__ __forceinline__ void worklist_append(int entry, int32_t *__restrict__ wl_count, int32_t *__restrict__ wl,
                                                int cap)
{
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const bool polish = entry != kNoEntry && entry >= 0, full = entry != kNoEntry && entry < 0;
    const unsigned mp = __ballot_sync(0xffffffffu, polish), mf = __ballot_sync(0xffffffffu, full);
    if (mp) {
        int wbase = 0;
        const int leader = __ffs(mp) - 1;
        if (lane == leader) wbase = atomicAdd(wl_count, __popc(mp));
        wbase = __shfl_sync(0xffffffffu, wbase, leader);
        if (polish) wl[wbase + __popc(mp & below)] = entry;
    }
    if (mf) {
        int wbase = 0;
        const int leader = __ffs(mf) - 1;
        if (lane == leader) wbase = atomicAdd(wl_count + 1, __popc(mf));
        wbase = __shfl_sync(0xffffffffu, wbase, leader);
        if (full) wl[cap - 1 - (wbase + __popc(mf & below))] = entry;
    }
}

// work-list entry q of [front entries | back entries], q < wl_total(...)
__device__ __forceinline__ int wl_total(const int32_t *__restrict__ wl_count, int cap)
{
    return min(wl_count[0] + wl_count[1], cap);
}
__device__ __forceinline__ int wl_entry(const int32_t *__restrict__ wl_count, const int32_t *__restrict__ wl, int cap,
                                        int q)
{
    const int nf = wl_count[0];
    return q < nf ? wl[q] : wl[cap - 1 - (q - nf)];
}

// ---------------------------------------------------------------------------
// lub_closest_points kernels
// ---------------------------------------------------------------------------
// float-float copies (hi, lo) of the particle positions, [3][n], for the
// separations of the FP32 stage
__global__ void __launch_bounds__(256) k_pos_ff(PView P, float2 *__restrict__ out)
{
    pdl_wait();
    pdl_trigger();
    const size_t N = (size_t)P.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        const double v[3] = {P.x[i], P.y[i], P.z[i]};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const ff p = ff_from_double(v[a]);
            out[a * N + i] = make_float2(p.hi, p.lo);
        }
    }
}

template <bool ENS>
__global__ void __launch_bounds__(128, 6) k_closest_mixed(PView P, const __grid_constant__ DView D0, Ens E,
                                                       const int32_t *__restrict__ pi, const int32_t *__restrict__ pj,
                                                       const int32_t *__restrict__ d_count, int32_t cap,
                                                       double *__restrict__ nout, double *__restrict__ gap,
                                                       uint8_t *__restrict__ status, uint8_t *__restrict__ iters,
                                                       int maxit, float tol32, float fp64_switch, int warm,
                                                       int32_t *__restrict__ wl_count, int32_t *__restrict__ wl,
                                                       const float2 *__restrict__ pff)
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
            int st, nit;
            entry = closest_mixed_one<ENS>(P, D0, E, pff, i, j, k, nout, C, warm, maxit, tol32, fp64_switch, n64, h, st,
                                           nit);
            store_pair(nout, gap, status, iters, C, k, n64, h, st, nit);
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
                                                        const int32_t *__restrict__ wl,
                                                        const float2 *__restrict__ pff)
{
    pdl_wait();
    pdl_trigger();
    const int count = wl_total(wl_count, cap);
    const size_t C = (size_t)cap;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < count; q += gridDim.x * blockDim.x) {
        const int v = wl_entry(wl_count, wl, cap, q);
        const bool full = v < 0;
        const int k = full ? -1 - v : v;
        V3<double> n64;
        double h;
        int st, nit;
        refine_one<ENS>(P, D0, E, pff, pi[k], pj[k], full, mk<double>(nout[k], nout[C + k], nout[2 * C + k]),
                        full ? 0.0 : gap[k], full ? 0 : status[k], maxit, n64, h, st, nit);
        store_pair(nout, gap, status, nullptr, C, k, n64, h, st, 0);
        if (iters) {
            const int total = (full ? 0 : iters[k]) + nit;
            iters[k] = (uint8_t)(total > 255 ? 255 : total);
        }
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
    uint8_t *__restrict__ status, uint8_t *__restrict__ iters, int maxit, float tol32, float fp64_switch,
    int32_t *__restrict__ wl_count, int32_t *__restrict__ wl, const float2 *__restrict__ pff, MlpDevice M)
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
            int st, nit;
            entry = closest_mixed_one<ENS>(P, D0, E, pff, __ldg(pi + k), __ldg(pj + k), k, nout, C, 1, maxit, tol32,
                                           fp64_switch, n64, h, st, nit);
            store_pair(nout, gap, status, iters, C, k, n64, h, st, nit);
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
                                                  T *__restrict__ torque)
{
    T out[12];
    T ci[6] = {0, 0, 0, 0, 0, 0}, cj[6] = {0, 0, 0, 0, 0, 0};
    if (done) {
        const V3<T> n = mk<T>((T)n64.x, (T)n64.y, (T)n64.z);
        pair_force<T>(P, R, i, j, n, h, st, out);
        store_force(FT, lever, C, k, out);
        side_contrib(out, 0, ci);
        if (j >= 0) side_contrib(out, 1, cj);
    }
    // the closest-point solve validated the indices of every pair without DEGENERATE
    const bool ok = done && !(st & LUB_ST_DEGENERATE);
    scatter_warp<T>(ok ? i : -1, ok ? j : -1, (size_t)P.n, ci, cj, force, torque);
}

// The fused pass in mixed precision after the FP32 stage (k_closest_mixed,
// which leaves every pair's normal, gap and status and marks the work-list
// pairs with LUB_ST_FP64): warps take 32 items at a time from two queues,
// the work-list entries (the refinement, then the pair's force and scatter),
// then the other pairs (force and scatter from the stored normal and gap).
// queue: two counters, zero at the launch.
template <bool ENS>
__global__ void __launch_bounds__(128) k_refine_resist(PView P, const __grid_constant__ DView D0, Ens E, RParams R,
                                                       const int32_t *__restrict__ pi, const int32_t *__restrict__ pj,
                                                       const int32_t *__restrict__ d_count, int32_t cap,
                                                       double *__restrict__ nout, double *__restrict__ gap,
                                                       uint8_t *__restrict__ status, uint8_t *__restrict__ iters,
                                                       float *__restrict__ FT, float *__restrict__ lever, int maxit,
                                                       const int32_t *__restrict__ wl_count,
                                                       const int32_t *__restrict__ wl, int32_t *__restrict__ queue,
                                                       float *__restrict__ force, float *__restrict__ torque,
                                                       const float2 *__restrict__ pff)
{
    pdl_wait();
    pdl_trigger();
    const int count = pair_count(d_count, cap), nwl = wl_total(wl_count, cap);
    const size_t C = (size_t)cap;
    const int lane = threadIdx.x & 31;
    // every warp takes work-list entries first (the refinement is FP32-pipe
    // work), then the other pairs
    for (;;) {
        int q0 = 0;
        if (lane == 0) q0 = atomicAdd(queue, 32);
        q0 = __shfl_sync(0xffffffffu, q0, 0);
        if (q0 >= nwl) break;
        const int q = q0 + lane;
        const bool active = q < nwl;
        int i = -1, j = -1, k = 0, st = 0, nit = 0;
        bool full = false;
        V3<double> n64 = mk<double>(0, 0, 0);
        double h = 0.0;
        if (active) {
            const int v = wl_entry(wl_count, wl, cap, q);
            full = v < 0;
            k = full ? -1 - v : v;
            i = pi[k];
            j = pj[k];
            refine_one<ENS>(P, D0, E, pff, i, j, full, mk<double>(nout[k], nout[C + k], nout[2 * C + k]),
                            full ? 0.0 : gap[k], full ? 0 : status[k], maxit, n64, h, st, nit);
        }
        force_and_scatter<float>(P, R, active, i, j, n64, h, st, FT, lever, C, k, force, torque);
        if (active) {
            store_pair(nout, gap, status, nullptr, C, k, n64, h, st, 0);
            if (iters) {
                const int total = (full ? 0 : iters[k]) + nit;
                iters[k] = (uint8_t)(total > 255 ? 255 : total);
            }
        }
    }
    for (;;) {
        int k0 = 0;
        if (lane == 0) k0 = atomicAdd(queue + 1, 32);
        k0 = __shfl_sync(0xffffffffu, k0, 0);
        if (k0 >= count) break;
        const int k = k0 + lane;
        int i = -1, j = -1, st = 0;
        bool done = k < count;
        V3<double> n64 = mk<double>(0, 0, 0);
        double h = 0.0;
        if (done) {
            st = status[k];
            if (st & LUB_ST_FP64) {
                done = false;  // a work-list pair: the first queue's
            } else {
                i = __ldg(pi + k);
                j = __ldg(pj + k);
                n64 = mk<double>(nout[k], nout[C + k], nout[2 * C + k]);
                h = gap[k];
            }
        }
        force_and_scatter<float>(P, R, done, i, j, n64, h, st, FT, lever, C, k, force, torque);
    }
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
        force_and_scatter<double>(P, R, k < count, i, j, n64, h, st, FT, lever, C, k, force, torque);
        if (k < count) store_pair(nout, gap, status, iters, C, k, n64, h, st, nit);
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// the network's start normals (learned warm start), then whether Newton starts from n
int start_normals(lub_ctx *ctx, const PView &P, const DView &D, const Ens &E, const lub_params &prm,
                  const int32_t *pi, const int32_t *pj, const int32_t *d_count, int32_t cap, double *n,
                  cudaStream_t st, int *warm)
{
    *warm = prm.warm_start == LUB_WARM_PREVIOUS;
    if (prm.warm_start == LUB_WARM_MLP) {
        int rc = launch_mlp_start(ctx, P, D, E, pi, pj, d_count, cap, n, nullptr, st);
        if (rc) return rc;
        *warm = 1;
    }
    return LUB_OK;
}

// The work list of the mixed mode in the context scratch: counters [front, back, queue 0,
// queue 1] and cap entries; with gap_in/status_in, also a gap and a status
// array for callers that pass none (the fused pass needs them between its
// kernels).
int work_list(lub_ctx *ctx, int32_t cap, cudaStream_t st, int32_t **wl_count, int32_t **wl,
              double **gap_in = nullptr, uint8_t **status_in = nullptr, const PView *P = nullptr,
              float2 **pff = nullptr)
{
    const size_t b_wl = ((4 * (size_t)cap + 255) / 256) * 256, b_gap = ((8 * (size_t)cap + 255) / 256) * 256,
                 b_st = (((size_t)cap + 255) / 256) * 256, b_pos = P ? 24 * (size_t)P->n : 0;
    int rc = lub_ensure_scratch(ctx, 256 + b_wl + b_gap + b_st + b_pos);
    if (rc) return rc;
    char *base = (char *)ctx->scratch;
    *wl_count = (int32_t *)base;
    *wl = (int32_t *)(base + 256);
    if (gap_in && !*gap_in) *gap_in = (double *)(base + 256 + b_wl);
    if (status_in && !*status_in) *status_in = (uint8_t *)(base + 256 + b_wl + b_gap);
    rc = zero_async(ctx, ctx->num_sms, *wl_count, 16, st);
    if (rc || !P) return rc;
    // the particles' float-float positions for the FP32 stage
    *pff = (float2 *)(base + 256 + b_wl + b_gap + b_st);
    if (P->n == 0) return LUB_OK;
    return lub_check_cuda(ctx, launch_pdl(k_pos_ff, grid_for(P->n, 256, ctx->num_sms, 8), 256, 0, st, *P, *pff),
                          "positions launch");
}

template <bool ENS>
int launch_closest_t(lub_ctx *ctx, const PView &P, const DView &D, const Ens &E, const lub_params &prm,
                     const int32_t *pi, const int32_t *pj, const int32_t *d_count, int32_t cap, double *n, double *gap,
                     uint8_t *status, uint8_t *iters, cudaStream_t st)
{
    int warm = 0, rc;
    // the learned start on the mma.sync engine runs inside the solve's kernel
    const bool fused_mlp = prm.warm_start == LUB_WARM_MLP && ctx->mlp_engine == LUB_MLP_MMA_SYNC;
    if (fused_mlp && !ctx->mlp_ready)
        return lub_set_error(ctx, LUB_ERR_ARG, "the learned warm start needs lub_mlp_set first");
    if (!fused_mlp && (rc = start_normals(ctx, P, D, E, prm, pi, pj, d_count, cap, n, st, &warm))) return rc;
    const int learned_grid = 2 * ctx->num_sms;
    if (prm.precision == LUB_MIXED) {
        int32_t *wl_count, *wl;
        float2 *pff = nullptr;
        if ((rc = work_list(ctx, cap, st, &wl_count, &wl, nullptr, nullptr, &P, &pff))) return rc;
        if (fused_mlp) {
            if ((rc = learned_smem(ctx, k_closest_mixed_learned<ENS>, 16 << ENS))) return rc;
            (void)launch_pdl(k_closest_mixed_learned<ENS>, learned_grid, 32 * INF_WARPS, sizeof(InfSmem), st, P, D, E,
                             pi, pj, d_count, cap, n, gap, status, iters, prm.max_newton, (float)prm.newton_tol,
                             (float)prm.fp64_switch, wl_count, wl, (const float2 *)pff, *(const MlpDevice *)ctx->mlp);
        } else {
            const Shape2 sh = tuned_shape(ctx, LUB_TUNE_CLOSEST_MIXED, cap);
            (void)launch_pdl(k_closest_mixed<ENS>, sh.grid, sh.block, 0, st, P, D, E, pi, pj, d_count, cap, n, gap,
                             status, iters, prm.max_newton, (float)prm.newton_tol, (float)prm.fp64_switch, warm,
                             wl_count, wl, (const float2 *)pff);
        }
        // small blocks so the (short) work list spreads over every SM
        const Shape2 sr = tuned_shape(ctx, LUB_TUNE_CLOSEST_REFINE, cap);
        (void)launch_pdl(k_closest_refine<ENS>, sr.grid, sr.block, 0, st, P, D, E, pi, pj, cap, n, gap, status, iters,
                         prm.max_newton, (const int32_t *)wl_count, (const int32_t *)wl, (const float2 *)pff);
    } else if (fused_mlp) {
        if ((rc = learned_smem(ctx, k_closest_fp64_learned<ENS>, 64 << ENS))) return rc;
        (void)launch_pdl(k_closest_fp64_learned<ENS>, learned_grid, 32 * INF_WARPS, sizeof(InfSmem), st, P, D, E, pi,
                         pj, d_count, cap, n, gap, status, iters, prm.max_newton, *(const MlpDevice *)ctx->mlp);
    } else {
        const Shape2 sh = tuned_shape(ctx, LUB_TUNE_CLOSEST_FP64, cap);
        (void)launch_pdl(k_closest_fp64<ENS>, sh.grid, sh.block, 0, st, P, D, E, pi, pj, d_count, cap, n, gap, status,
                         iters, prm.max_newton, warm);
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
    if (!accumulate) {
        if ((rc = zero_force_torque(ctx, force, torque, 3 * (size_t)P.n * esz, st))) return rc;
    }
    if (cap == 0) return LUB_OK;
    int warm = 0;
    if ((rc = start_normals(ctx, P, D, E, prm, pi, pj, d_count, cap, n, st, &warm))) return rc;
    const RParams R = make_rparams(prm);
    if (prm.precision == LUB_MIXED) {
        // the FP32 stage, then the work list's refinement and every pair's force
        // in one queue-driven launch (gap and status in the context when not given)
        int32_t *wl_count, *wl;
        float2 *pff = nullptr;
        if ((rc = work_list(ctx, cap, st, &wl_count, &wl, &gap, &status, &P, &pff))) return rc;
        const Shape2 sh = tuned_shape(ctx, LUB_TUNE_CLOSEST_MIXED, cap);
        (void)launch_pdl(k_closest_mixed<ENS>, sh.grid, sh.block, 0, st, P, D, E, pi, pj, d_count, cap, n, gap, status,
                         iters, prm.max_newton, (float)prm.newton_tol, (float)prm.fp64_switch, warm, wl_count, wl,
                         (const float2 *)pff);
        const Shape2 sr = tuned_shape(ctx, LUB_TUNE_RESISTANCE, cap);
        const int grid = sr.grid < 8 * ctx->num_sms ? sr.grid : 8 * ctx->num_sms;
        (void)launch_pdl(k_refine_resist<ENS>, grid, sr.block, 0, st, P, D, E, R, pi, pj, d_count, cap, n, gap, status,
                         iters, (float *)FT, (float *)lever, prm.max_newton, (const int32_t *)wl_count,
                         (const int32_t *)wl, wl_count + 2, (float *)force, (float *)torque, (const float2 *)pff);
    } else {
        const Shape2 sh = tuned_shape(ctx, LUB_TUNE_CLOSEST_FP64, cap);
        (void)launch_pdl(k_fused_fp64<ENS>, sh.grid, sh.block, 0, st, P, D, E, R, pi, pj, d_count, cap, n, gap, status, iters,
                                                       (double *)FT, (double *)lever, prm.max_newton, warm,
                                                       (double *)force, (double *)torque);
    }
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
