// Per-pair resistance and force scatter shared by the separate calls
// (lub_resistance, lub_apply) and the fused pass (lub_correct): the local
// geometry at the closest points, the resistance elements of the Appendix,
// K~, the contact branch and the lab-frame pair force (Sec. III B); and the
// warp-level scatter of pair forces and torques to the particles
// (Eq. lub:resistance).  See resistance.cu and apply.cu for the formulas.
#pragma once

#include "ff.cuh"
#include "lub_internal.cuh"

namespace {

// The per-call particle record of the mixed mode (pff, written by
// k_particles_ff): five float4 per particle, so that a kernel fetches a
// particle's data with four 16-byte loads from two or three sectors instead
// of a dozen scalar loads from as many arrays:
//   [0] x.hi x.lo y.hi y.lo    [1] z.hi z.lo r_par r_perp
//   [2] ox.hi ox.lo oy.hi oy.lo [3] oz.hi oz.lo vx vy    [4] vz wx wy wz
// (float-float centre and symmetry axis, semi-axes, velocities).
constexpr int kRec = 5;
__device__ __forceinline__ float4 rec_ld(const float2 *__restrict__ pff, int k, int q)
{
    return __ldg(reinterpret_cast<const float4 *>(pff) + (size_t)k * kRec + q);
}

// the float-float symmetry axis from records 2 and 3
__device__ __forceinline__ void ff_axis_rec(const float4 &r2, const float4 &r3, ff o[3])
{
    o[0] = ff{r2.x, r2.y};
    o[1] = ff{r2.z, r2.w};
    o[2] = ff{r3.x, r3.y};
}

// FP32 shape with the axis rounded from its float-float value
__device__ __forceinline__ Shape<float> shape_ff(const ff o[3], float rpar, float rperp)
{
    Shape<float> s;
    s.o = mk<float>(o[0].hi, o[1].hi, o[2].hi);
    s.rpar = rpar;
    s.rperp = rperp;
    s.a2 = rperp * rperp;
    s.e = rpar * rpar - s.a2;
    return s;
}

// n.(w x rho) for the support offset rho = +-M n / sigma(n) of a spheroid (+
// for i at n, - for j at -n), without its sign: M n = a2 n + e (o.n) o and
// n.(w x n) = 0, so only k n.(w x o) with k = e (o.n) / sigma(n) remains.
// Float-float, for a unit float-float n, the float-float axis o and the
// (exact) float angular velocity w; zero for a sphere (e = 0).
__device__ __forceinline__ ff rot_normal_ff(const ff n[3], const ff o[3], float rpar, float rperp, float wx, float wy,
                                            float wz)
{
    if (rpar == rperp) return ff_make(0.0f);
    const ff a2 = two_prod(rperp, rperp), e = ff_sub(two_prod(rpar, rpar), a2);
    const ff c = ff_dot3_c(o, n);
    const ff k = ff_mul(ff_mul(e, c), ff_rsqrt(ff_add(a2, ff_mul(e, ff_mul(c, c)))));
    // w x o, each component compensated (w is exact)
    const ff wo[3] = {ff_cross_comp_f(wy, o[2], wz, o[1]), ff_cross_comp_f(wz, o[0], wx, o[2]),
                      ff_cross_comp_f(wx, o[1], wy, o[0])};
    return ff_mul(k, ff_dot3_c(n, wo));
}

// The normal relative surface velocity u3 = n.(V_j - V_i), V = v + w x (y* - r)
// (Sec. III B), in float-float.  It is a difference of terms of the size of
// the velocities and nearly cancels for some pairs, where the force bound
// relative to it asks for more than FP32: with rho_i = M_i n / sigma_i,
// rho_j = -M_j n / sigma_j,
//   u3 = n.(v_j - v_i) - k_i n.(w_i x o_i) - k_j n.(w_j x o_j),
// v_j - v_i exact (TwoSum), the rest in float-float.  j < 0: a wall at rest.
// (shapes, velocities and angular velocities as floats; j < 0: a wall at rest)
__device__ __forceinline__ float normal_velocity_ff(const ff n[3], const ff oi[3], float rpi, float rqi,
                                                    const V3<float> &vi, const V3<float> &wi, int j, const ff oj[3],
                                                    float rpj, float rqj, const V3<float> &vj, const V3<float> &wj)
{
    ff u = ff_make(0.0f);
    V3<float> vjj = mk<float>(0.f, 0.f, 0.f);
    if (j >= 0) {
        vjj = vj;
        u = ff_neg(rot_normal_ff(n, oj, rpj, rqj, wj.x, wj.y, wj.z));
    }
    const ff dv[3] = {two_sum(vjj.x, -vi.x), two_sum(vjj.y, -vi.y), two_sum(vjj.z, -vi.z)};
    u = ff_add(u, ff_dot3_c(n, dv));
    u = ff_sub(u, rot_normal_ff(n, oi, rpi, rqi, wi.x, wi.y, wi.z));
    return __fadd_rn(u.hi, u.lo);
}

template <typename T>
struct Surf {
    V3<T> x1;
    T c1, c2, G0, G2;
};

__device__ __forceinline__ float log1p_t(float x) { return log1pf(x); }
__device__ __forceinline__ double log1p_t(double x) { return log1p(x); }

// Local geometry at surface offset rho = y* - r with outward normal nrm.
template <typename T>
__device__ __forceinline__ Surf<T> surface_at(const Shape<T> &s, const V3<T> &rho, const V3<T> &nrm)
{
    Surf<T> o;
    const T ipar = rcp_fast(s.rpar), iperp = rcp_fast(s.rperp);
    const T zt = dot(rho, s.o);
    const V3<T> rp = axpy(-zt, s.o, rho);  // component normal to the axis
    const T rr2 = dot(rp, rp);
    const T spr = zt * ipar;                         // sin p, unnormalised
    const T cpr = sqrt_fast(rr2) * iperp;            // cos p, unnormalised
    const T hn = rsqrt_t(spr * spr + cpr * cpr);
    const T sp = spr * hn, cp = cpr * hn;
    V3<T> er;
    if (rr2 > T(1e-24) * s.a2) {
        er = scl(rsqrt_t(rr2), rp);
    } else {  // pole: any direction normal to the axis (umbilic point)
        V3<T> e = (fabs((double)s.o.x) < 0.6) ? mk<T>(1, 0, 0) : mk<T>(0, 1, 0);
        er = normalized(axpy(-dot(e, s.o), s.o, e));
    }
    // d y~/dp = -R_perp sin p e_r + R_par cos p o
    V3<T> s1v = axpy(-s.rperp * sp, er, scl(s.rpar * cp, s.o));
    o.x1 = normalized(axpy(-dot(s1v, nrm), nrm, s1v));
    const T s1sq = s.rperp * s.rperp * sp * sp + s.rpar * s.rpar * cp * cp;
    const T is1 = rsqrt_t(s1sq);
    const T is2 = is1 * is1;
    o.c1 = s.rpar * s.rperp * is1 * is2;            // 1/S1 = R_par R_perp / s1^3
    o.c2 = s.rpar * iperp * is1;                    // 1/S2 = R_par / (R_perp s1)
    const T kk = T(0.5) * s.e * sp * cp;            // (R_par^2 - R_perp^2) sin p cos p / 2
    o.G0 = kk * s.rpar * s.rperp * is2 * is2 * is2;  // / s1^6
    o.G2 = kk * s.rpar * iperp * is2 * is2;         // / (R_perp s1^4)
    return o;
}

// The gap's terms at the element cut-offs (Eq. lub:resistance-correction) in
// the arithmetic of T: he = h, or h_c where the contact model clips a
// smaller gap; d_x = he - Delta_x for the three cut-offs, which cancels near
// each cut-off; in_x = he < Delta_x; fr = h_c - h where the contact force
// acts (h <= h_c with h_c > 0), else 0; le0 = h <= 0.  T = double: double
// arithmetic.  T = float: from a float-float gap (the fused pass hands it
// over as such; a double gap is split with integer operations, no FP64-pipe
// work), the differences in float-float, so d_x keeps its relative accuracy
// near the cut-off.
template <typename T>
struct CutTerms {
    T he, dn, dt, dr, fr;
    bool in_n, in_t, in_r, contact, le0;
};

__device__ __forceinline__ CutTerms<double> cut_terms(const RParams &R, double h, double)
{
    CutTerms<double> c;
    c.he = (R.contact && h < R.h_c) ? R.h_c : h;
    c.dn = c.he - R.delta_n;
    c.dt = c.he - R.delta_t;
    c.dr = c.he - R.delta_r;
    c.in_n = c.he < R.delta_n;
    c.in_t = c.he < R.delta_t;
    c.in_r = c.he < R.delta_r;
    c.contact = R.contact && h <= R.h_c;
    c.fr = c.contact ? (h > 0.0 ? R.h_c - h : R.h_c) : 0.0;
    c.le0 = h <= 0.0;
    return c;
}

__device__ __forceinline__ CutTerms<float> cut_terms_ff(const RParams &R, ff he)
{
    CutTerms<float> c;
    c.le0 = he.hi <= 0.f;
    const float hi = he.hi;
    const ff hc{R.hc_ff[0], R.hc_ff[1]};
    const ff dc = ff_sub(he, hc);
    const float dcf = dc.hi + dc.lo;  // h - h_c
    c.contact = R.contact && dcf <= 0.f;
    if (R.contact && dcf < 0.f) he = hc;
    c.he = he.hi + he.lo;
    const ff dn = ff_sub(he, ff{R.dn_ff[0], R.dn_ff[1]}), dt = ff_sub(he, ff{R.dt_ff[0], R.dt_ff[1]}),
             dr = ff_sub(he, ff{R.dr_ff[0], R.dr_ff[1]});
    c.dn = dn.hi + dn.lo;
    c.dt = dt.hi + dt.lo;
    c.dr = dr.hi + dr.lo;
    c.in_n = c.dn < 0.f;
    c.in_t = c.dt < 0.f;
    c.in_r = c.dr < 0.f;
    c.fr = c.contact ? (hi > 0.f ? -dcf : R.hc_ff[0]) : 0.f;
    return c;
}

// Appendix: coefficients m_0..m_3 of a cubic given in a frame rotated by
// alpha (cos c, sin s), in the unrotated frame.
template <typename T>
__device__ __forceinline__ void m_rot(T c, T s, T a0, T a1, T a2, T a3, T m[4])
{
    const T c2 = c * c, s2 = s * s;
    m[0] = a0 * c2 * c - a1 * s * c2 + a2 * s2 * c - a3 * s2 * s;
    m[1] = T(3) * a0 * s * c2 + a1 * (c2 * c - T(2) * s2 * c) + a2 * (s2 * s - T(2) * s * c2) + T(3) * a3 * s2 * c;
    m[2] = T(3) * a0 * c * s2 + a1 * (T(2) * c2 * s - s2 * s) + a2 * (c2 * c - T(2) * c * s2) - T(3) * a3 * c2 * s;
    m[3] = a0 * s2 * s + a1 * c * s2 + a2 * c2 * s + a3 * c2 * c;
}

// The normal (x3), the shapes and the velocities of a pair's particles in the
// arithmetic of T, and (mixed mode) the normal relative surface velocity u3
// formed in float-float; FP64 mode forms u3 with the rest.
template <typename T>
struct PairKin {
    V3<T> n, vi, Wi, vj, Wj;
    Shape<T> si, sj;
    T u3;
};

template <typename T>
__device__ __forceinline__ void pair_force_body(const RParams &R, int j, const CutTerms<T> &cut, const PairKin<T> &K,
                                                T out[12]);

// Force and torque on i (lab frame, torque about y*_i) and the lever arms of
// one pair, mixed mode, from its unit normal nf (direction of h, outward
// from i) and gap hf in float-float: out = (F_i, T_i, y*_i - r_i, y*_j -
// r_j).  st carries the pair's status bits in and gains OVERLAP when h <= 0
// without a contact model; pairs with NOCONV or DEGENERATE (or such an
// overlap) give zeros.  Needs the per-call particle records pff (rec_ld):
// the frames, curvatures and K~ run in FP32 with the axes rounded from it,
// the normal relative velocity u3 in float-float (normal_velocity_ff), and
// no step uses the FP64 pipe.  The local relative velocities u come first
// and each group of K~ elements is applied to them as soon as it is formed,
// which keeps few values live at a time.
__device__ __forceinline__ void pair_force_ff(const RParams &R, int i, int j, const ff nf[3], ff hf, int &st,
                                              float out[12], const float2 *__restrict__ pff)
{
#pragma unroll
    for (int a = 0; a < 12; ++a) out[a] = 0.f;
    if (st & (LUB_ST_NOCONV | LUB_ST_DEGENERATE)) return;
    const CutTerms<float> cut = cut_terms_ff(R, hf);
    if (!R.contact && cut.le0) {
        st |= LUB_ST_OVERLAP;
        return;
    }
    PairKin<float> K;
    ff oi[3], oj[3];
    K.n = mk<float>(nf[0].hi, nf[1].hi, nf[2].hi);
    const float4 a1 = rec_ld(pff, i, 1), a2 = rec_ld(pff, i, 2), a3 = rec_ld(pff, i, 3), a4 = rec_ld(pff, i, 4);
    ff_axis_rec(a2, a3, oi);
    K.si = shape_ff(oi, a1.z, a1.w);
    K.vi = mk<float>(a3.z, a3.w, a4.x);
    K.Wi = mk<float>(a4.y, a4.z, a4.w);
    K.sj = {};
    K.vj = K.Wj = mk<float>(0.f, 0.f, 0.f);
    if (j >= 0) {
        const float4 b1 = rec_ld(pff, j, 1), b2 = rec_ld(pff, j, 2), b3 = rec_ld(pff, j, 3), b4 = rec_ld(pff, j, 4);
        ff_axis_rec(b2, b3, oj);
        K.sj = shape_ff(oj, b1.z, b1.w);
        K.vj = mk<float>(b3.z, b3.w, b4.x);
        K.Wj = mk<float>(b4.y, b4.z, b4.w);
    }
    K.u3 = normal_velocity_ff(nf, oi, K.si.rpar, K.si.rperp, K.vi, K.Wi, j, oj, K.sj.rpar, K.sj.rperp, K.vj, K.Wj);
    pair_force_body<float>(R, j, cut, K, out);
}

// The same from a double normal n64 and gap h: T = float splits them into
// float-float (integer operations) for pair_force_ff; T = double is the FP64
// mode (pff unused).
template <typename T>
__device__ __forceinline__ void pair_force(const PView &P, const RParams &R, int i, int j, const V3<double> &n64,
                                           double h, int &st, T out[12], const float2 *__restrict__ pff)
{
    if constexpr (sizeof(T) == 4) {
        const ff nf[3] = {ff_split_bits(n64.x), ff_split_bits(n64.y), ff_split_bits(n64.z)};
        pair_force_ff(R, i, j, nf, ff_split_bits(h), st, out, pff);
    } else {
#pragma unroll
        for (int a = 0; a < 12; ++a) out[a] = 0.0;
        if (st & (LUB_ST_NOCONV | LUB_ST_DEGENERATE)) return;
        const CutTerms<double> cut = cut_terms(R, h, 0.0);
        if (!R.contact && cut.le0) {
            st |= LUB_ST_OVERLAP;
            return;
        }
        PairKin<double> K;
        K.n = n64;
        K.si = load_shape<double>(P, i);
        K.vi = mk<double>(__ldg(P.vx + i), __ldg(P.vy + i), __ldg(P.vz + i));
        K.Wi = mk<double>(__ldg(P.wx + i), __ldg(P.wy + i), __ldg(P.wz + i));
        K.sj = {};
        K.vj = K.Wj = mk<double>(0.0, 0.0, 0.0);
        if (j >= 0) {
            K.sj = load_shape<double>(P, j);
            K.vj = mk<double>(__ldg(P.vx + j), __ldg(P.vy + j), __ldg(P.vz + j));
            K.Wj = mk<double>(__ldg(P.wx + j), __ldg(P.wy + j), __ldg(P.wz + j));
        }
        K.u3 = 0.0;
        pair_force_body<double>(R, j, cut, K, out);
    }
}

// the geometry at both contact points, K~ and the lab-frame force and torque
// (out must hold zeros on entry)
template <typename T>
__device__ __forceinline__ void pair_force_body(const RParams &R, int j, const CutTerms<T> &cut, const PairKin<T> &K,
                                                T out[12])
{
    constexpr bool MIXED = sizeof(T) == 4;
    const V3<T> n = K.n, vi = K.vi, Wi = K.Wi, vj = K.vj, Wj = K.Wj;
    const Shape<T> &si = K.si, &sj = K.sj;
    T u3 = K.u3;
    // geometry at y*_i, the local frame x1, x2, x3 = n, and the relative velocities
    const V3<T> rho_i = support_offset(si, n);
    const Surf<T> A = surface_at(si, rho_i, n);
    const V3<T> x1 = A.x1, x2 = cross(n, x1);
    V3<T> dV = scl(T(-1), add(vi, cross(Wi, rho_i)));
    V3<T> dW = scl(T(-1), Wi);
    T c1p = 0, c2p = 0, G0p = 0, G2p = 0, cf = 1, sf = 0;
    V3<T> rho_j = mk<T>(0, 0, 0);
    if (j >= 0) {
        rho_j = scl(T(-1), support_offset(sj, n));
        const Surf<T> B = surface_at(sj, rho_j, scl(T(-1), n));
        c1p = B.c1;
        c2p = B.c2;
        G0p = B.G0;
        G2p = B.G2;
        cf = dot(B.x1, x1);
        sf = dot(B.x1, x2);
        const T r = rsqrt_t(cf * cf + sf * sf);
        cf *= r;
        sf *= r;
        dV = add(dV, add(vj, cross(Wj, rho_j)));
        dW = add(dW, Wj);
    }
    const T u1 = dot(x1, dV), u2 = dot(x2, dV);
    if constexpr (!MIXED) u3 = dot(n, dV);
    const T u4 = dot(x1, dW), u5 = dot(x2, dW), u6 = dot(n, dW);
    out[6] = rho_i.x; out[7] = rho_i.y; out[8] = rho_i.z;
    out[9] = rho_j.x; out[10] = rho_j.y; out[11] = rho_j.z;
    // combined-gap matrix and its eigen-decomposition (Appendix)
    const T A11 = T(0.5) * (A.c1 + cf * cf * c1p + sf * sf * c2p);
    const T A12 = T(0.5) * sf * cf * (c1p - c2p);
    const T A22 = T(0.5) * (A.c2 + sf * sf * c1p + cf * cf * c2p);
    const T hd = T(0.5) * (A11 - A22);
    const T rad = sqrt_fast(hd * hd + A12 * A12);
    const T l1 = T(0.5) * (A11 + A22) + rad;
    const T il1 = rcp_fast(l1);
    const T l2 = (A11 * A22 - A12 * A12) * il1;
    const T il2 = rcp_fast(l2);
    const T mu = MIXED ? (T)R.mu_f : (T)R.mu;
    const T PI = T(3.14159265358979323846);
    const T r1 = sqrt_fast(l1), r2 = sqrt_fast(l2);
    const T isq = rcp_fast(r1 * r2);
    const T il12 = rcp_fast(l1 + l2);
    const T H33 = T(3) * PI * isq * il12;
    const T hq = cut.in_n ? -cut.dn * rcp_fast(cut.he) * (MIXED ? (T)R.idn_f : rcp_fast((T)R.delta_n)) : T(0);
    T F1 = 0, F2 = 0, F3 = hq * H33 * u3, T4 = 0, T5 = 0, T6 = 0;
    if (R.model != LUB_MODEL_NORMAL) {
        T v0 = A12, v1 = l2 - A11;
        const T w0 = l2 - A22, w1 = A12;
        if (w0 * w0 + w1 * w1 > v0 * v0 + v1 * v1) {
            v0 = w0;
            v1 = w1;
        }
        T sx, cx;
        const T vn = v0 * v0 + v1 * v1;
        if (vn > T(0)) {
            const T r = rsqrt_t(vn);
            sx = v0 * r;
            cx = v1 * r;
        } else {
            sx = 0;
            cx = 1;
        }
        const T lt = cut.in_t ? log1p_t(cut.dt * (MIXED ? (T)R.idt_f : rcp_fast((T)R.delta_t))) : T(0);
        const T lr = cut.in_r ? log1p_t(cut.dr * (MIXED ? (T)R.idr_f : rcp_fast((T)R.delta_r))) : T(0);
        // K: ln h coefficients (Appendix, (1 - lambda S)/S = c - lambda)
        const T iD1 = rcp_fast((T(3) * l1 + T(2) * l2) * l1);
        const T iD2 = rcp_fast((T(2) * l1 + T(3) * l2) * l2);
        const T c2x = cx * cx, s2x = sx * sx, scx = sx * cx;
        const T c1 = A.c1, c2 = A.c2;
        const T a1 = c1 - l1, a2 = c1 - l2, b1 = c2 - l1, b2 = c2 - l2;
        const T p3 = T(3) * PI * isq;
        {  // translation-translation
            const T L11 = -PI * isq * (T(3) * c2x * a1 * a1 * iD1 + T(3) * s2x * a2 * a2 * iD2 + T(1));
            const T L12 = p3 * scx * (a1 * b1 * iD1 - a2 * b2 * iD2);
            const T L22 = -PI * isq * (T(3) * s2x * b1 * b1 * iD1 + T(3) * c2x * b2 * b2 * iD2 + T(1));
            F1 += lt * (L11 * u1 + L12 * u2);
            F2 += lt * (L12 * u1 + L22 * u2);
        }
        {  // translation-rotation
            const T L14 = p3 * scx * (a1 * iD1 - a2 * iD2);
            const T L15 = p3 * (c2x * a1 * iD1 + s2x * a2 * iD2);
            const T L24 = -p3 * (s2x * b1 * iD1 + c2x * b2 * iD2);
            const T L25 = p3 * scx * (-b1 * iD1 + b2 * iD2);
            F1 += lt * (L14 * u4 + L15 * u5);
            F2 += lt * (L24 * u4 + L25 * u5);
            T4 += lt * (L14 * u1 + L24 * u2);
            T5 += lt * (L15 * u1 + L25 * u2);
        }
        {  // rotation-rotation
            const T L44 = -p3 * (s2x * iD1 + c2x * iD2);
            const T L45 = p3 * scx * (-iD1 + iD2);
            const T L55 = -p3 * (c2x * iD1 + s2x * iD2);
            T4 += lr * (L44 * u4 + L45 * u5);
            T5 += lr * (L45 * u4 + L55 * u5);
        }
        {  // normal-twist coupling
            const T L36 = T(-1.5) * PI * isq * il12 * scx * (c1 - c2) * (il1 - il2);
            F3 += lt * L36 * u6;
            T6 += lt * L36 * u3;
        }
        {  // cubic couplings K13, K23, K34, K35 (Gamma_1 = Gamma_3 = 0)
            T beta[4], kap[4];
            m_rot<T>(cf, sf, G0p, T(0), G2p, T(0), beta);
            m_rot<T>(cx, sx, A.G0 + beta[0], beta[1], A.G2 + beta[2], beta[3], kap);
            const T ir1 = rcp_fast(r1), ir2 = rcp_fast(r2);
            kap[0] *= ir1 * ir1 * ir1;
            kap[1] *= ir1 * ir1 * ir2;
            kap[2] *= ir1 * ir2 * ir2;
            kap[3] *= ir2 * ir2 * ir2;
            const T i3 = rcp_fast(T(3) * l1 + T(2) * l2), i2 = rcp_fast(T(2) * l1 + T(3) * l2);
            const T Q0 = T(3) * kap[0] * l1 + kap[2] * l2;  // 3 k0 l1 + k2 l2
            const T Q1 = kap[1] * l1 + T(3) * kap[3] * l2;  // k1 l1 + 3 k3 l2
            const T Sa = (T(7) * l1 + T(2) * l2) * kap[0] + (l1 + T(2) * l2) * kap[2];
            const T Sb = (T(2) * l1 + l2) * kap[1] + (T(2) * l1 + T(7) * l2) * kap[3];
            const T pre13 = T(-1.5) * PI * isq * il12;
            const T L13 = pre13 * ((T(2) * r1 * Q0 - T(1.5) * c1 * ir1 * Sa) * cx * i3 +
                                   (T(2) * r2 * Q1 - T(1.5) * c1 * ir2 * Sb) * sx * i2 +
                                   T(3) * A.G0 * (c2x * il1 + s2x * il2) + A.G2 * (s2x * il1 + c2x * il2));
            const T L23 = pre13 * ((T(-2) * r1 * Q0 + T(1.5) * c2 * ir1 * Sa) * sx * i3 +
                                   (T(2) * r2 * Q1 - T(1.5) * c2 * ir2 * Sb) * cx * i2 +
                                   T(2) * A.G2 * scx * (il2 - il1));
            const T pre34 = T(2.25) * PI * isq * il12;
            const T Bq = Sb * ir2 * i2, Aq = Sa * ir1 * i3;
            const T L34 = pre34 * (Bq * cx - Aq * sx);
            const T L35 = -pre34 * (Aq * cx + Bq * sx);
            F1 += lt * L13 * u3;
            F2 += lt * L23 * u3;
            F3 += lt * (L13 * u1 + L23 * u2 + L34 * u4 + L35 * u5);
            T4 += lt * L34 * u3;
            T5 += lt * L35 * u3;
        }
    }
    F1 *= mu;
    F2 *= mu;
    F3 *= mu;
    if (cut.contact) F3 -= (MIXED ? (T)R.eps_f : (T)R.eps_c) * cut.fr;
    const V3<T> F = axpy(F1, x1, axpy(F2, x2, scl(F3, n)));
    const V3<T> Tq = scl(mu, axpy(T4, x1, axpy(T5, x2, scl(T6, n))));
    out[0] = F.x; out[1] = F.y; out[2] = F.z;
    out[3] = Tq.x; out[4] = Tq.y; out[5] = Tq.z;
}

// contribution of a pair to particle i (side 0) or j (side 1) from
// out = (F_i, T_i, lever_i, lever_j): +-(F, T + lever x F)
template <typename T>
__device__ __forceinline__ void side_contrib(const T out[12], int side, T c[6])
{
    const V3<T> F = mk<T>(out[0], out[1], out[2]);
    const V3<T> Tq = mk<T>(out[3], out[4], out[5]);
    const V3<T> l = side ? mk<T>(out[9], out[10], out[11]) : mk<T>(out[6], out[7], out[8]);
    const V3<T> t = add(Tq, cross(l, F));
    const T sg = side ? T(-1) : T(1);
    c[0] = sg * F.x; c[1] = sg * F.y; c[2] = sg * F.z;
    c[3] = sg * t.x; c[4] = sg * t.y; c[5] = sg * t.z;
}

// Warp-collective (every lane of the warp calls it): atomic adds of the i-
// and j-side contributions ci, cj to force/torque [3][n].  Lanes with i < 0
// add nothing, lanes with j < 0 (walls) add no j side.  The i sides of a run
// of lanes with equal i (pairs sorted by i) are summed first by a segmented
// warp scan (runs are told apart by their index among the warp's runs, so
// that equal i in two separate runs never mix; the shuffle steps stop at the
// warp's longest run, where every further step would add nothing), and the
// run's last lane makes one atomic add.
template <typename T>
__device__ __forceinline__ void scatter_warp(int i, int j, size_t N, T ci[6], const T cj[6], T *__restrict__ force,
                                             T *__restrict__ torque)
{
    const int lane = threadIdx.x & 31;
    const int iprev = __shfl_up_sync(0xffffffffu, i, 1), inext = __shfl_down_sync(0xffffffffu, i, 1);
    const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || i != iprev);
    const unsigned upto = heads & (0xffffffffu >> (31 - lane));
    const int run = __popc(upto);  // runs started at or before this lane
    // the longest run of the warp, less one (the lane's offset in its run)
    const int span = (int)__reduce_max_sync(0xffffffffu, (unsigned)(lane - (31 - __clz(upto))));
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        if (off > span) break;  // the same for every lane
        const int rup = __shfl_up_sync(0xffffffffu, run, off);
        const bool same = lane >= off && rup == run;
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            const T y = __shfl_up_sync(0xffffffffu, ci[a], off);
            if (same) ci[a] += y;
        }
    }
    const bool tail = lane == 31 || inext != i;
    if (i >= 0 && tail) {
        atomicAdd(force + i, ci[0]);
        atomicAdd(force + N + i, ci[1]);
        atomicAdd(force + 2 * N + i, ci[2]);
        atomicAdd(torque + i, ci[3]);
        atomicAdd(torque + N + i, ci[4]);
        atomicAdd(torque + 2 * N + i, ci[5]);
    }
    if (i >= 0 && j >= 0) {
        atomicAdd(force + j, cj[0]);
        atomicAdd(force + N + j, cj[1]);
        atomicAdd(force + 2 * N + j, cj[2]);
        atomicAdd(torque + j, cj[3]);
        atomicAdd(torque + N + j, cj[4]);
        atomicAdd(torque + 2 * N + j, cj[5]);
    }
}

}  // namespace
