// K2: fused local geometry + resistance + pair force (Sec. III B, Appendix).
//
// Per pair, from the normal n and gap h of K1:
//   y*_i - r_i = M_i n / sigma_i(n),  y*_j - r_j = -M_j n / sigma_j(n)
//   principal direction x1 along d y~/dp and curvatures c = 1/S of
//   Eqs. lub:curvature-directions / lub:curvature-radii, cubic coefficients
//   Gamma_0, Gamma_2 (Sec. III B), at both points (walls: c = Gamma = 0)
//   cos/sin of phi from x1' = cos(phi) x1 + sin(phi) x2 (x2 = x3 x x1)
//   combined-gap matrix, eigenvalues lambda_1 >= lambda_2, l2 = (sin chi, cos chi)
//   beta = m(phi, Gamma'), k = Gamma + beta, kappa_i = m_i(chi, k) / (sqrt(l1)^(3-i) sqrt(l2)^i)
//   the 16 elements of K (ln h and 1/h coefficients), K~ with Delta_n, Delta_t, Delta_r
//   clip h_eff = max(h, h_c), Hookean repulsion F_r along -x3 (Eqs. lub:frep, lub:model)
//   u = (x_a.(V_j - V_i), x_a.(w_j - w_i)), V = v + w x (y* - r)
//   (Fb, Tb) = mu K~ u, F_i = sum Fb_a x_a, T_i = sum Tb_a x_a.
// No trigonometric functions: cos/sin of phi and chi come from dot products
// and the eigenvector.  The log terms are computed as log1p((h - Delta)/Delta)
// with h - Delta taken in double, so K~ keeps its relative accuracy up to the
// cut-off.  One thread per pair.
#include "lub_internal.cuh"

namespace {

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
    const T zt = dot(rho, s.o);
    const V3<T> rp = axpy(-zt, s.o, rho);  // component normal to the axis
    const T rr2 = dot(rp, rp);
    const T spr = zt / s.rpar;                       // sin p, unnormalised
    const T cpr = sqrt_t(rr2) / s.rperp;             // cos p, unnormalised
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
    o.c2 = s.rpar / s.rperp * is1;                  // 1/S2 = R_par / (R_perp s1)
    const T kk = T(0.5) * s.e * sp * cp;            // (R_par^2 - R_perp^2) sin p cos p / 2
    o.G0 = kk * s.rpar * s.rperp * is2 * is2 * is2;  // / s1^6
    o.G2 = kk * s.rpar / s.rperp * is2 * is2;       // / (R_perp s1^4)
    return o;
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

template <typename T, bool ENS>
__global__ void __launch_bounds__(128) k_resistance(PView P, const __grid_constant__ DView D0, Ens E, RParams R, const int32_t *__restrict__ pi,
                                                    const int32_t *__restrict__ pj,
                                                    const int32_t *__restrict__ d_count, int32_t cap,
                                                    const double *__restrict__ nin, const double *__restrict__ gap,
                                                    uint8_t *__restrict__ status, T *__restrict__ FT,
                                                    T *__restrict__ lever)
{
    const int count = pair_count(d_count, cap);
    const size_t C = (size_t)cap;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
        int st = status[k];
        const double h = gap[k];
        const int i = __ldg(pi + k), j = __ldg(pj + k);
        T out[12];
#pragma unroll
        for (int a = 0; a < 12; ++a) out[a] = T(0);
        // indices are checked here too: status may not come from lub_closest_points
        bool alien;
        const DView &D = pair_domain<ENS>(D0, E, i, j, &alien);
        if (alien || i < 0 || i >= P.n || j >= P.n || j < -D.n_walls || j == i) st |= LUB_ST_DEGENERATE;
        bool skip = (st & (LUB_ST_NOCONV | LUB_ST_DEGENERATE)) != 0;
        if (!skip && R.h_c <= 0.0 && h <= 0.0) {
            st |= LUB_ST_OVERLAP;
            skip = true;
        }
        if (!skip) {
            const double he = (R.h_c > 0.0 && h < R.h_c) ? R.h_c : h;
            const V3<T> n = mk<T>((T)nin[k], (T)nin[C + k], (T)nin[2 * C + k]);
            const Shape<T> si = load_shape<T>(P, i);
            const V3<T> rho_i = support_offset(si, n);
            const Surf<T> A = surface_at(si, rho_i, n);
            const V3<T> x1 = A.x1, x3 = n, x2 = cross(x3, x1);
            T c1p = 0, c2p = 0, G0p = 0, G2p = 0, cf = 1, sf = 0;
            V3<T> rho_j = mk<T>(0, 0, 0);
            V3<T> Vj = mk<T>(0, 0, 0), Wj = mk<T>(0, 0, 0);
            if (j >= 0) {
                const Shape<T> sj = load_shape<T>(P, j);
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
                const V3<T> vj = mk<T>(__ldg(P.vx + j), __ldg(P.vy + j), __ldg(P.vz + j));
                Wj = mk<T>(__ldg(P.wx + j), __ldg(P.wy + j), __ldg(P.wz + j));
                Vj = add(vj, cross(Wj, rho_j));
            }
            // combined-gap matrix and its eigen-decomposition (Appendix)
            const T A11 = T(0.5) * (A.c1 + cf * cf * c1p + sf * sf * c2p);
            const T A12 = T(0.5) * sf * cf * (c1p - c2p);
            const T A22 = T(0.5) * (A.c2 + sf * sf * c1p + cf * cf * c2p);
            const T hd = T(0.5) * (A11 - A22);
            const T rad = sqrt_t(hd * hd + A12 * A12);
            const T l1 = T(0.5) * (A11 + A22) + rad;
            const T l2 = (A11 * A22 - A12 * A12) / l1;
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
            // cubic terms
            T beta[4], kap[4];
            m_rot<T>(cf, sf, G0p, T(0), G2p, T(0), beta);
            m_rot<T>(cx, sx, A.G0 + beta[0], beta[1], A.G2 + beta[2], beta[3], kap);
            const T r1 = sqrt_t(l1), r2 = sqrt_t(l2);
            const T ir1 = T(1) / r1, ir2 = T(1) / r2;
            kap[0] *= ir1 * ir1 * ir1;
            kap[1] *= ir1 * ir1 * ir2;
            kap[2] *= ir1 * ir2 * ir2;
            kap[3] *= ir2 * ir2 * ir2;
            // K: ln h coefficients (Appendix, (1 - lambda S)/S = c - lambda)
            const T PI = T(3.14159265358979323846);
            const T isq = T(1) / (r1 * r2);
            const T iD1 = T(1) / ((T(3) * l1 + T(2) * l2) * l1);
            const T iD2 = T(1) / ((T(2) * l1 + T(3) * l2) * l2);
            const T c2x = cx * cx, s2x = sx * sx, scx = sx * cx;
            const T c1 = A.c1, c2 = A.c2;
            const T a1 = c1 - l1, a2 = c1 - l2, b1 = c2 - l1, b2 = c2 - l2;
            const T il12 = T(1) / (l1 + l2);
            const T p3 = T(3) * PI * isq;
            const T L11 = -PI * isq * (T(3) * c2x * a1 * a1 * iD1 + T(3) * s2x * a2 * a2 * iD2 + T(1));
            const T L12 = p3 * scx * (a1 * b1 * iD1 - a2 * b2 * iD2);
            const T L14 = p3 * scx * (a1 * iD1 - a2 * iD2);
            const T L15 = p3 * (c2x * a1 * iD1 + s2x * a2 * iD2);
            const T L22 = -PI * isq * (T(3) * s2x * b1 * b1 * iD1 + T(3) * c2x * b2 * b2 * iD2 + T(1));
            const T L24 = -p3 * (s2x * b1 * iD1 + c2x * b2 * iD2);
            const T L25 = p3 * scx * (-b1 * iD1 + b2 * iD2);
            const T L44 = -p3 * (s2x * iD1 + c2x * iD2);
            const T L45 = p3 * scx * (-iD1 + iD2);
            const T L55 = -p3 * (c2x * iD1 + s2x * iD2);
            const T L36 = T(-1.5) * PI * isq * il12 * scx * (c1 - c2) * (T(1) / l1 - T(1) / l2);
            const T H33 = T(3) * PI * isq * il12;
            // cubic couplings K13, K23, K34, K35 (Gamma_1 = Gamma_3 = 0)
            const T i3 = T(1) / (T(3) * l1 + T(2) * l2), i2 = T(1) / (T(2) * l1 + T(3) * l2);
            const T Q0 = T(3) * kap[0] * l1 + kap[2] * l2;                     // 3 k0 l1 + k2 l2
            const T Q1 = kap[1] * l1 + T(3) * kap[3] * l2;                     // k1 l1 + 3 k3 l2
            const T Sa = (T(7) * l1 + T(2) * l2) * kap[0] + (l1 + T(2) * l2) * kap[2];
            const T Sb = (T(2) * l1 + l2) * kap[1] + (T(2) * l1 + T(7) * l2) * kap[3];
            const T pre13 = T(-1.5) * PI * isq * il12;
            const T L13 = pre13 * ((T(2) * r1 * Q0 - T(1.5) * c1 * ir1 * Sa) * cx * i3 +
                                   (T(2) * r2 * Q1 - T(1.5) * c1 * ir2 * Sb) * sx * i2 +
                                   T(3) * A.G0 * (c2x / l1 + s2x / l2) + A.G2 * (s2x / l1 + c2x / l2));
            const T L23 = pre13 * ((T(-2) * r1 * Q0 + T(1.5) * c2 * ir1 * Sa) * sx * i3 +
                                   (T(2) * r2 * Q1 - T(1.5) * c2 * ir2 * Sb) * cx * i2 +
                                   T(2) * A.G2 * scx * (T(1) / l2 - T(1) / l1));
            const T pre34 = T(2.25) * PI * isq * il12;
            const T Bq = Sb * ir2 * i2, Aq = Sa * ir1 * i3;
            const T L34 = pre34 * (Bq * cx - Aq * sx);
            const T L35 = -pre34 * (Aq * cx + Bq * sx);
            // K~: subtract the value at the element's cut-off (Eq. lub:resistance-correction)
            const T lt = (he < R.delta_t) ? log1p_t((T)((he - R.delta_t) / R.delta_t)) : T(0);
            const T lr = (he < R.delta_r) ? log1p_t((T)((he - R.delta_r) / R.delta_r)) : T(0);
            const T hq = (he < R.delta_n) ? (T)((R.delta_n - he) / (he * R.delta_n)) : T(0);
            // relative surface velocities in the local frame
            const V3<T> vi = mk<T>(__ldg(P.vx + i), __ldg(P.vy + i), __ldg(P.vz + i));
            const V3<T> Wi = mk<T>(__ldg(P.wx + i), __ldg(P.wy + i), __ldg(P.wz + i));
            const V3<T> Vi = add(vi, cross(Wi, rho_i));
            const V3<T> dV = sub(Vj, Vi), dW = sub(Wj, Wi);
            const T u1 = dot(x1, dV), u2 = dot(x2, dV), u3 = dot(x3, dV);
            const T u4 = dot(x1, dW), u5 = dot(x2, dW), u6 = dot(x3, dW);
            const T mu = (T)R.mu;
            T F1 = mu * (lt * (L11 * u1 + L12 * u2 + L13 * u3 + L14 * u4 + L15 * u5));
            T F2 = mu * (lt * (L12 * u1 + L22 * u2 + L23 * u3 + L24 * u4 + L25 * u5));
            T F3 = mu * (lt * (L13 * u1 + L23 * u2 + L34 * u4 + L35 * u5 + L36 * u6) + hq * H33 * u3);
            T T4 = mu * (lt * (L14 * u1 + L24 * u2 + L34 * u3) + lr * (L44 * u4 + L45 * u5));
            T T5 = mu * (lt * (L15 * u1 + L25 * u2 + L35 * u3) + lr * (L45 * u4 + L55 * u5));
            T T6 = mu * (lt * (L36 * u3));
            if (R.h_c > 0.0 && h <= R.h_c) {
                const double Fr = (h > 0.0) ? R.eps_c * (R.h_c - h) : R.eps_c * R.h_c;
                F3 -= (T)Fr;
            }
            const V3<T> F = axpy(F1, x1, axpy(F2, x2, scl(F3, x3)));
            const V3<T> Tq = axpy(T4, x1, axpy(T5, x2, scl(T6, x3)));
            out[0] = F.x; out[1] = F.y; out[2] = F.z;
            out[3] = Tq.x; out[4] = Tq.y; out[5] = Tq.z;
            out[6] = rho_i.x; out[7] = rho_i.y; out[8] = rho_i.z;
            out[9] = rho_j.x; out[10] = rho_j.y; out[11] = rho_j.z;
        }
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            FT[a * C + k] = out[a];
            lever[a * C + k] = out[6 + a];
        }
        status[k] = (uint8_t)st;
    }
}

}  // namespace

int launch_resistance(lub_ctx *ctx, const PView &P, const DView &D, const Ens &E, const lub_params &prm,
                      const int32_t *pi, const int32_t *pj, const int32_t *d_count, int32_t cap, const double *n,
                      const double *gap, uint8_t *status, void *FT, void *lever, cudaStream_t st)
{
    if (cap == 0) return LUB_OK;
    RParams R{prm.mu, prm.delta_n, prm.delta_t, prm.delta_r, prm.h_c, prm.eps_c};
    const Shape2 sh = tuned_shape(ctx, LUB_TUNE_RESISTANCE, cap);
    const bool ens = E.nb > 0;
    if (prm.precision == LUB_MIXED) {
        if (ens)
            k_resistance<float, true><<<sh.grid, sh.block, 0, st>>>(P, D, E, R, pi, pj, d_count, cap, n, gap, status,
                                                                    (float *)FT, (float *)lever);
        else
            k_resistance<float, false><<<sh.grid, sh.block, 0, st>>>(P, D, E, R, pi, pj, d_count, cap, n, gap, status,
                                                                     (float *)FT, (float *)lever);
    } else {
        if (ens)
            k_resistance<double, true><<<sh.grid, sh.block, 0, st>>>(P, D, E, R, pi, pj, d_count, cap, n, gap,
                                                                     status, (double *)FT, (double *)lever);
        else
            k_resistance<double, false><<<sh.grid, sh.block, 0, st>>>(P, D, E, R, pi, pj, d_count, cap, n, gap,
                                                                      status, (double *)FT, (double *)lever);
    }
    return lub_check_cuda(ctx, cudaGetLastError(), "k_resistance launch");
}
