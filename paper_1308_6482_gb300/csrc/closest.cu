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
// One thread per pair.  In LUB_MIXED the iterations run in FP32, the gap is
// always evaluated in FP64 (h is stationary in n, so the FP32 normal costs
// only O(dn^2)), and pairs with h/a below fp64_switch get FP64 Newton steps.
#include "lub_internal.cuh"

namespace {

struct NewtonOut {
    int iters;
    bool converged;
};

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
__device__ NewtonOut newton_sphere(const Shape<T> &si, const Shape<T> &sj, const V3<T> &d, V3<T> &n,
                                   int maxit, T tol, T noise)
{
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
            T idet = T(1) / det;
            s1 = (P22 * g1 - P12 * g2) * idet;
            s2 = (P11 * g2 - P12 * g1) * idet;
        } else {
            T sc = T(1) / (fabs(P11) + fabs(P22) + fabs(P12) + Ai + Aj);
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

template <bool MIXED>
__global__ void __launch_bounds__(128) k_closest(PView P, DView D, const int32_t *__restrict__ pi,
                                                 const int32_t *__restrict__ pj,
                                                 const int32_t *__restrict__ d_count, int32_t cap,
                                                 double *__restrict__ nout, double *__restrict__ gap,
                                                 uint8_t *__restrict__ status, uint8_t *__restrict__ iters,
                                                 int maxit, float tol32, float fp64_switch, int warm)
{
    const int count = pair_count(d_count, cap);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
        const int i = __ldg(pi + k), j = __ldg(pj + k);
        int st = 0;
        int nit = 0;
        V3<double> n64 = mk<double>(0, 0, 0);
        double h = 0.0;
        bool bad = (i < 0 || i >= P.n || j >= P.n || j < -D.n_walls || j == i);
        if (!bad) bad = !shape_ok(__ldg(P.rpar + i), __ldg(P.rperp + i));
        if (!bad && j >= 0) bad = !shape_ok(__ldg(P.rpar + j), __ldg(P.rperp + j));
        if (bad) {
            st = LUB_ST_DEGENERATE;
        } else if (j < 0) {
            // plane wall w: n = -dir e_z, h = dir (z_i - wall_z) - sigma_i(e_z)
            const int w = -1 - j;
            const double dir = (double)D.wall_dir[w];
            Shape<double> si = load_shape<double>(P, i);
            n64 = mk<double>(0.0, 0.0, -dir);
            h = dir * (__ldg(P.z + i) - D.wall_z[w]) - support(si, mk<double>(0.0, 0.0, 1.0));
        } else {
            V3<double> d = min_image(D, sub(load_pos(P, j), load_pos(P, i)));
            double dl = sqrt(dot(d, d));
            if (!(dl > 0.0) || !isfinite(dl)) {
                st = LUB_ST_DEGENERATE;
            } else {
                const float rpi = __ldg(P.rpar + i), rqi = __ldg(P.rperp + i);
                const float rpj = __ldg(P.rpar + j), rqj = __ldg(P.rperp + j);
                if (rpi == rqi && rpj == rqj) {
                    // two spheres: n = d/|d|, h = |d| - R_i - R_j
                    n64 = scl(1.0 / dl, d);
                    h = dl - (double)rpi - (double)rpj;
                } else {
                    Shape<double> si64 = load_shape<double>(P, i), sj64 = load_shape<double>(P, j);
                    V3<double> start = scl(1.0 / dl, d);
                    if (warm) {
                        V3<double> w0 = mk<double>(nout[k], nout[cap + k], nout[2 * (size_t)cap + k]);
                        double wl = dot(w0, w0);
                        if (wl > 0.25 && wl < 4.0 && isfinite(wl)) start = scl(rsqrt(wl), w0);
                    }
                    const double scale = dl + (double)fmaxf(rpi, rqi) + (double)fmaxf(rpj, rqj);
                    bool conv;
                    if (MIXED) {
                        Shape<float> si = load_shape<float>(P, i), sj = load_shape<float>(P, j);
                        V3<float> n = cvt<float>(start);
                        V3<float> df = cvt<float>(d);
                        NewtonOut o = newton_sphere<float>(si, sj, df, n, maxit, tol32,
                                                           (float)(4e-7 * scale));
                        nit = o.iters;
                        conv = o.converged;
                        n64 = normalized(cvt<double>(n));
                        h = dot(n64, d) - support(si64, n64) - support(sj64, n64);
                        const double amin = (double)fminf(fminf(rpi, rqi), fminf(rpj, rqj));
                        if (!conv || h < (double)fp64_switch * amin) {
                            // FP64 Newton: refinement near contact, or full solve as fallback
                            V3<double> nn = conv ? n64 : start;
                            NewtonOut o2 = newton_sphere<double>(si64, sj64, d, nn, conv ? 4 : maxit, 1e-11,
                                                                 1e-14 * scale);
                            nit += o2.iters;
                            conv = o2.converged;
                            n64 = normalized(nn);
                            h = dot(n64, d) - support(si64, n64) - support(sj64, n64);
                            st |= LUB_ST_FP64;
                        }
                    } else {
                        V3<double> nn = start;
                        NewtonOut o = newton_sphere<double>(si64, sj64, d, nn, maxit, 1e-11, 1e-14 * scale);
                        nit = o.iters;
                        conv = o.converged;
                        n64 = normalized(nn);
                        h = dot(n64, d) - support(si64, n64) - support(sj64, n64);
                    }
                    // consistency check of Sec. III A: the normals point to the other centre
                    if (!conv || !(dot(n64, d) > 0.0) || !isfinite(h)) st |= LUB_ST_NOCONV;
                }
            }
        }
        if (!(st & LUB_ST_DEGENERATE) && h <= 0.0) st |= LUB_ST_OVERLAP;
        nout[k] = n64.x;
        nout[cap + k] = n64.y;
        nout[2 * (size_t)cap + k] = n64.z;
        gap[k] = h;
        status[k] = (uint8_t)st;
        if (iters) iters[k] = (uint8_t)(nit > 255 ? 255 : nit);
    }
}

}  // namespace

int launch_closest(lub_ctx *ctx, const PView &P, const DView &D, const lub_params &prm, const int32_t *pi,
                   const int32_t *pj, const int32_t *d_count, int32_t cap, double *n, double *gap,
                   uint8_t *status, uint8_t *iters, cudaStream_t st)
{
    if (cap == 0) return LUB_OK;
    const int block = 128;
    const int grid = grid_for(cap, block, ctx->num_sms, 8);
    const int warm = prm.warm_start == LUB_WARM_PREVIOUS;
    if (prm.precision == LUB_MIXED)
        k_closest<true><<<grid, block, 0, st>>>(P, D, pi, pj, d_count, cap, n, gap, status, iters, prm.max_newton,
                                                (float)prm.newton_tol, (float)prm.fp64_switch, warm);
    else
        k_closest<false><<<grid, block, 0, st>>>(P, D, pi, pj, d_count, cap, n, gap, status, iters,
                                                 prm.max_newton, (float)prm.newton_tol, (float)prm.fp64_switch,
                                                 warm);
    return lub_check_cuda(ctx, cudaGetLastError(), "k_closest launch");
}
