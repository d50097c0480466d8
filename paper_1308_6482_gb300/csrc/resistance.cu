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
#include "pair_force.cuh"

namespace {

template <typename T, bool ENS>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 6 : 1) k_resistance(PView P, const __grid_constant__ DView D0, Ens E, RParams R,
                                                    const int32_t *__restrict__ pi, const int32_t *__restrict__ pj,
                                                    const int32_t *__restrict__ d_count, int32_t cap,
                                                    const double *__restrict__ nin, const double *__restrict__ gap,
                                                    uint8_t *__restrict__ status, T *__restrict__ FT,
                                                    T *__restrict__ lever, const float2 *__restrict__ pff)
{
    pdl_wait();
    pdl_trigger();
    const int count = pair_count(d_count, cap);
    const size_t C = (size_t)cap;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
        int st = status[k];
        const double h = gap[k];
        const int i = __ldg(pi + k), j = __ldg(pj + k);
        // indices are checked here too: status may not come from lub_closest_points
        bool alien;
        const DView &D = pair_domain<ENS>(D0, E, i, j, &alien);
        if (alien || i < 0 || i >= P.n || j >= P.n || j < -D.n_walls || j == i) st |= LUB_ST_DEGENERATE;
        const V3<double> n = mk<double>(nin[k], nin[C + k], nin[2 * C + k]);
        T out[12];
        pair_force<T>(P, R, i, j, n, h, st, out, pff);
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            FT[a * C + k] = out[a];
            lever[a * C + k] = out[6 + a];
        }
        status[k] = (uint8_t)st;
    }
}

// resistance and the atomic scatter of lub_apply in one pass (FT, lever optional)
template <typename T, bool ENS>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 7 : 1) k_resistance_apply(PView P, const __grid_constant__ DView D0, Ens E, RParams R,
                                                          const int32_t *__restrict__ pi,
                                                          const int32_t *__restrict__ pj,
                                                          const int32_t *__restrict__ d_count, int32_t cap,
                                                          const double *__restrict__ nin,
                                                          const double *__restrict__ gap,
                                                          uint8_t *__restrict__ status, T *__restrict__ FT,
                                                          T *__restrict__ lever, T *__restrict__ force,
                                                          T *__restrict__ torque, const float2 *__restrict__ pff,
                                                          const float4 *__restrict__ nh)
{
    pdl_wait();
    pdl_trigger();
    const int count = pair_count(d_count, cap);
    const size_t C = (size_t)cap;
    // warp-uniform loop bound: the whole warp takes part in the scatter
    for (int base = blockIdx.x * blockDim.x; base < count; base += gridDim.x * blockDim.x) {
        const int k = base + threadIdx.x;
        int i = -1, j = -1, st = LUB_ST_DEGENERATE;
        T out[12];
        T ci[6] = {0, 0, 0, 0, 0, 0}, cj[6] = {0, 0, 0, 0, 0, 0};
        if (k < count) {
            st = status[k];
            i = __ldg(pi + k);
            j = __ldg(pj + k);
            bool alien;
            const DView &D = pair_domain<ENS>(D0, E, i, j, &alien);
            if (alien || i < 0 || i >= P.n || j >= P.n || j < -D.n_walls || j == i) st |= LUB_ST_DEGENERATE;
            bool done = false;
            if constexpr (sizeof(T) == 4) {
                if (nh) {  // the fused pass: normal and gap in float-float from the closest-point kernels
                    const float4 a = nh[k], b = nh[C + k];
                    const ff nf[3] = {{a.x, a.y}, {a.z, a.w}, {b.x, b.y}};
                    pair_force_ff(R, i, j, nf, ff{b.z, b.w}, st, out, pff);
                    done = true;
                }
            }
            if (!done) {
                const V3<double> n = mk<double>(nin[k], nin[C + k], nin[2 * C + k]);
                pair_force<T>(P, R, i, j, n, gap[k], st, out, pff);
            }
            if (FT)
#pragma unroll
                for (int a = 0; a < 6; ++a) FT[a * C + k] = out[a];
            if (lever)
#pragma unroll
                for (int a = 0; a < 6; ++a) lever[a * C + k] = out[6 + a];
            status[k] = (uint8_t)st;
            side_contrib(out, 0, ci);
            if (j >= 0) side_contrib(out, 1, cj);
        }
        const bool ok = !(st & LUB_ST_DEGENERATE);
        scatter_warp<T>(ok ? i : -1, ok ? j : -1, (size_t)P.n, ci, cj, force, torque);
    }
}

}  // namespace

// the mixed mode's per-call particle records in the context scratch
static int particle_table(lub_ctx *ctx, const PView &P, cudaStream_t st, const float2 **pff)
{
    int rc = lub_ensure_scratch(ctx, particles_ff_bytes(P.n));
    if (rc) return rc;
    *pff = (const float2 *)ctx->scratch;
    return launch_particles_ff(ctx, P, (float2 *)ctx->scratch, st);
}

int launch_resistance_apply(lub_ctx *ctx, const PView &P, const DView &D, const Ens &E, const lub_params &prm,
                            const int32_t *pi, const int32_t *pj, const int32_t *d_count, int32_t cap,
                            const double *n, const double *gap, uint8_t *status, void *FT, void *lever, void *force,
                            void *torque, int accumulate, cudaStream_t st, const float2 *pff, const float4 *nh)
{
    const size_t esz = prm.precision == LUB_MIXED ? sizeof(float) : sizeof(double);
    int rc;
    if (!accumulate && P.n > 0) {
        if ((rc = zero_force_torque(ctx, force, torque, 3 * (size_t)P.n * esz, st))) return rc;
    }
    if (cap == 0) return LUB_OK;
    const RParams R = make_rparams(prm);
    const Shape2 sh = tuned_shape(ctx, LUB_TUNE_RESISTANCE, cap);
    const bool ens = E.nb > 0;
    if (prm.precision == LUB_MIXED) {
        if (!pff && (rc = particle_table(ctx, P, st, &pff))) return rc;
        lub_trace_mark(ctx, LUB_TRACE_RESISTANCE, st);
        if (ens)
            (void)launch_pdl(k_resistance_apply<float, true>, sh.grid, sh.block, 0, st, P, D, E, R, pi, pj, d_count,
                             cap, n, gap, status, (float *)FT, (float *)lever, (float *)force, (float *)torque, pff,
                             nh);
        else
            (void)launch_pdl(k_resistance_apply<float, false>, sh.grid, sh.block, 0, st, P, D, E, R, pi, pj, d_count,
                             cap, n, gap, status, (float *)FT, (float *)lever, (float *)force, (float *)torque, pff,
                             nh);
    } else {
        const float2 *none = nullptr;
        const float4 *no_nh = nullptr;
        lub_trace_mark(ctx, LUB_TRACE_RESISTANCE, st);
        if (ens)
            (void)launch_pdl(k_resistance_apply<double, true>, sh.grid, sh.block, 0, st, P, D, E, R, pi, pj, d_count,
                             cap, n, gap, status, (double *)FT, (double *)lever, (double *)force, (double *)torque,
                             none, no_nh);
        else
            (void)launch_pdl(k_resistance_apply<double, false>, sh.grid, sh.block, 0, st, P, D, E, R, pi, pj, d_count,
                             cap, n, gap, status, (double *)FT, (double *)lever, (double *)force, (double *)torque,
                             none, no_nh);
    }
    lub_trace_mark(ctx, LUB_TRACE_RESISTANCE, st);
    return lub_check_cuda(ctx, cudaGetLastError(), "k_resistance_apply launch");
}

int launch_resistance(lub_ctx *ctx, const PView &P, const DView &D, const Ens &E, const lub_params &prm,
                      const int32_t *pi, const int32_t *pj, const int32_t *d_count, int32_t cap, const double *n,
                      const double *gap, uint8_t *status, void *FT, void *lever, cudaStream_t st)
{
    if (cap == 0) return LUB_OK;
    const RParams R = make_rparams(prm);
    const Shape2 sh = tuned_shape(ctx, LUB_TUNE_RESISTANCE, cap);
    const bool ens = E.nb > 0;
    if (prm.precision == LUB_MIXED) {
        const float2 *pff = nullptr;
        int rc = particle_table(ctx, P, st, &pff);
        if (rc) return rc;
        lub_trace_mark(ctx, LUB_TRACE_RESISTANCE, st);
        if (ens)
            (void)launch_pdl(k_resistance<float, true>, sh.grid, sh.block, 0, st, P, D, E, R, pi, pj, d_count, cap, n,
                             gap, status, (float *)FT, (float *)lever, pff);
        else
            (void)launch_pdl(k_resistance<float, false>, sh.grid, sh.block, 0, st, P, D, E, R, pi, pj, d_count, cap, n,
                             gap, status, (float *)FT, (float *)lever, pff);
    } else {
        const float2 *none = nullptr;
        lub_trace_mark(ctx, LUB_TRACE_RESISTANCE, st);
        if (ens)
            (void)launch_pdl(k_resistance<double, true>, sh.grid, sh.block, 0, st, P, D, E, R, pi, pj, d_count, cap, n,
                             gap, status, (double *)FT, (double *)lever, none);
        else
            (void)launch_pdl(k_resistance<double, false>, sh.grid, sh.block, 0, st, P, D, E, R, pi, pj, d_count, cap, n,
                             gap, status, (double *)FT, (double *)lever, none);
    }
    lub_trace_mark(ctx, LUB_TRACE_RESISTANCE, st);
    return lub_check_cuda(ctx, cudaGetLastError(), "k_resistance launch");
}
