// Particle sub-stepping (Sec. II): the particle update runs at a fraction of
// the lattice-Boltzmann time step so that the strongly varying explicit
// lubrication forces are followed in time, while the forces exchanged with
// the fluid stay constant over the LB step.  One sub-step of length dt,
// semi-implicit (symplectic) Euler on the rigid-body equations of each
// spheroid, in double precision:
//   v <- v + dt (F_ext + f) / m,            r <- r + dt v
//   L  = I_lab(q) w + dt (T_ext + t),       w_mid = I_lab(q)^-1 L
//   q <- exp(dt w_mid / 2) q,               w <- I_lab(q_new)^-1 L
// with m = rho V, V = 4/3 pi R_par R_perp^2, body inertia
// I_par = 2/5 m R_perp^2 (about the symmetry axis o), I_perp = 1/5 m
// (R_par^2 + R_perp^2), I_lab^-1 = (1/I_perp) (1 - o o^T) + (1/I_par) o o^T.
// Torque-free motion keeps L exactly; f, t are the lubrication force and
// torque (about the centre) from lub_apply or lub_resistance_apply.
#include "lub_internal.cuh"

namespace {

struct Axis {
    double x, y, z;
};

__device__ __forceinline__ Axis axis_of(double w, double x, double y, double z)
{
    const double s = 2.0 / (w * w + x * x + y * y + z * z);
    return Axis{s * (x * z + w * y), s * (y * z - w * x), 1.0 - s * (x * x + y * y)};
}

// I_lab^-1 applied to a, or I_lab applied to a (inverse = false)
__device__ __forceinline__ void inertia_apply(const Axis &o, double ipar, double iperp, const double a[3],
                                              double out[3], bool inverse)
{
    const double oa = o.x * a[0] + o.y * a[1] + o.z * a[2];
    const double cpar = inverse ? 1.0 / ipar : ipar, cperp = inverse ? 1.0 / iperp : iperp;
    out[0] = cperp * (a[0] - oa * o.x) + cpar * oa * o.x;
    out[1] = cperp * (a[1] - oa * o.y) + cpar * oa * o.y;
    out[2] = cperp * (a[2] - oa * o.z) + cpar * oa * o.z;
}

template <typename T>
__global__ void k_rigid_step(int n, double *__restrict__ x, double *__restrict__ y, double *__restrict__ z,
                             float *__restrict__ qw, float *__restrict__ qx, float *__restrict__ qy,
                             float *__restrict__ qz, float *__restrict__ vx, float *__restrict__ vy,
                             float *__restrict__ vz, float *__restrict__ wx, float *__restrict__ wy,
                             float *__restrict__ wz, const float *__restrict__ rpar, const float *__restrict__ rperp,
                             const T *__restrict__ force, const T *__restrict__ torque,
                             const float *__restrict__ fext, const float *__restrict__ text, double rho, double dt)
{
    const size_t N = (size_t)n;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const double a = rperp[k], c = rpar[k];
        const double m = rho * (4.0 / 3.0) * 3.14159265358979323846 * c * a * a;
        const double ipar = 0.4 * m * a * a, iperp = 0.2 * m * (c * c + a * a);
        double F[3], Tq[3];
        for (int d = 0; d < 3; ++d) {
            F[d] = (double)force[d * N + k] + (fext ? (double)fext[d * N + k] : 0.0);
            Tq[d] = (double)torque[d * N + k] + (text ? (double)text[d * N + k] : 0.0);
        }
        // translation
        const double v0 = (double)vx[k] + dt * F[0] / m, v1 = (double)vy[k] + dt * F[1] / m,
                     v2 = (double)vz[k] + dt * F[2] / m;
        x[k] += dt * v0;
        y[k] += dt * v1;
        z[k] += dt * v2;
        vx[k] = (float)v0;
        vy[k] = (float)v1;
        vz[k] = (float)v2;
        // rotation
        double q0 = qw[k], q1 = qx[k], q2 = qy[k], q3 = qz[k];
        const double qn = 1.0 / sqrt(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
        q0 *= qn;
        q1 *= qn;
        q2 *= qn;
        q3 *= qn;
        const Axis o = axis_of(q0, q1, q2, q3);
        const double w[3] = {wx[k], wy[k], wz[k]};
        double L[3], wm[3];
        inertia_apply(o, ipar, iperp, w, L, false);
        for (int d = 0; d < 3; ++d) L[d] += dt * Tq[d];
        inertia_apply(o, ipar, iperp, L, wm, true);
        // q <- exp(dt wm / 2) q (unit quaternion of the rotation by |wm| dt about wm)
        const double ang = dt * sqrt(wm[0] * wm[0] + wm[1] * wm[1] + wm[2] * wm[2]);
        double r0 = 1.0, r1 = 0.0, r2 = 0.0, r3 = 0.0;
        if (ang > 0.0) {
            const double s = sin(0.5 * ang) * dt / ang;
            r0 = cos(0.5 * ang);
            r1 = s * wm[0];
            r2 = s * wm[1];
            r3 = s * wm[2];
        }
        double n0 = r0 * q0 - r1 * q1 - r2 * q2 - r3 * q3;
        double n1 = r0 * q1 + r1 * q0 + r2 * q3 - r3 * q2;
        double n2 = r0 * q2 - r1 * q3 + r2 * q0 + r3 * q1;
        double n3 = r0 * q3 + r1 * q2 - r2 * q1 + r3 * q0;
        const double nn = 1.0 / sqrt(n0 * n0 + n1 * n1 + n2 * n2 + n3 * n3);
        n0 *= nn;
        n1 *= nn;
        n2 *= nn;
        n3 *= nn;
        qw[k] = (float)n0;
        qx[k] = (float)n1;
        qy[k] = (float)n2;
        qz[k] = (float)n3;
        const Axis o2 = axis_of(n0, n1, n2, n3);
        double wn[3];
        inertia_apply(o2, ipar, iperp, L, wn, true);
        wx[k] = (float)wn[0];
        wy[k] = (float)wn[1];
        wz[k] = (float)wn[2];
    }
}

// ---------------------------------------------------------------------------
// seeded random rigid motions (no counterpart in the paper): the input
// preparation of the time-stepped workloads, on the device so that a loop of
// motion + correction steps can be captured into one CUDA graph.
// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC 2011): ten rounds of two 32x32 -> 64-bit multiplies,
// the key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
    constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += W0;
            k.y += W1;
        }
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// two standard normal draws from two 32-bit words (Box-Muller on uniforms in (0, 1])
__device__ __forceinline__ float2 box_muller(uint32_t a, uint32_t b)
{
    const float u1 = (float)((a >> 8) + 1u) * 0x1p-24f;
    const float u2 = (float)(b >> 8) * 0x1p-24f;
    const float r = sqrtf(-2.0f * logf(u1));
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    return make_float2(r * c, r * s);
}

// particle k, step s = step0 (+ *step_dev): counter (k, s low, s high, draw),
// key = seed; six normals: the displacement (sigma_r each) and the rotation
// vector (sigma_t each); q <- exp(theta / 2) q, renormalised.  next_dev
// (another address) receives s + 1.
__global__ void __launch_bounds__(256) k_random_motion(int n, double *__restrict__ x, double *__restrict__ y,
                                                       double *__restrict__ z, float *__restrict__ qw,
                                                       float *__restrict__ qx, float *__restrict__ qy,
                                                       float *__restrict__ qz, uint2 key, int64_t step0,
                                                       const int64_t *__restrict__ step_dev,
                                                       int64_t *__restrict__ next_dev, float sig_r, float sig_t)
{
    const uint64_t step = (uint64_t)(step0 + (step_dev ? *step_dev : 0));
    if (next_dev && blockIdx.x == 0 && threadIdx.x == 0) *next_dev = (int64_t)step + 1;
    const uint32_t step_lo = (uint32_t)step, step_hi = (uint32_t)(step >> 32);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const uint4 r0 = philox4x32_10(make_uint4((uint32_t)k, step_lo, step_hi, 0u), key);
        const uint4 r1 = philox4x32_10(make_uint4((uint32_t)k, step_lo, step_hi, 1u), key);
        const float2 g0 = box_muller(r0.x, r0.y), g1 = box_muller(r0.z, r0.w), g2 = box_muller(r1.x, r1.y);
        x[k] += (double)(sig_r * g0.x);
        y[k] += (double)(sig_r * g0.y);
        z[k] += (double)(sig_r * g1.x);
        const float t0 = sig_t * g1.y, t1 = sig_t * g2.x, t2 = sig_t * g2.y;
        const float a = sqrtf(t0 * t0 + t1 * t1 + t2 * t2);
        float sh, ch;
        sincosf(0.5f * a, &sh, &ch);
        const float sc = a > 0.f ? sh / a : 0.5f;
        const float dw = ch, dx = sc * t0, dy = sc * t1, dz = sc * t2;
        const float w = qw[k], xx = qx[k], yy = qy[k], zz = qz[k];
        const float nw = dw * w - dx * xx - dy * yy - dz * zz;
        const float nx = dw * xx + dx * w + dy * zz - dz * yy;
        const float ny = dw * yy - dx * zz + dy * w + dz * xx;
        const float nz = dw * zz + dx * yy - dy * xx + dz * w;
        const float inv = rsqrtf(nw * nw + nx * nx + ny * ny + nz * nz);
        qw[k] = nw * inv;
        qx[k] = nx * inv;
        qy[k] = ny * inv;
        qz[k] = nz * inv;
    }
}

}  // namespace

int launch_random_motion(lub_ctx *ctx, const lub_particles *p, uint64_t seed, int64_t step, const int64_t *step_dev,
                         int64_t *next_dev, double sig_r, double sig_t, cudaStream_t st)
{
    if (p->n == 0 && !next_dev) return LUB_OK;
    double *x = const_cast<double *>(p->x), *y = const_cast<double *>(p->y), *z = const_cast<double *>(p->z);
    float *qw = const_cast<float *>(p->qw), *qx = const_cast<float *>(p->qx), *qy = const_cast<float *>(p->qy),
          *qz = const_cast<float *>(p->qz);
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    k_random_motion<<<grid_for(p->n, 256, ctx->num_sms, 8), 256, 0, st>>>(
        p->n, x, y, z, qw, qx, qy, qz, key, step, step_dev, next_dev, (float)sig_r, (float)sig_t);
    return lub_check_cuda(ctx, cudaGetLastError(), "k_random_motion launch");
}

int launch_rigid_step(lub_ctx *ctx, const lub_particles *p, const void *force, const void *torque, int precision,
                      const float *fext, const float *text, double rho, double dt, cudaStream_t st)
{
    if (p->n == 0) return LUB_OK;
    // the particle arrays are written in place: the caller owns them as writable memory
    double *x = const_cast<double *>(p->x), *y = const_cast<double *>(p->y), *z = const_cast<double *>(p->z);
    float *qw = const_cast<float *>(p->qw), *qx = const_cast<float *>(p->qx), *qy = const_cast<float *>(p->qy),
          *qz = const_cast<float *>(p->qz);
    float *vx = const_cast<float *>(p->vx), *vy = const_cast<float *>(p->vy), *vz = const_cast<float *>(p->vz);
    float *wx = const_cast<float *>(p->wx), *wy = const_cast<float *>(p->wy), *wz = const_cast<float *>(p->wz);
    const int grid = grid_for(p->n, 256, ctx->num_sms, 8);
    if (precision == LUB_MIXED)
        k_rigid_step<float><<<grid, 256, 0, st>>>(p->n, x, y, z, qw, qx, qy, qz, vx, vy, vz, wx, wy, wz, p->r_par,
                                                  p->r_perp, (const float *)force, (const float *)torque, fext, text,
                                                  rho, dt);
    else
        k_rigid_step<double><<<grid, 256, 0, st>>>(p->n, x, y, z, qw, qx, qy, qz, vx, vy, vz, wx, wy, wz, p->r_par,
                                                   p->r_perp, (const double *)force, (const double *)torque, fext,
                                                   text, rho, dt);
    return lub_check_cuda(ctx, cudaGetLastError(), "k_rigid_step launch");
}
