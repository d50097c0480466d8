// The learned warm start's inference, shared by the start kernel (mlp.cu)
// and the closest-point kernels that run it in front of Newton (closest.cu):
// the 12 pair features, the warp-level BF16 tensor-core forward pass of the
// 12 -> 128 -> 128 -> 4 network, and Newton's start normal from its outputs.
// See mlp.cu for the network and its training.
#pragma once

#include <cuda_bf16.h>

#include "lub_internal.cuh"
#include "lub_mlp.cuh"

namespace {

constexpr int NI = 12, NH = 128, NO = 4;

// ---------------------------------------------------------------------------
// features (the same device code for training and inference)
// ---------------------------------------------------------------------------
// The 12 features (FP32): in i's body frame turned about its symmetry axis
// until d lies in the half-plane y = 0, x >= 0: [0] rho / R_perp,i,
// [1] d_z / R_perp,i, [2..4] j's axis; [5..8] ln of the four semi-axes;
// [9] asinh(g(d^)/a); [10, 11] ln(sigma(d^) / R_perp) of i and j.  Invariant
// under rigid motions of the pair and rotations of either particle about its
// own axis, like the targets.
__device__ __forceinline__ void pair_features(const PView &P, const DView &D, int i, int j, const float *mean,
                                              const float *istd, float f[NI])
{
    const V3<double> dd = min_image(D, sub(load_pos(P, j), load_pos(P, i)));
    const V3<float> d = cvt<float>(dd);
    float qa[4] = {P.qw[i], P.qx[i], P.qy[i], P.qz[i]};
    const float na = rsqrtf(qa[0] * qa[0] + qa[1] * qa[1] + qa[2] * qa[2] + qa[3] * qa[3]);
    for (int a = 0; a < 4; ++a) qa[a] *= na;
    // i's rotation R(q_a); body coordinates are R^T applied to lab vectors
    const float w = qa[0], x = qa[1], y = qa[2], z = qa[3];
    const float R00 = 1 - 2 * (y * y + z * z), R01 = 2 * (x * y - w * z), R02 = 2 * (x * z + w * y);
    const float R10 = 2 * (x * y + w * z), R11 = 1 - 2 * (x * x + z * z), R12 = 2 * (y * z - w * x);
    const float R20 = 2 * (x * z - w * y), R21 = 2 * (y * z + w * x), R22 = 1 - 2 * (x * x + y * y);
    const float rpi = P.rpar[i], rqi = P.rperp[i], rpj = P.rpar[j], rqj = P.rperp[j];
    const float dbx = R00 * d.x + R10 * d.y + R20 * d.z;
    const float dby = R01 * d.x + R11 * d.y + R21 * d.z;
    const float dbz = R02 * d.x + R12 * d.y + R22 * d.z;
    const float rho = sqrtf(dbx * dbx + dby * dby);
    const float c = rho > 0.f ? dbx / rho : 1.f, s = rho > 0.f ? dby / rho : 0.f;
    const V3<float> oj = quat_axis<float>(P.qw[j], P.qx[j], P.qy[j], P.qz[j]);
    const float obx = R00 * oj.x + R10 * oj.y + R20 * oj.z;
    const float oby = R01 * oj.x + R11 * oj.y + R21 * oj.z;
    const float obz = R02 * oj.x + R12 * oj.y + R22 * oj.z;
    const float inv = 1.0f / rqi;
    f[0] = rho * inv;
    f[1] = dbz * inv;
    f[2] = c * obx + s * oby;
    f[3] = -s * obx + c * oby;
    f[4] = obz;
    f[5] = logf(rpi);
    f[6] = logf(rqi);
    f[7] = logf(rpj);
    f[8] = logf(rqj);
    const float dl = sqrtf(dot(d, d));
    const V3<float> e = scl(1.0f / dl, d);
    const Shape<float> si = load_shape<float>(P, i), sj = load_shape<float>(P, j);
    const float wi = support(si, e), wj = support(sj, e);
    const float amin = fminf(fminf(rpi, rqi), fminf(rpj, rqj));
    f[9] = asinhf((dl - wi - wj) / amin);
    f[10] = logf(wi / rqi);
    f[11] = logf(wj / rqj);
    if (mean)
        for (int a = 0; a < NI; ++a) f[a] = (f[a] - mean[a]) * istd[a];
}

// ---------------------------------------------------------------------------
// inference: BF16 tensor cores (mma.sync m16n8k16, FP32 accumulate)
// ---------------------------------------------------------------------------
// One warp runs 32 pairs (two 16-row m-tiles) through the three layers with
// the activations in registers: the accumulator fragment of two adjacent
// 8-column n-tiles is, element for element, the A fragment of one 16-deep
// k-tile of the next layer, so layer 1's output becomes layer 2's A operand
// without leaving the registers, and layer 2 is produced 16 columns at a time
// and folded straight into layer 3.  Only the features (in) and the four
// outputs (out) pass through shared memory.  The weights sit in shared memory
// in fragment order (conflict-free 16-byte loads).
constexpr int INF_WARPS = 8;
constexpr int XS = 24;  // row stride (bf16) of the staged features: conflict-free A-fragment loads

__device__ __forceinline__ void mma_bf16(float c[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// GELU of two accumulators, returned as the packed BF16 pair the next layer
// reads: the tanh form of Hendrycks & Gimpel (2016), evaluated in BF16x2
// arithmetic with the hardware tanh.  The inputs are rounded to BF16 first;
// the result is within a few BF16 ulps of the exact (erf) form the network is
// trained with.
__device__ __forceinline__ uint32_t gelu2(float a, float b)
{
    const uint32_t x = pack_bf16(a, b);
    const uint32_t c0 = 0x3F4C3F4Cu;  // sqrt(2/pi) = 0.7979 -> 0.7969 in BF16
    const uint32_t c1 = 0x3D123D12u;  // 0.044715 sqrt(2/pi) = 0.03568 -> 0.03564
    const uint32_t hf = 0x3F003F00u;  // 0.5
    uint32_t x2, v, u, t, h, r;
    asm("mul.rn.bf16x2 %0, %1, %1;" : "=r"(x2) : "r"(x));
    asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(v) : "r"(x2), "r"(c1), "r"(c0));
    asm("mul.rn.bf16x2 %0, %1, %2;" : "=r"(u) : "r"(x), "r"(v));
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(t) : "r"(u));
    asm("mul.rn.bf16x2 %0, %1, %2;" : "=r"(h) : "r"(x), "r"(hf));
    asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(r) : "r"(h), "r"(t), "r"(h));
    return r;
}

struct InfSmem {
    uint4 F1[8 * 32];
    uint4 F2[64 * 32];
    uint2 F3[8 * 32];
    float b1[NH], b2[NH], b3[8];
    float mean[NI], istd[NI];
    __nv_bfloat16 x[INF_WARPS][32 * XS];
    float4 y[INF_WARPS][32];
};

// the 4 network outputs of the calling lane's pair (features f, standardised,
// zero for an invalid pair); warp-collective
__device__ __forceinline__ float4 warp_mlp(const InfSmem &S, __nv_bfloat16 *xs, float4 *ys, const float f[NI],
                                           int lane)
{
    const int g = lane >> 2, t = lane & 3;
    // stage the features: row = lane, 12 values + 4 zeros of padding
    uint32_t *xr = reinterpret_cast<uint32_t *>(xs + lane * XS);
#pragma unroll
    for (int a = 0; a < 6; ++a) xr[a] = pack_bf16(f[2 * a], f[2 * a + 1]);
    xr[6] = 0u;
    xr[7] = 0u;
    __syncwarp();
    uint32_t A1[2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        const uint32_t *r0 = reinterpret_cast<const uint32_t *>(xs + (16 * mt + g) * XS) + t;
        const uint32_t *r1 = reinterpret_cast<const uint32_t *>(xs + (16 * mt + g + 8) * XS) + t;
        A1[mt][0] = r0[0];
        A1[mt][1] = r1[0];
        A1[mt][2] = r0[4];
        A1[mt][3] = r1[4];
    }
    // layer 1 -> A fragments of layer 2
    uint32_t A2[2][8][4];
#pragma unroll
    for (int p = 0; p < 8; ++p) {
        const uint4 bb = S.F1[p * 32 + lane];
        const float2 bl = *reinterpret_cast<const float2 *>(&S.b1[16 * p + 2 * t]);
        const float2 bh = *reinterpret_cast<const float2 *>(&S.b1[16 * p + 8 + 2 * t]);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            float c0[4] = {bl.x, bl.y, bl.x, bl.y}, c1[4] = {bh.x, bh.y, bh.x, bh.y};
            mma_bf16(c0, A1[mt][0], A1[mt][1], A1[mt][2], A1[mt][3], bb.x, bb.y);
            mma_bf16(c1, A1[mt][0], A1[mt][1], A1[mt][2], A1[mt][3], bb.z, bb.w);
            A2[mt][p][0] = gelu2(c0[0], c0[1]);
            A2[mt][p][1] = gelu2(c0[2], c0[3]);
            A2[mt][p][2] = gelu2(c1[0], c1[1]);
            A2[mt][p][3] = gelu2(c1[2], c1[3]);
        }
    }
    // layer 2, 16 columns at a time, each folded into layer 3 as one k-tile
    const float2 b3 = *reinterpret_cast<const float2 *>(&S.b3[2 * t]);
    float y[2][4] = {{b3.x, b3.y, b3.x, b3.y}, {b3.x, b3.y, b3.x, b3.y}};
#pragma unroll 1
    for (int p = 0; p < 8; ++p) {
        const float2 bl = *reinterpret_cast<const float2 *>(&S.b2[16 * p + 2 * t]);
        const float2 bh = *reinterpret_cast<const float2 *>(&S.b2[16 * p + 8 + 2 * t]);
        float c[2][2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            c[mt][0][0] = c[mt][0][2] = bl.x;
            c[mt][0][1] = c[mt][0][3] = bl.y;
            c[mt][1][0] = c[mt][1][2] = bh.x;
            c[mt][1][1] = c[mt][1][3] = bh.y;
        }
#pragma unroll
        for (int kt = 0; kt < 8; ++kt) {
            const uint4 bb = S.F2[(p * 8 + kt) * 32 + lane];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                mma_bf16(c[mt][0], A2[mt][kt][0], A2[mt][kt][1], A2[mt][kt][2], A2[mt][kt][3], bb.x, bb.y);
                mma_bf16(c[mt][1], A2[mt][kt][0], A2[mt][kt][1], A2[mt][kt][2], A2[mt][kt][3], bb.z, bb.w);
            }
        }
        const uint2 b = S.F3[p * 32 + lane];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
            mma_bf16(y[mt], gelu2(c[mt][0][0], c[mt][0][1]), gelu2(c[mt][0][2], c[mt][0][3]),
                     gelu2(c[mt][1][0], c[mt][1][1]), gelu2(c[mt][1][2], c[mt][1][3]), b.x, b.y);
    }
    // outputs: columns 0..3 live in lanes t = 0, 1 of each row group
    float *yf = reinterpret_cast<float *>(ys);
    if (t < 2) {
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            yf[(16 * mt + g) * 4 + 2 * t] = y[mt][0];
            yf[(16 * mt + g) * 4 + 2 * t + 1] = y[mt][1];
            yf[(16 * mt + g + 8) * 4 + 2 * t] = y[mt][2];
            yf[(16 * mt + g + 8) * 4 + 2 * t + 1] = y[mt][3];
        }
    }
    __syncwarp();
    const float4 out = ys[lane];
    __syncwarp();
    return out;
}

// rotation of a particle (columns: body axes in the lab frame)
struct Rot {
    float m[3][3];
};

__device__ __forceinline__ Rot rot_of(const PView &P, int k)
{
    const float w = P.qw[k], x = P.qx[k], y = P.qy[k], z = P.qz[k];
    const float s = 2.0f / (w * w + x * x + y * y + z * z);
    Rot R;
    R.m[0][0] = 1 - s * (y * y + z * z);
    R.m[0][1] = s * (x * y - w * z);
    R.m[0][2] = s * (x * z + w * y);
    R.m[1][0] = s * (x * y + w * z);
    R.m[1][1] = 1 - s * (x * x + z * z);
    R.m[1][2] = s * (y * z - w * x);
    R.m[2][0] = s * (x * z - w * y);
    R.m[2][1] = s * (y * z + w * x);
    R.m[2][2] = 1 - s * (x * x + y * y);
    return R;
}

// Outward unit normal (lab frame) of particle k at the surface point whose
// parameters are those of the support point along lab direction e, shifted by
// (dp, dq).  With the support point's body direction b = R^T e, its parameters
// are p0 = atan2(R_par b_z, R_perp |b_xy|), q0 = atan2(b_y, b_x) (q0 = 0 on
// the axis); cos and sin of p0 + dp and q0 + dq follow by the angle-addition
// rules, so only the small shifts go through sin/cos.
__device__ __forceinline__ V3<float> shifted_normal(const PView &P, int k, const Rot &R, const V3<float> &e, float dp,
                                                    float dq)
{
    const float bx = R.m[0][0] * e.x + R.m[1][0] * e.y + R.m[2][0] * e.z;
    const float by = R.m[0][1] * e.x + R.m[1][1] * e.y + R.m[2][1] * e.z;
    const float bz = R.m[0][2] * e.x + R.m[1][2] * e.y + R.m[2][2] * e.z;
    const float rpar = P.rpar[k], rperp = P.rperp[k];
    const float rho = sqrtf(bx * bx + by * by);
    const float cp0u = rperp * rho, sp0u = rpar * bz;
    const float ih = rsqrtf(cp0u * cp0u + sp0u * sp0u);
    const float cp0 = cp0u * ih, sp0 = sp0u * ih;
    const float cq0 = rho > 0.f ? bx / rho : 1.f, sq0 = rho > 0.f ? by / rho : 0.f;
    float sdp, cdp, sdq, cdq;
    __sincosf(dp, &sdp, &cdp);
    __sincosf(dq, &sdq, &cdq);
    const float cp = cp0 * cdp - sp0 * sdp, sp = sp0 * cdp + cp0 * sdp;
    const float cq = cq0 * cdq - sq0 * sdq, sq = sq0 * cdq + cq0 * sdq;
    // normal direction of x^2/a^2 + y^2/a^2 + z^2/c^2 = 1 at (p, q), up to a positive factor
    const V3<float> nb = mk<float>(rpar * cp * cq, rpar * cp * sq, rperp * sp);
    const V3<float> nl = mk<float>(R.m[0][0] * nb.x + R.m[0][1] * nb.y + R.m[0][2] * nb.z,
                                   R.m[1][0] * nb.x + R.m[1][1] * nb.y + R.m[1][2] * nb.z,
                                   R.m[2][0] * nb.x + R.m[2][1] * nb.y + R.m[2][2] * nb.z);
    return normalized(nl);
}

// a pair's indices, domain and validity, and its standardised features f
// (zero for an invalid pair)
struct PairIn {
    int i, j;
    const DView *D;
    bool ok;
};

template <bool ENS>
__device__ __forceinline__ PairIn pair_inputs(const PView &P, const DView &D0, const Ens &E,
                                              const int32_t *__restrict__ pi, const int32_t *__restrict__ pj, int k,
                                              int count, const float *mean, const float *istd, float f[NI])
{
    PairIn in{-1, -1, &D0, false};
    if (k < count) {
        in.i = pi[k];
        in.j = pj[k];
        bool alien;
        in.D = &pair_domain<ENS>(D0, E, in.i, in.j, &alien);
        in.ok = !alien && in.i >= 0 && in.i < P.n && in.j >= 0 && in.j < P.n && in.i != in.j &&
                shape_ok(P.rpar[in.i], P.rperp[in.i]) && shape_ok(P.rpar[in.j], P.rperp[in.j]);
    }
    if (in.ok) {
        pair_features(P, *in.D, in.i, in.j, mean, istd, f);
        for (int a = 0; a < NI; ++a)
            if (!isfinite(f[a])) in.ok = false;
    }
    if (!in.ok)
        for (int a = 0; a < NI; ++a) f[a] = 0.f;
    return in;
}

// the network's outputs y of pair k to pq, and Newton's start normal to n0
__device__ __forceinline__ void pair_outputs(const PView &P, const PairIn &in, const float4 y, int k, int count,
                                             size_t C, double *__restrict__ n0, float *__restrict__ pq)
{
    if (k < count && pq) {
        pq[k] = in.ok ? y.x : 0.f;
        pq[C + k] = in.ok ? y.y : 0.f;
        pq[2 * C + k] = in.ok ? y.z : 0.f;
        pq[3 * C + k] = in.ok ? y.w : 0.f;
    }
    if (k < count && n0) {
        V3<float> s0 = mk<float>(0, 0, 0);
        if (in.ok) {
            // corrections to the parameters of the line-of-centres start
            const V3<float> d = cvt<float>(min_image(*in.D, sub(load_pos(P, in.j), load_pos(P, in.i))));
            const V3<float> e = normalized(d);
            const V3<float> ni = shifted_normal(P, in.i, rot_of(P, in.i), e, y.x, y.y);
            const V3<float> nj = shifted_normal(P, in.j, rot_of(P, in.j), scl(-1.0f, e), y.z, y.w);
            const V3<float> s = sub(ni, nj);
            const float l2 = dot(s, s);
            if (l2 > 1e-12f && isfinite(l2)) s0 = scl(rsqrtf(l2), s);
        }
        n0[k] = s0.x;
        n0[C + k] = s0.y;
        n0[2 * C + k] = s0.z;
    }
}

// the weights, biases and feature scaling of the installed network into a
// block's shared memory (all threads of the block)
__device__ __forceinline__ void stage_weights(InfSmem &S, const MlpDevice &M)
{
    for (int k = threadIdx.x; k < 8 * 32; k += blockDim.x) {
        S.F1[k] = M.F1[k];
        S.F3[k] = M.F3[k];
    }
    for (int k = threadIdx.x; k < 64 * 32; k += blockDim.x) S.F2[k] = M.F2[k];
    for (int k = threadIdx.x; k < NH; k += blockDim.x) {
        S.b1[k] = M.b1[k];
        S.b2[k] = M.b2[k];
    }
    for (int k = threadIdx.x; k < 8; k += blockDim.x) S.b3[k] = M.b3[k];
    for (int k = threadIdx.x; k < NI; k += blockDim.x) {
        S.mean[k] = M.mean[k];
        S.istd[k] = M.istd[k];
    }
}

}  // namespace
