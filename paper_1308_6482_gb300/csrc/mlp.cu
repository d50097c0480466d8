// Learned warm start of the closest-point solve: a 12 -> 128 -> 128 -> 4 MLP
// (GELU) mapping a pair's relative pose to the surface parameters
// (p_i, q_i, p_j, q_j) of Eq. lub:spheroid at its closest points.
//
//   features  12 per pair, invariant under the motions that leave the
//             targets unchanged (rigid motions, rotations of a particle about
//             its own axis): d and j's axis in i's body frame turned about
//             i's axis until d lies in its x-z half-plane; ln of the four
//             semi-axes; asinh of the support-function gap estimate along d
//             over the smallest semi-axis; the two half-widths along d;
//             standardised with the training set's mean and 1/std.
//   outputs   corrections to the surface parameters of the line-of-centres
//             start (the support points of i along d^ and of j along -d^), so
//             a zero output gives back the cold start n0 = d^ exactly and the
//             network only learns a small, continuous correction;
//   training  FP32 kernels: linear forward (optionally + GELU), a weighted
//             squared error with the azimuth differences wrapped to (-pi, pi],
//             backward through the layers, Adam.  Parameters packed [W1 | b1 | W2 | b2 | W3 | b3]
//             with W row-major [out][in].
//   inference BF16 weights and activations on the tensor cores (mma.sync
//             m16n8k16, FP32 accumulate), one warp per 32 pairs with the
//             activations in registers; the predicted (p, q) give the outward
//             normals n_i, n_j at the predicted points and Newton's start
//             n0 = (n_i - n_j)/|n_i - n_j|.
#include <cuda_bf16.h>

#include "lub_internal.cuh"
#include "lub_mlp.cuh"
#include "mlp_infer.cuh"

namespace {


__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_d_f(float x)
{
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.3989422804014327f;
}

__device__ __forceinline__ float wrap_pi_f(float x)
{
    const float tp = 6.283185307179586f;
    return x - tp * floorf(x / tp + 0.5f);
}

__global__ void k_mlp_features(PView P, DView D, const int32_t *__restrict__ pi, const int32_t *__restrict__ pj,
                               int n, const float *__restrict__ mean, const float *__restrict__ istd,
                               float *__restrict__ feat)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        float f[NI];
        pair_features(P, D, pi[k], pj[k], mean, istd, f);
        for (int a = 0; a < NI; ++a) feat[(size_t)k * NI + a] = f[a];
    }
}

// ---------------------------------------------------------------------------
// training (FP32)
// ---------------------------------------------------------------------------
constexpr int TS = 32;  // tile edge of the small GEMMs

// Y[m][n] = sum_k X[m][k] W[n][k] + b[n]; Z = Y; H = gelu(Y) if act
__global__ void k_linear_fwd(const float *__restrict__ X, const float *__restrict__ W, const float *__restrict__ b,
                             int M, int K, int N, float *__restrict__ Z, float *__restrict__ H, int act)
{
    __shared__ float xs[TS][TS + 1], ws[TS][TS + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    const int m0 = blockIdx.y * TS, n0 = blockIdx.x * TS;
    float acc[4] = {0, 0, 0, 0};
    for (int k0 = 0; k0 < K; k0 += TS) {
        for (int r = ty; r < TS; r += 8) {
            const int m = m0 + r, k = k0 + tx, n = n0 + r;
            xs[r][tx] = (m < M && k < K) ? X[(size_t)m * K + k] : 0.f;
            ws[r][tx] = (n < N && k < K) ? W[(size_t)n * K + k] : 0.f;
        }
        __syncthreads();
        for (int kk = 0; kk < TS; ++kk) {
            const float wv = ws[tx][kk];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] += xs[ty + 8 * q][kk] * wv;
        }
        __syncthreads();
    }
    const int n = n0 + tx;
    if (n >= N) return;
    for (int q = 0; q < 4; ++q) {
        const int m = m0 + ty + 8 * q;
        if (m >= M) continue;
        const float v = acc[q] + b[n];
        Z[(size_t)m * N + n] = v;
        if (act) H[(size_t)m * N + n] = gelu_f(v);
    }
}

// dX[m][k] = sum_n dZ[m][n] W[n][k]   (optionally times gelu'(Zprev[m][k]))
__global__ void k_linear_bwd_x(const float *__restrict__ dZ, const float *__restrict__ W, int M, int K, int N,
                               const float *__restrict__ Zprev, float *__restrict__ dX)
{
    __shared__ float ds[TS][TS + 1], ws[TS][TS + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int m0 = blockIdx.y * TS, k0 = blockIdx.x * TS;
    float acc[4] = {0, 0, 0, 0};
    for (int n0 = 0; n0 < N; n0 += TS) {
        for (int r = ty; r < TS; r += 8) {
            const int m = m0 + r, n = n0 + tx;
            ds[r][tx] = (m < M && n < N) ? dZ[(size_t)m * N + n] : 0.f;
            const int nn = n0 + r, k = k0 + tx;
            ws[r][tx] = (nn < N && k < K) ? W[(size_t)nn * K + k] : 0.f;
        }
        __syncthreads();
        for (int nn = 0; nn < TS; ++nn) {
            const float wv = ws[nn][tx];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] += ds[ty + 8 * q][nn] * wv;
        }
        __syncthreads();
    }
    const int k = k0 + tx;
    if (k >= K) return;
    for (int q = 0; q < 4; ++q) {
        const int m = m0 + ty + 8 * q;
        if (m >= M) continue;
        float v = acc[q];
        if (Zprev) v *= gelu_d_f(Zprev[(size_t)m * K + k]);
        dX[(size_t)m * K + k] = v;
    }
}

// dW[n][k] = sum_m dZ[m][n] X[m][k];  db[n] = sum_m dZ[m][n]
__global__ void k_linear_bwd_w(const float *__restrict__ dZ, const float *__restrict__ X, int M, int K, int N,
                               float *__restrict__ dW, float *__restrict__ db)
{
    __shared__ float ds[TS][TS + 1], xs[TS][TS + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int n0 = blockIdx.y * TS, k0 = blockIdx.x * TS;
    float acc[4] = {0, 0, 0, 0};
    float bacc = 0.f;
    for (int m0 = 0; m0 < M; m0 += TS) {
        for (int r = ty; r < TS; r += 8) {
            const int m = m0 + r;
            ds[r][tx] = (m < M && n0 + tx < N) ? dZ[(size_t)m * N + n0 + tx] : 0.f;
            xs[r][tx] = (m < M && k0 + tx < K) ? X[(size_t)m * K + k0 + tx] : 0.f;
        }
        __syncthreads();
        for (int mm = 0; mm < TS; ++mm) {
            const float xv = xs[mm][tx];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] += ds[mm][ty + 8 * q] * xv;
        }
        if (blockIdx.x == 0 && ty == 0)
            for (int mm = 0; mm < TS; ++mm) bacc += ds[mm][tx];
        __syncthreads();
    }
    const int k = k0 + tx;
    for (int q = 0; q < 4; ++q) {
        const int n = n0 + ty + 8 * q;
        if (n < N && k < K) dW[(size_t)n * K + k] = acc[q];
    }
    if (blockIdx.x == 0 && ty == 0 && n0 + tx < N) db[n0 + tx] = bacc;
}

// weighted loss terms and dY = w r / M (azimuth errors wrapped); per-row losses to lrow
__global__ void k_mlp_loss(const float *__restrict__ Y, const float *__restrict__ T, const float *__restrict__ Wt,
                           int M, float *__restrict__ dY, float *__restrict__ lrow)
{
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
        float l = 0.f;
        for (int o = 0; o < NO; ++o) {
            float r = Y[(size_t)m * NO + o] - T[(size_t)m * NO + o];
            if (o & 1) r = wrap_pi_f(r);
            const float wgt = Wt ? Wt[(size_t)m * NO + o] : 1.f;
            l += 0.5f * wgt * r * r;
            dY[(size_t)m * NO + o] = wgt * r / (float)M;
        }
        lrow[m] = l;
    }
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const float gk = g[k];
        const float mk = b1 * m[k] + (1.f - b1) * gk;
        const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    }
}

// ---------------------------------------------------------------------------
// inference on the 5th-generation tensor cores (tcgen05, accumulators in TMEM)
// ---------------------------------------------------------------------------
// A CTA of 256 threads takes 128 pairs at a time; warps w and w + 4 share
// TMEM lane quarter w, so every row (pair) has two threads, each taking 64 of
// its 128 columns in the epilogues; the first thread of a row also computes
// the pair's features and its outputs:
//   features -> X (128 x 16, shared memory)
//   layer 1:  one tcgen05.mma (M 128, N 128, K 16) into TMEM columns [0, 128)
//   epilogue: each thread loads its half row (tcgen05.ld), adds the bias,
//             applies GELU and writes BF16 into H (128 x 128, shared memory)
//   layer 2:  eight MMAs (K 16 each) into the same columns (the epilogue has
//             read them), epilogue to H
//   layer 3:  eight MMAs (N 16: outputs padded 4 -> 16) into columns [0, 16)
//   outputs:  the first thread of each row loads its four outputs and forms
//             Newton's start.
// One elected thread issues the MMAs and commits them to an mbarrier the CTA
// waits on.  Operands are K-major without swizzle: 8-row x 16-byte core
// matrices, element (r, k) of an R x K operand at byte
//   (r / 8) SBO + (k / 8) 128 + (r % 8) 16 + (k % 8) 2,   SBO = K / 8 x 128,
// so the K-th 16-element step of an MMA starts 256 bytes further.  The
// weights (B operands) sit in global memory as an image of the shared-memory
// block and arrive with one bulk copy (cp.async.bulk) per CTA.  Every wait is
// bounded: a timeout raises an error bit, waits (bounded) for the MMAs in
// flight, frees the TMEM and returns.
constexpr int TC_ROWS = 128;
constexpr int TC_THREADS = 256;           // two threads per row: each takes 64 of its 128 columns
constexpr uint32_t TC_TMEM_COLS = 128;    // every layer's accumulator in columns [0, 128)
// bound of every mbarrier wait, in polls; a test build compiles a short one in
#ifndef LUB_TC_SPIN_LIMIT
#define LUB_TC_SPIN_LIMIT (1l << 24)
#endif
constexpr long kTcSpinLimit = LUB_TC_SPIN_LIMIT;
#ifdef LUB_TESTING
// a test build's hook: the elected thread issues no MMA and no commit, so
// every wait for an MMA runs out (with no MMA in flight when TMEM is freed)
__device__ int g_test_skip_mma = 0;
#endif

__host__ __device__ constexpr uint32_t cm_offset(int r, int k, int K)
{
    return (uint32_t)((r >> 3) * (K / 8 * 128) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

struct TcImage {                     // the bytes of one bulk copy (multiple of 16)
    __nv_bfloat16 W1[128 * 16];      // B of layer 1: N 128 x K 16 (inputs 12 -> 16)
    __nv_bfloat16 W2[128 * 128];     // B of layer 2
    __nv_bfloat16 W3[16 * 128];      // B of layer 3: N 16 (outputs 4 -> 16) x K 128
    float b1[128], b2[128], b3[16];
    float mean[NI], istd[NI];
};
static_assert(sizeof(TcImage) % 16 == 0, "bulk copies move multiples of 16 bytes");

struct TcSmem {
    TcImage w;
    __nv_bfloat16 X[TC_ROWS * 16];   // A of layer 1
    __nv_bfloat16 H[TC_ROWS * 128];  // A of layers 2 and 3
    unsigned long long mbar_w, mbar_mma;
    uint32_t tmem;
    int stop;
    // padding: above 76 KB a third CTA never fits an SM, so two CTAs x 256
    // columns never exceed the SM's 512 TMEM columns (allocation never waits)
    unsigned char pad[4096];
};
static_assert(sizeof(TcSmem) > 228 * 1024 / 3, "at most two CTAs per SM");

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, leading (K) and stride (row) byte
// offsets, the fixed version bits of this architecture, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: D F32, A and B BF16, both K-major, M x N
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(dtmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mbar)
                 : "memory");
}

// bounded wait for the phase `parity` of an mbarrier; false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    for (long it = 0; it < kTcSpinLimit; ++it) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
        if (it > 64) __nanosleep(32);
    }
    return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void async_proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 consecutive TMEM columns of this thread's lane (row)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32])
{
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                   "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                   "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

// epilogue of a hidden layer: TMEM columns [c0, c0 + 64) of this thread's row
// + bias, GELU, BF16 into the same columns of its row of H
__device__ __forceinline__ void tc_hidden_epilogue(uint32_t trow, int c0, const float *bias, __nv_bfloat16 *H,
                                                   int row)
{
#pragma unroll 1
    for (int c = c0; c < c0 + 64; c += 32) {
        float v[32];
        tmem_ld32(trow + c, v);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            uint4 u;
            u.x = gelu2(v[8 * g + 0] + bias[c + 8 * g + 0], v[8 * g + 1] + bias[c + 8 * g + 1]);
            u.y = gelu2(v[8 * g + 2] + bias[c + 8 * g + 2], v[8 * g + 3] + bias[c + 8 * g + 3]);
            u.z = gelu2(v[8 * g + 4] + bias[c + 8 * g + 4], v[8 * g + 5] + bias[c + 8 * g + 5]);
            u.w = gelu2(v[8 * g + 6] + bias[c + 8 * g + 6], v[8 * g + 7] + bias[c + 8 * g + 7]);
            *reinterpret_cast<uint4 *>(reinterpret_cast<unsigned char *>(H) + cm_offset(row, c + 8 * g, 128)) = u;
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// the network's start normal for each pair of a tile (used by closest.cu)
// ---------------------------------------------------------------------------
template <bool ENS>
__global__ void __launch_bounds__(32 * INF_WARPS, 2) k_mlp_start(PView P, const __grid_constant__ DView D0, Ens E, const int32_t *__restrict__ pi,
                                                                const int32_t *__restrict__ pj,
                                                                const int32_t *__restrict__ d_count, int32_t cap,
                                                                MlpDevice M, double *__restrict__ n0,
                                                                float *__restrict__ pq)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    InfSmem &S = *reinterpret_cast<InfSmem *>(smem_raw);
    const int count = pair_count(d_count, cap);
    stage_weights(S, M);  // once per block
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const size_t C = (size_t)cap;
    for (int base = (blockIdx.x * INF_WARPS + w) * 32; base < count; base += gridDim.x * INF_WARPS * 32) {
        const int k = base + lane;
        float f[NI];
        PairIn in = pair_inputs<ENS>(P, D0, E, pi, pj, k, count, S.mean, S.istd, f);
        const float4 y = warp_mlp(S, S.x[w], S.y[w], f, lane);
        pair_outputs(P, in, y, k, count, C, n0, pq);
    }
}

template <bool ENS>
__global__ void __launch_bounds__(TC_THREADS) k_mlp_start_tc(PView P, const __grid_constant__ DView D0, Ens E,
                                                          const int32_t *__restrict__ pi,
                                                          const int32_t *__restrict__ pj,
                                                          const int32_t *__restrict__ d_count, int32_t cap,
                                                          const TcImage *__restrict__ img, double *__restrict__ n0,
                                                          float *__restrict__ pq, int32_t *__restrict__ err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TcSmem &S = *reinterpret_cast<TcSmem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = tid & (TC_ROWS - 1), half = tid >> 7;  // row = 32 (warp % 4) + lane
    const uint32_t mbw = smem_u32(&S.mbar_w), mbm = smem_u32(&S.mbar_mma);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(&S.tmem)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mbw));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mbm));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        S.stop = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem;
    const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16);  // this warp's lane quarter
    // the weights: one bulk copy into the shared block
    if (tid == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mbw),
                     "r"((uint32_t)sizeof(TcImage)) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     :: "r"(smem_u32(&S.w)), "l"(img), "r"((uint32_t)sizeof(TcImage)), "r"(mbw) : "memory");
    }
    bool alive = mbar_wait(mbw, 0);
    uint32_t phase = 0;
#ifdef LUB_TESTING
    const bool skip_mma = g_test_skip_mma != 0;
#else
    constexpr bool skip_mma = false;
#endif
    const uint32_t sX = smem_u32(S.X), sH = smem_u32(S.H);
    const uint32_t sW1 = smem_u32(S.w.W1), sW2 = smem_u32(S.w.W2), sW3 = smem_u32(S.w.W3);
    const int count = pair_count(d_count, cap);
    const size_t C = (size_t)cap;
    for (int base = blockIdx.x * TC_ROWS; base < count; base += gridDim.x * TC_ROWS) {
        if (!alive) S.stop = 1;
        __syncthreads();
        if (S.stop) break;
        const int k = base + row;
        float f[NI];
        PairIn in{-1, -1, &D0, false};
        if (half == 0) {
            in = pair_inputs<ENS>(P, D0, E, pi, pj, k, count, S.w.mean, S.w.istd, f);
            uint4 lo, hi;
            lo.x = pack_bf16(f[0], f[1]);
            lo.y = pack_bf16(f[2], f[3]);
            lo.z = pack_bf16(f[4], f[5]);
            lo.w = pack_bf16(f[6], f[7]);
            hi.x = pack_bf16(f[8], f[9]);
            hi.y = pack_bf16(f[10], f[11]);
            hi.z = 0u;
            hi.w = 0u;
            unsigned char *X = reinterpret_cast<unsigned char *>(S.X);
            *reinterpret_cast<uint4 *>(X + cm_offset(row, 0, 16)) = lo;
            *reinterpret_cast<uint4 *>(X + cm_offset(row, 8, 16)) = hi;
        }
        // layer 1
        async_proxy_fence();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0 && !skip_mma) {
            tc_mma(tmem, tc_desc(sX, 128, 256), tc_desc(sW1, 128, 256), tc_idesc(128, 128), 0u);
            tc_commit(mbm);
        }
        alive = mbar_wait(mbm, phase) && alive;
        phase ^= 1u;
        tc_fence_after();
        tc_hidden_epilogue(trow, 64 * half, S.w.b1, S.H, row);
        // layer 2
        async_proxy_fence();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0 && !skip_mma) {
            for (uint32_t kk = 0; kk < 8; ++kk)
                tc_mma(tmem, tc_desc(sH + 256 * kk, 128, 2048), tc_desc(sW2 + 256 * kk, 128, 2048),
                       tc_idesc(128, 128), kk);
            tc_commit(mbm);
        }
        alive = mbar_wait(mbm, phase) && alive;
        phase ^= 1u;
        tc_fence_after();
        // every thread has read its layer-2 input from H before it is overwritten:
        // the MMAs that read H completed (the wait above)
        tc_hidden_epilogue(trow, 64 * half, S.w.b2, S.H, row);
        // layer 3
        async_proxy_fence();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0 && !skip_mma) {
            for (uint32_t kk = 0; kk < 8; ++kk)
                tc_mma(tmem, tc_desc(sH + 256 * kk, 128, 2048), tc_desc(sW3 + 256 * kk, 128, 2048), tc_idesc(128, 16),
                       kk);
            tc_commit(mbm);
        }
        alive = mbar_wait(mbm, phase) && alive;
        phase ^= 1u;
        tc_fence_after();
        float v[32];
        tmem_ld32(trow, v);  // all warps: the load is warp-collective
        if (half == 0) {
            const float4 y = make_float4(v[0] + S.w.b3[0], v[1] + S.w.b3[1], v[2] + S.w.b3[2], v[3] + S.w.b3[3]);
            pair_outputs(P, in, y, k, count, C, n0, pq);
        }
        tc_fence_before();
    }
    if (!alive && err) atomicOr(err, 8);
    // a timeout may leave MMAs in flight: wait for the last commit (bounded) before freeing TMEM
    if (!alive) mbar_wait(mbm, phase);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TC_TMEM_COLS));
}

size_t mlp_start_smem() { return sizeof(InfSmem); }

template <bool ENS>
int launch_mlp_start_t(lub_ctx *ctx, const PView &P, const DView &D, const Ens &E, const int32_t *pi,
                       const int32_t *pj, const int32_t *d_count, int32_t cap, double *n0, float *pq, cudaStream_t st)
{
    if (ctx->mlp_engine == LUB_MLP_TCGEN05) {
        const size_t smem = sizeof(TcSmem);
        if (!(ctx->mlp_smem_set & (4 << ENS))) {
            int rc = lub_check_cuda(ctx,
                                    cudaFuncSetAttribute(k_mlp_start_tc<ENS>,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                                    "shared memory attribute");
            if (rc) return rc;
            ctx->mlp_smem_set |= 4 << ENS;
        }
        const MlpDevice &M = *(const MlpDevice *)ctx->mlp;
        const int tiles = (cap + TC_ROWS - 1) / TC_ROWS;
        const int grid = tiles < 2 * ctx->num_sms ? (tiles > 0 ? tiles : 1) : 2 * ctx->num_sms;
        k_mlp_start_tc<ENS><<<grid, TC_THREADS, smem, st>>>(P, D, E, pi, pj, d_count, cap,
                                                         (const TcImage *)M.tc_image, n0, pq, ctx->d_flags + 1);
        return lub_check_cuda(ctx, cudaGetLastError(), "k_mlp_start_tc launch");
    }
    const size_t smem = mlp_start_smem();
    if (!(ctx->mlp_smem_set & (1 << ENS))) {
        int rc = lub_check_cuda(
            ctx, cudaFuncSetAttribute(k_mlp_start<ENS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
            "shared memory attribute");
        if (rc) return rc;
        ctx->mlp_smem_set |= 1 << ENS;
    }
    k_mlp_start<ENS><<<ctx->num_sms * 2, 32 * INF_WARPS, smem, st>>>(P, D, E, pi, pj, d_count, cap,
                                                                     *(const MlpDevice *)ctx->mlp, n0, pq);
    return lub_check_cuda(ctx, cudaGetLastError(), "k_mlp_start launch");
}

int launch_mlp_start(lub_ctx *ctx, const PView &P, const DView &D, const Ens &E, const int32_t *pi, const int32_t *pj,
                     const int32_t *d_count, int32_t cap, double *n0, float *pq, cudaStream_t st)
{
    if (!ctx->mlp_ready) return lub_set_error(ctx, LUB_ERR_ARG, "the learned warm start needs lub_mlp_set first");
    if (cap == 0) return LUB_OK;
    return E.nb ? launch_mlp_start_t<true>(ctx, P, D, E, pi, pj, d_count, cap, n0, pq, st)
                : launch_mlp_start_t<false>(ctx, P, D, E, pi, pj, d_count, cap, n0, pq, st);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
int launch_mlp_features(lub_ctx *ctx, const PView &P, const DView &D, const int32_t *pi, const int32_t *pj, int n,
                        const float *mean, const float *istd, float *feat, cudaStream_t st)
{
    if (n <= 0) return LUB_OK;
    k_mlp_features<<<grid_for(n, 128, ctx ? ctx->num_sms : 152, 16), 128, 0, st>>>(P, D, pi, pj, n, mean, istd, feat);
    return lub_check_cuda(ctx, cudaGetLastError(), "k_mlp_features launch");
}

int launch_mlp_forward_backward(lub_ctx *ctx, const float *params, const float *x, const float *tgt,
                                const float *wgt, int M, float *grads, float *work, float *loss_rows, cudaStream_t st)
{
    const float *W1 = params, *b1 = W1 + NH * NI, *W2 = b1 + NH, *b2 = W2 + NH * NH, *W3 = b2 + NH, *b3 = W3 + NO * NH;
    float *gW1 = grads, *gb1 = gW1 + NH * NI, *gW2 = gb1 + NH, *gb2 = gW2 + NH * NH, *gW3 = gb2 + NH,
          *gb3 = gW3 + NO * NH;
    // work: z1 h1 z2 h2 [M x 128] each, y dy [M x 4], d2 d1 [M x 128]
    float *z1 = work, *h1 = z1 + (size_t)M * NH, *z2 = h1 + (size_t)M * NH, *h2 = z2 + (size_t)M * NH;
    float *y = h2 + (size_t)M * NH, *dy = y + (size_t)M * NO, *d2 = dy + (size_t)M * NO, *d1 = d2 + (size_t)M * NH;
    const dim3 blk(32, 8);
    auto grid = [&](int cols, int rows) { return dim3((cols + TS - 1) / TS, (rows + TS - 1) / TS); };
    k_linear_fwd<<<grid(NH, M), blk, 0, st>>>(x, W1, b1, M, NI, NH, z1, h1, 1);
    k_linear_fwd<<<grid(NH, M), blk, 0, st>>>(h1, W2, b2, M, NH, NH, z2, h2, 1);
    k_linear_fwd<<<grid(NO, M), blk, 0, st>>>(h2, W3, b3, M, NH, NO, y, nullptr, 0);
    k_mlp_loss<<<grid_for(M, 256, ctx ? ctx->num_sms : 152, 8), 256, 0, st>>>(y, tgt, wgt, M, dy, loss_rows);
    // layer 3
    k_linear_bwd_w<<<grid(NH, NO), blk, 0, st>>>(dy, h2, M, NH, NO, gW3, gb3);
    k_linear_bwd_x<<<grid(NH, M), blk, 0, st>>>(dy, W3, M, NH, NO, z2, d2);
    // layer 2
    k_linear_bwd_w<<<grid(NH, NH), blk, 0, st>>>(d2, h1, M, NH, NH, gW2, gb2);
    k_linear_bwd_x<<<grid(NH, M), blk, 0, st>>>(d2, W2, M, NH, NH, z1, d1);
    // layer 1
    k_linear_bwd_w<<<grid(NI, NH), blk, 0, st>>>(d1, x, M, NI, NH, gW1, gb1);
    return lub_check_cuda(ctx, cudaGetLastError(), "mlp forward/backward launch");
}

int launch_mlp_adam(lub_ctx *ctx, float *params, const float *grads, float *m, float *v, int n, int t, float lr,
                    float b1, float b2, float eps, cudaStream_t st)
{
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    k_adam<<<grid_for(n, 256, ctx ? ctx->num_sms : 152, 4), 256, 0, st>>>(params, grads, m, v, n, lr, b1, b2, eps, c1,
                                                                          c2);
    return lub_check_cuda(ctx, cudaGetLastError(), "mlp adam launch");
}

// pack FP32 parameters into the BF16 inference layout owned by the context
// B-fragment element of mma.m16n8k16 for B = W^T (W row-major [n][k], nv x kv
// valid, zero padding): lane (g, t) holds W[8 nt + g][16 kt + 2 t + 8 h + {0, 1}]
__device__ __forceinline__ uint32_t frag_b(const float *W, int nv, int kv, int nt, int kt, int lane, int h)
{
    const int n = 8 * nt + (lane >> 2), k = 16 * kt + 2 * (lane & 3) + 8 * h;
    const float lo = (n < nv && k < kv) ? W[n * kv + k] : 0.f;
    const float hi = (n < nv && k + 1 < kv) ? W[n * kv + k + 1] : 0.f;
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// the tcgen05 image: W in the core-matrix layout of the B operands, biases,
// standardisation (mean, istd are copied in by the host after this kernel)
__global__ void k_mlp_pack_tc(const float *__restrict__ params, TcImage *__restrict__ T)
{
    const float *W1 = params, *b1 = W1 + NH * NI, *W2 = b1 + NH, *b2 = W2 + NH * NH, *W3 = b2 + NH, *b3 = W3 + NO * NH;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < NH * NH; e += gridDim.x * blockDim.x) {
        const int n = e / NH, k = e % NH;
        T->W2[cm_offset(n, k, 128) / 2] = __float2bfloat16_rn(W2[n * NH + k]);
        if (e < 128 * 16) {
            const int n1 = e / 16, k1 = e % 16;
            T->W1[cm_offset(n1, k1, 16) / 2] = __float2bfloat16_rn(k1 < NI ? W1[n1 * NI + k1] : 0.f);
        }
        if (e < 16 * 128) {
            const int n3 = e / NH, k3 = e % NH;
            T->W3[cm_offset(n3, k3, 128) / 2] = __float2bfloat16_rn(n3 < NO ? W3[n3 * NH + k3] : 0.f);
        }
        if (e < NH) {
            T->b1[e] = b1[e];
            T->b2[e] = b2[e];
        }
        if (e < 16) T->b3[e] = e < NO ? b3[e] : 0.f;
    }
}

__global__ void k_mlp_pack(const float *__restrict__ params, MlpDevice M)
{
    const float *W1 = params, *b1 = W1 + NH * NI, *W2 = b1 + NH, *b2 = W2 + NH * NH, *W3 = b2 + NH, *b3 = W3 + NO * NH;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 64 * 32; e += gridDim.x * blockDim.x) {
        const int lane = e & 31, kt = (e >> 5) & 7, p = e >> 8;
        M.F2[e] = make_uint4(frag_b(W2, NH, NH, 2 * p, kt, lane, 0), frag_b(W2, NH, NH, 2 * p, kt, lane, 1),
                             frag_b(W2, NH, NH, 2 * p + 1, kt, lane, 0), frag_b(W2, NH, NH, 2 * p + 1, kt, lane, 1));
        if (e < 8 * 32) {
            const int q = e >> 5;
            M.F1[e] = make_uint4(frag_b(W1, NH, NI, 2 * q, 0, lane, 0), frag_b(W1, NH, NI, 2 * q, 0, lane, 1),
                                 frag_b(W1, NH, NI, 2 * q + 1, 0, lane, 0), frag_b(W1, NH, NI, 2 * q + 1, 0, lane, 1));
            M.F3[e] = make_uint2(frag_b(W3, NO, NH, 0, q, lane, 0), frag_b(W3, NO, NH, 0, q, lane, 1));
        }
        if (e < NH) {
            M.b1[e] = b1[e];
            M.b2[e] = b2[e];
        }
        if (e < 8) M.b3[e] = e < NO ? b3[e] : 0.f;
    }
}

size_t mlp_tc_image_bytes() { return sizeof(TcImage); }

int launch_mlp_pack(lub_ctx *ctx, const float *params, const MlpDevice &M, cudaStream_t st)
{
    k_mlp_pack_tc<<<16, 256, 0, st>>>(params, (TcImage *)M.tc_image);
    k_mlp_pack<<<8, 256, 0, st>>>(params, M);
    return lub_check_cuda(ctx, cudaGetLastError(), "mlp pack launch");
}

#ifdef LUB_TESTING
// Test build only (no counterpart in the product library): on != 0 makes the
// tcgen05 network issue no MMA, so that its bounded mbarrier waits run out.
extern "C" int lub_test_skip_tc_mma(int32_t on)
{
    return cudaMemcpyToSymbol(g_test_skip_mma, &on, sizeof(int)) == cudaSuccess ? LUB_OK : LUB_ERR_CUDA;
}
#endif
