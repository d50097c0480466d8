// Internal declarations of liblub: context, device helpers and kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lub.h"

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct lub_ctx {
    std::string err;
    int device = -1;
    int num_sms = 0;
    // growable device scratch
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    int32_t *d_flags = nullptr;  // [0]: the last pair build's flags (bit 0: a semi-axis above the
                                 // bound; bit 2: a scan timed out; bit 4: the sweep's range check);
                                 // [1]: timed-out waits since the last lub_sync_status (bit 2: a
                                 // scan, bit 3: the tcgen05 network)
    void *mlp = nullptr;         // MlpDevice of the learned warm start (lub_mlp_set)
    void *mlp_mem = nullptr;     // its device storage
    bool mlp_ready = false;
    int mlp_smem_set = 0;        // bit k: shared-memory attribute set for instantiation k
    int mlp_engine = 0;          // LUB_MLP_MMA_SYNC or LUB_MLP_TCGEN05
    // device copies of the ensemble tables (slot 0: domains, slot 1: cell grids),
    // with the host bytes they were uploaded from; buffers only grow, retired
    // ones are freed with the context
    struct Table {
        std::vector<char> host;
        void *dev = nullptr;
        size_t cap = 0;
    } table[2];
    std::vector<void *> retired;
    // launch shapes chosen by lub_autotune (0 = built-in default)
    int tune_block[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int tune_per_sm[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    // kernel trace (lub_trace_enable): events recorded around each traced
    // kernel since the last read (start, end, start, end, ...), and spares
    bool trace = false;
    std::vector<cudaEvent_t> trace_ev[LUB_TRACE_COUNT];
    std::vector<cudaEvent_t> trace_pool;
};

// one trace event of kernel `id` on st (before or after its launch); no-op
// unless tracing is on and st is not capturing
void lub_trace_mark(lub_ctx *ctx, int id, cudaStream_t st);
void lub_trace_free(lub_ctx *ctx);

// device copy of a host table, re-uploaded only when its bytes change
int lub_upload_table(lub_ctx *ctx, int slot, const void *host, size_t bytes, cudaStream_t st, const void **dev);

int lub_set_error(lub_ctx *ctx, int code, const char *fmt, ...);
int lub_check_cuda(lub_ctx *ctx, cudaError_t e, const char *what);
int lub_ensure_scratch(lub_ctx *ctx, size_t bytes);

// ---------------------------------------------------------------------------
// plain-old-data views passed to kernels by value
// ---------------------------------------------------------------------------
struct PView {
    const double *x, *y, *z;
    const float *qw, *qx, *qy, *qz;
    const float *rpar, *rperp;
    const float *vx, *vy, *vz, *wx, *wy, *wz;
    int32_t n;
};

struct DView {
    double L[3];
    double invL[3];
    int32_t periodic[3];
    int32_t n_walls;
    double wall_z[2];
    int32_t wall_dir[2];
    // the box lengths as float-float (hi, lo) and 1/L in float, for the
    // separations of the FP32 stage; pad keeps the struct free of padding
    // bytes (ensemble tables are compared bytewise)
    float Lff[3][2];
    float invLf[3];
    int32_t pad;
};

// ensemble mode: per-suspension domain and particle range [p0, p1)
struct EnsDom {
    DView D;
    int32_t p0, p1;
};

struct Ens {
    const EnsDom *dom;  // device [nb]
    int32_t nb;         // 0: one suspension
};

// suspension of particle k (k clamped into the table's range)
__device__ __forceinline__ int batch_of(const Ens &E, int k)
{
    int lo = 0, hi = E.nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&E.dom[mid].p0) <= k)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// domain of the pair (i, j): D itself for one suspension, i's suspension's in
// ensemble mode; a particle partner j outside that suspension makes the pair
// invalid (*alien = true)
// (a reference: D should be a __grid_constant__ kernel parameter, read in place)
template <bool ENS>
__device__ __forceinline__ const DView &pair_domain(const DView &D, const Ens &E, int i, int j, bool *alien)
{
    if (!ENS) {
        *alien = false;
        return D;
    }
    const EnsDom &B = E.dom[batch_of(E, i)];
    *alien = j >= 0 && (j < __ldg(&B.p0) || j >= __ldg(&B.p1));
    return B.D;
}

struct RParams {
    double mu, delta_n, delta_t, delta_r, h_c, eps_c;
    int model;    // LUB_MODEL_FULL or LUB_MODEL_NORMAL
    int contact;  // h_c > 0: the contact model (clip and Hookean repulsion) is on
    // for the FP32 path: the cut-offs and h_c as float-float (hi, lo), mu,
    // eps_c and the reciprocals of the cut-offs as float (no FP64 per pair)
    float dn_ff[2], dt_ff[2], dr_ff[2], hc_ff[2];
    float mu_f, eps_f, idn_f, idt_f, idr_f;
};

inline RParams make_rparams(const lub_params &p)
{
    RParams R{p.mu, p.delta_n, p.delta_t, p.delta_r, p.h_c, p.eps_c, p.model, p.h_c > 0.0 ? 1 : 0,
              {0, 0}, {0, 0}, {0, 0}, {0, 0}, (float)p.mu, (float)p.eps_c, (float)(1.0 / p.delta_n),
              (float)(1.0 / p.delta_t), (float)(1.0 / p.delta_r)};
    auto split = [](double v, float o[2]) {
        o[0] = (float)v;
        o[1] = (float)(v - (double)o[0]);
    };
    split(p.delta_n, R.dn_ff);
    split(p.delta_t, R.dt_ff);
    split(p.delta_r, R.dr_ff);
    split(p.h_c, R.hc_ff);
    return R;
}

inline PView make_pview(const lub_particles *p)
{
    PView v;
    v.x = p->x; v.y = p->y; v.z = p->z;
    v.qw = p->qw; v.qx = p->qx; v.qy = p->qy; v.qz = p->qz;
    v.rpar = p->r_par; v.rperp = p->r_perp;
    v.vx = p->vx; v.vy = p->vy; v.vz = p->vz;
    v.wx = p->wx; v.wy = p->wy; v.wz = p->wz;
    v.n = p->n;
    return v;
}

inline DView make_dview(const lub_domain *d)
{
    DView v;
    for (int k = 0; k < 3; ++k) {
        v.L[k] = d->L[k];
        v.invL[k] = 1.0 / d->L[k];
        v.periodic[k] = d->periodic[k];
    }
    v.n_walls = d->n_walls;
    for (int k = 0; k < 2; ++k) {
        v.wall_z[k] = d->wall_z[k];
        v.wall_dir[k] = d->wall_dir[k];
    }
    for (int k = 0; k < 3; ++k) {
        v.Lff[k][0] = (float)d->L[k];
        v.Lff[k][1] = (float)(d->L[k] - (double)v.Lff[k][0]);
        v.invLf[k] = (float)(1.0 / d->L[k]);
    }
    v.pad = 0;
    return v;
}

// ---------------------------------------------------------------------------
// small vector type, templated on the working precision
// ---------------------------------------------------------------------------
template <typename T>
struct V3 {
    T x, y, z;
};

template <typename T>
__device__ __forceinline__ V3<T> mk(T x, T y, T z)
{
    V3<T> r;
    r.x = x; r.y = y; r.z = z;
    return r;
}
template <typename T>
__device__ __forceinline__ T dot(const V3<T> &a, const V3<T> &b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename T>
__device__ __forceinline__ V3<T> cross(const V3<T> &a, const V3<T> &b)
{
    return mk<T>(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
template <typename T>
__device__ __forceinline__ V3<T> add(const V3<T> &a, const V3<T> &b) { return mk<T>(a.x + b.x, a.y + b.y, a.z + b.z); }
template <typename T>
__device__ __forceinline__ V3<T> sub(const V3<T> &a, const V3<T> &b) { return mk<T>(a.x - b.x, a.y - b.y, a.z - b.z); }
template <typename T>
__device__ __forceinline__ V3<T> scl(T s, const V3<T> &a) { return mk<T>(s * a.x, s * a.y, s * a.z); }
template <typename T>
__device__ __forceinline__ V3<T> axpy(T s, const V3<T> &a, const V3<T> &b)  // s a + b
{
    return mk<T>(s * a.x + b.x, s * a.y + b.y, s * a.z + b.z);
}

// Double-precision reciprocal and reciprocal square root by Newton-Raphson
// from an FP32 seed (x_{k+1} = x_k (2 - a x_k) and y_{k+1} = y_k (3 - a y_k^2)/2;
// two steps take the seed's ~2^-22 relative error below double rounding).
// GB300's FP64 pipe is about 60 times slower than FP32, and these use a
// handful of FP64 multiply-adds where a full-precision division or square
// root takes several times more.  Inputs are positive, normal and within the
// float range here (squared lengths, shape factors, determinants).
__device__ __forceinline__ double rcp64(double a)
{
    double x = (double)__frcp_rn((float)a);
    x = x * fma(-a, x, 2.0);
    x = x * fma(-a, x, 2.0);
    return x;
}

__device__ __forceinline__ double rsqrt64(double a)
{
    double y = (double)rsqrtf((float)a);
    const double h = 0.5 * a;
    y = y * fma(-h * y, y, 1.5);
    y = y * fma(-h * y, y, 1.5);
    return y;
}

// Reciprocal and square root of the FP32 resistance path: the hardware
// approximations (about 1 ulp), far inside the accuracy the path needs; the
// FP64 path keeps the Newton-refined double versions.
__device__ __forceinline__ float rcp_fast(float v)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ double rcp_fast(double v) { return rcp64(v); }
__device__ __forceinline__ float sqrt_fast(float v)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

__device__ __forceinline__ float rsqrt_t(float v) { return rsqrtf(v); }
__device__ __forceinline__ double rsqrt_t(double v) { return rsqrt64(v); }
__device__ __forceinline__ float sqrt_t(float v) { return sqrtf(v); }
__device__ __forceinline__ double sqrt_t(double v) { return v > 0.0 ? v * rsqrt64(v) : 0.0; }
// (the FP32 Newton step and the FP32 axis of the pair build's records take
// the hardware reciprocal: about 1 ulp, far inside what either needs)
__device__ __forceinline__ float rcp_t(float v) { return rcp_fast(v); }
__device__ __forceinline__ double rcp_t(double v) { return rcp64(v); }
__device__ __forceinline__ double sqrt_fast(double v) { return sqrt_t(v); }

template <typename T>
__device__ __forceinline__ V3<T> normalized(const V3<T> &a)
{
    return scl(rsqrt_t(dot(a, a)), a);
}

template <typename T, typename S>
__device__ __forceinline__ V3<T> cvt(const V3<S> &a)
{
    return mk<T>((T)a.x, (T)a.y, (T)a.z);
}

// ---------------------------------------------------------------------------
// particle shape
// ---------------------------------------------------------------------------
// Axis of rotational symmetry (body z) in the lab frame: third column of the
// rotation matrix of q/|q|, q scalar first.
template <typename T>
__device__ __forceinline__ V3<T> quat_axis(float qw, float qx, float qy, float qz)
{
    T w = qw, x = qx, y = qy, z = qz;
    T s = T(2) * rcp_t(w * w + x * x + y * y + z * z);
    return mk<T>(s * (x * z + w * y), s * (y * z - w * x), T(1) - s * (x * x + y * y));
}

// The shape of a spheroid in the form M = a2 I + e o o^T with a2 = r_perp^2,
// e = r_par^2 - r_perp^2, o the symmetry axis.  Then for unit n
// sigma(n)^2 = n^T M n = a2 + e (o.n)^2 and M n = a2 n + e (o.n) o.
template <typename T>
struct Shape {
    V3<T> o;
    T a2, e;
    T rpar, rperp;
};

template <typename T>
__device__ __forceinline__ Shape<T> load_shape(const PView &P, int k)
{
    Shape<T> s;
    s.o = quat_axis<T>(__ldg(P.qw + k), __ldg(P.qx + k), __ldg(P.qy + k), __ldg(P.qz + k));
    s.rpar = (T)__ldg(P.rpar + k);
    s.rperp = (T)__ldg(P.rperp + k);
    s.a2 = s.rperp * s.rperp;
    s.e = s.rpar * s.rpar - s.a2;
    return s;
}

template <typename T>
__device__ __forceinline__ T support(const Shape<T> &s, const V3<T> &n)
{
    T c = dot(s.o, n);
    return sqrt_t(s.a2 * dot(n, n) + s.e * c * c);
}

// M n / sigma(n): offset from the centre of the surface point whose outward
// normal is n.
template <typename T>
__device__ __forceinline__ V3<T> support_offset(const Shape<T> &s, const V3<T> &n)
{
    T c = dot(s.o, n);
    T inv = rsqrt_t(s.a2 * dot(n, n) + s.e * c * c);
    return axpy(s.e * c * inv, s.o, scl(s.a2 * inv, n));
}

__device__ __forceinline__ V3<double> load_pos(const PView &P, int k)
{
    return mk<double>(__ldg(P.x + k), __ldg(P.y + k), __ldg(P.z + k));
}

// minimum image of r_j - r_i: subtract L * floor(d / L + 1/2) along periodic
// axes (d / L as d * (1/L): the two differ only within an ulp of d = +-L/2,
// far outside any interaction range)
__device__ __forceinline__ V3<double> min_image(const DView &D, V3<double> d)
{
    if (D.periodic[0]) d.x -= D.L[0] * floor(d.x * D.invL[0] + 0.5);
    if (D.periodic[1]) d.y -= D.L[1] * floor(d.y * D.invL[1] + 0.5);
    if (D.periodic[2]) d.z -= D.L[2] * floor(d.z * D.invL[2] + 0.5);
    return d;
}

__device__ __forceinline__ bool shape_ok(float rpar, float rperp)
{
    return rpar > 0.f && rperp > 0.f && isfinite(rpar) && isfinite(rperp);
}

__device__ __forceinline__ int pair_count(const int32_t *d_count, int32_t capacity)
{
    int c = *d_count;
    if (c > capacity) c = capacity;
    if (c < 0) c = 0;
    return c;
}

// ---------------------------------------------------------------------------
// launchers (defined in the .cu files)
// ---------------------------------------------------------------------------
int launch_closest(lub_ctx *ctx, const PView &P, const DView &D, const Ens &E, const lub_params &prm,
                   const int32_t *pi, const int32_t *pj, const int32_t *d_count, int32_t cap, double *n,
                   double *gap, uint8_t *status, uint8_t *iters, cudaStream_t st);
int launch_correct(lub_ctx *ctx, const PView &P, const DView &D, const Ens &E, const lub_params &prm,
                   const int32_t *pi, const int32_t *pj, const int32_t *d_count, int32_t cap, double *n, double *gap,
                   uint8_t *status, uint8_t *iters, void *FT, void *lever, void *force, void *torque, int accumulate,
                   cudaStream_t st);
// pff: the mixed mode's per-call particle records when the caller has built
// them on this stream (lub_correct), else null (built here); nh: the
// closest-point kernels' normals and gaps in float-float (lub_correct, mixed
// mode: n and gap are then not read), else null
int launch_resistance_apply(lub_ctx *ctx, const PView &P, const DView &D, const Ens &E, const lub_params &prm,
                            const int32_t *pi, const int32_t *pj, const int32_t *d_count, int32_t cap,
                            const double *n, const double *gap, uint8_t *status, void *FT, void *lever, void *force,
                            void *torque, int accumulate, cudaStream_t st, const float2 *pff = nullptr,
                            const float4 *nh = nullptr);
int launch_links(lub_ctx *ctx, const PView &P, const DView &D, const Ens &E, const int32_t *pi, const int32_t *pj,
                 const int32_t *d_count, int32_t cap, double mu, double qbar, double *force, double *torque,
                 int32_t *nlinks, cudaStream_t st);
int launch_resistance(lub_ctx *ctx, const PView &P, const DView &D, const Ens &E, const lub_params &prm,
                      const int32_t *pi, const int32_t *pj, const int32_t *d_count, int32_t cap,
                      const double *n, const double *gap, uint8_t *status, void *FT, void *lever,
                      cudaStream_t st);
int launch_apply(lub_ctx *ctx, const int32_t *pi, const int32_t *pj, const int32_t *d_count, int32_t cap,
                 const void *FT, const void *lever, int32_t n, void *force, void *torque, int precision,
                 int accumulate, int deterministic, cudaStream_t st);
int launch_pairs_build(lub_ctx *ctx, const PView &P, const DView &D, const lub_params &prm, float rmax,
                       int32_t *pi, int32_t *pj, int32_t cap, int32_t *d_count, cudaStream_t st);
// ensemble form: host domains and offsets of the nb suspensions, E their device table
int launch_pairs_build_ens(lub_ctx *ctx, const PView &P, const Ens &E, const DView *hdom, const int32_t *hoff,
                           const lub_params &prm, float rmax, int32_t *pi, int32_t *pj, int32_t cap, int32_t *d_count,
                           cudaStream_t st);
int launch_max_semi_axis(lub_ctx *ctx, const PView &P, float *h_out, cudaStream_t st);
int launch_rigid_step(lub_ctx *ctx, const lub_particles *p, const void *force, const void *torque, int precision,
                      const float *fext, const float *text, double rho, double dt, cudaStream_t st);
int launch_random_motion(lub_ctx *ctx, const lub_particles *p, uint64_t seed, int64_t step, const int64_t *step_dev,
                         int64_t *next_dev, double sig_r, double sig_t, cudaStream_t st);
int launch_carry_normals(lub_ctx *ctx, int32_t n_particles, const int32_t *qi, const int32_t *qj, const double *qn,
                         const int32_t *q_count, int32_t qcap, const int32_t *pi, const int32_t *pj,
                         const int32_t *d_count, int32_t cap, double *n, cudaStream_t st);

// device-wide exclusive scan of n int32 values (in place), total -> *d_total
// (one launch; a bounded wait that times out sets bit 2 (value 4) of *err).
// Its state, the first scan_state_words(n) words of tmp, must start at zero:
// the call clears it unless state_zeroed (an earlier kernel of the same
// stream cleared it).
int scan_exclusive(lub_ctx *ctx, int32_t *data, int64_t n, int32_t *d_total, void *tmp, size_t tmp_bytes,
                   cudaStream_t st, int32_t *err = nullptr, bool state_zeroed = false);
size_t scan_tmp_bytes(int64_t n);
inline int64_t scan_state_words(int64_t n) { return (int64_t)(scan_tmp_bytes(n) / 8); }

// Zero `bytes` of device memory with a kernel in the chain of programmatic
// dependent launches (a memset between two kernels would make the second wait
// for the memset's completion and launch): it waits for the kernel before it,
// like every kernel of a step, and releases the next one.  num_sms sizes the
// grid.
int zero_async(lub_ctx *ctx, int num_sms, void *ptr, size_t bytes, cudaStream_t st);

// zero the per-particle force and torque arrays (bytes each); one launch when
// the torque array directly follows the force array (one caller buffer)
inline int zero_force_torque(lub_ctx *ctx, void *force, void *torque, size_t bytes, cudaStream_t st)
{
    if (bytes == 0) return LUB_OK;
    if ((char *)torque == (char *)force + bytes) return zero_async(ctx, ctx->num_sms, force, 2 * bytes, st);
    int rc = zero_async(ctx, ctx->num_sms, force, bytes, st);
    if (!rc) rc = zero_async(ctx, ctx->num_sms, torque, bytes, st);
    return rc;
}

// Programmatic dependent launch (sm_90 and later).  The kernels of a step are
// launched with programmatic stream serialisation, so the hardware may
// schedule a kernel's blocks while its predecessor in the stream finishes.
// Every kernel launched that way calls pdl_wait() before anything else: it
// returns once the predecessor grid has completed and its memory operations
// are visible, so the stream order of the data is that of plain launches.
// pdl_trigger() then lets the successor be scheduled.  Launched without the
// attribute (or after a memset or a host operation), both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t st,
                              Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

inline int grid_for(int64_t work, int block, int num_sms, int per_sm = 16)
{
    int64_t g = (work + block - 1) / block;
    int64_t cap = (int64_t)num_sms * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

// launch shape of a tunable kernel (LUB_TUNE_*) for `work` items
struct Shape2 {
    int grid, block;
};
struct TuneDefault {
    int block, per_sm, max_block;
};
// defaults: grids large enough that the hardware block scheduler, not the
// grid-stride loop, balances the uneven per-pair work (Newton iteration
// counts, refinement) on large inputs
constexpr TuneDefault kTuneDefaults[LUB_TUNE_COUNT] = {
    {64, 256, 128},  // LUB_TUNE_CLOSEST_MIXED (the autotuner's choice at 1M and 32k particles)
    {32, 8, 32},     // LUB_TUNE_CLOSEST_REFINE (the autotuner's choice at 1M particles and in the ensemble)
    {128, 64, 128},  // LUB_TUNE_CLOSEST_FP64
    {64, 256, 128},  // LUB_TUNE_RESISTANCE (the autotuner's choice at 1M particles)
    {256, 32, 256},  // LUB_TUNE_APPLY
    {128, 32, 256},  // LUB_TUNE_SWEEP (the autotuner's choice at 1M particles)
};
inline Shape2 tuned_shape(const lub_ctx *ctx, int id, int64_t work)
{
    int block = kTuneDefaults[id].block, per_sm = kTuneDefaults[id].per_sm;
    if (ctx && ctx->tune_block[id] > 0) {
        block = ctx->tune_block[id];
        per_sm = ctx->tune_per_sm[id];
    }
    Shape2 s;
    s.block = block;
    s.grid = grid_for(work, block, ctx ? ctx->num_sms : 152, per_sm);
    return s;
}

// The per-call particle records of the mixed mode (five float4 per
// particle: float-float centre and axis, semi-axes, velocities; see rec_ld),
// written by one kernel on the stream; `out` (16-byte aligned) holds
// particles_ff_bytes(n) bytes.
inline size_t particles_ff_bytes(int64_t n) { return 80 * (size_t)(n > 0 ? n : 0); }
// zero16 (4 words) and zf, zt ([3][n] floats each): cleared by the same launch
int launch_particles_ff(lub_ctx *ctx, const PView &P, float2 *out, cudaStream_t st, int32_t *zero16 = nullptr,
                        float *zf = nullptr, float *zt = nullptr);

// pair build on caller-provided scratch (no allocation)
size_t pairs_scratch_bytes(int64_t n, int64_t max_cells);
int pairs_build_on_scratch(int num_sms, void *scratch, size_t scratch_bytes, int64_t max_cells, const PView &P,
                           const DView &D, const lub_params &prm, float rmax, int32_t *pi, int32_t *pj, int32_t cap,
                           int32_t *d_count, cudaStream_t st);
