// C ABI of liblub: argument checks, context and scratch management, dispatch
// to the kernel launchers.  See include/lub.h for the contract of each call.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "lub_internal.cuh"
#include "lub_mlp.cuh"

int lub_set_error(lub_ctx *ctx, int code, const char *fmt, ...)
{
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return code;
}

int lub_check_cuda(lub_ctx *ctx, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return LUB_OK;
    return lub_set_error(ctx, LUB_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int lub_ensure_scratch(lub_ctx *ctx, size_t bytes)
{
    if (bytes <= ctx->scratch_bytes) return LUB_OK;
    size_t want = bytes + bytes / 4 + 4096;
    if (ctx->scratch) {
        cudaError_t e = cudaFree(ctx->scratch);
        ctx->scratch = nullptr;
        ctx->scratch_bytes = 0;
        if (e != cudaSuccess) return lub_check_cuda(ctx, e, "cudaFree scratch");
    }
    cudaError_t e = cudaMalloc(&ctx->scratch, want);
    if (e != cudaSuccess) {
        ctx->scratch = nullptr;
        (void)cudaGetLastError();
        return lub_set_error(ctx, LUB_ERR_NOMEM, "cudaMalloc of %zu bytes of scratch failed: %s", want,
                             cudaGetErrorString(e));
    }
    ctx->scratch_bytes = want;
    return LUB_OK;
}

int lub_upload_table(lub_ctx *ctx, int slot, const void *host, size_t bytes, cudaStream_t st, const void **dev)
{
    lub_ctx::Table &T = ctx->table[slot];
    if (T.dev && T.host.size() == bytes && memcmp(T.host.data(), host, bytes) == 0) {
        *dev = T.dev;
        return LUB_OK;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    int rc = lub_check_cuda(ctx, cudaStreamIsCapturing(st, &cs), "cudaStreamIsCapturing");
    if (rc) return rc;
    if (cs != cudaStreamCaptureStatusNone)
        return lub_set_error(ctx, LUB_ERR_ARG,
                             "the ensemble tables changed while the stream is captured: make one eager call with "
                             "this ensemble first");
    if (bytes > T.cap) {
        // a graph captured earlier may still read the old buffer: keep it until the context goes
        if (T.dev) ctx->retired.push_back(T.dev);
        T.dev = nullptr;
        T.cap = 0;
        T.host.clear();
        cudaError_t e = cudaMalloc(&T.dev, bytes);
        if (e != cudaSuccess) {
            T.dev = nullptr;
            (void)cudaGetLastError();
            return lub_set_error(ctx, LUB_ERR_NOMEM, "cudaMalloc of an ensemble table failed");
        }
        T.cap = bytes;
    }
    rc = lub_check_cuda(ctx, cudaMemcpyAsync(T.dev, host, bytes, cudaMemcpyHostToDevice, st), "table upload");
    if (!rc) rc = lub_check_cuda(ctx, cudaStreamSynchronize(st), "table upload sync");
    if (rc) return rc;
    T.host.assign((const char *)host, (const char *)host + bytes);
    *dev = T.dev;
    return LUB_OK;
}

namespace {

int check_particles(lub_ctx *ctx, const lub_particles *p, bool need_vel)
{
    if (!p) return lub_set_error(ctx, LUB_ERR_ARG, "particles is NULL");
    if (p->n < 0) return lub_set_error(ctx, LUB_ERR_ARG, "particles.n = %d < 0", p->n);
    if (p->n == 0) return LUB_OK;
    if (!p->x || !p->y || !p->z || !p->qw || !p->qx || !p->qy || !p->qz || !p->r_par || !p->r_perp)
        return lub_set_error(ctx, LUB_ERR_ARG, "a particle pose or shape array is NULL");
    if (need_vel && (!p->vx || !p->vy || !p->vz || !p->wx || !p->wy || !p->wz))
        return lub_set_error(ctx, LUB_ERR_ARG, "a particle velocity array is NULL");
    return LUB_OK;
}

int check_domain(lub_ctx *ctx, const lub_domain *d)
{
    if (!d) return lub_set_error(ctx, LUB_ERR_ARG, "domain is NULL");
    if (d->n_walls < 0 || d->n_walls > 2) return lub_set_error(ctx, LUB_ERR_ARG, "n_walls must be 0, 1 or 2");
    for (int a = 0; a < 3; ++a)
        if (!(d->L[a] > 0.0) || !isfinite(d->L[a])) return lub_set_error(ctx, LUB_ERR_ARG, "L[%d] must be > 0", a);
    for (int w = 0; w < d->n_walls; ++w) {
        if (d->wall_dir[w] != 1 && d->wall_dir[w] != -1)
            return lub_set_error(ctx, LUB_ERR_ARG, "wall_dir[%d] must be +1 or -1", w);
        if (!isfinite(d->wall_z[w])) return lub_set_error(ctx, LUB_ERR_ARG, "wall_z[%d] is not finite", w);
    }
    if (d->n_walls > 0 && d->periodic[2])
        return lub_set_error(ctx, LUB_ERR_ARG, "walls are normal to z: z cannot be periodic");
    return LUB_OK;
}

// The suspension(s) of a call: D for one suspension; in ensemble mode the
// per-suspension table E (uploaded when it changes) and, if asked, the host
// copy of each suspension's domain.
int prepare_domains(lub_ctx *ctx, const lub_particles *p, const lub_domain *dom, cudaStream_t st, DView *D, Ens *E,
                    std::vector<DView> *hdom = nullptr)
{
    E->dom = nullptr;
    E->nb = 0;
    memset(D, 0, sizeof(*D));
    if (!p->batch_offsets) {
        int rc = check_domain(ctx, dom);
        if (rc) return rc;
        *D = make_dview(dom);
        return LUB_OK;
    }
    const int nb = p->n_batches;
    if (nb < 1) return lub_set_error(ctx, LUB_ERR_ARG, "n_batches = %d must be >= 1 with batch_offsets", nb);
    if (!dom) return lub_set_error(ctx, LUB_ERR_ARG, "domain is NULL");
    const int32_t *off = p->batch_offsets;
    if (off[0] != 0 || off[nb] != p->n)
        return lub_set_error(ctx, LUB_ERR_ARG, "batch_offsets must run from 0 to n = %d", p->n);
    std::vector<EnsDom> tab((size_t)nb);
    for (int b = 0; b < nb; ++b) {
        if (off[b + 1] < off[b]) return lub_set_error(ctx, LUB_ERR_ARG, "batch_offsets decrease at %d", b);
        int rc = check_domain(ctx, dom + b);
        if (rc) {
            const std::string m = ctx->err;
            return lub_set_error(ctx, rc, "suspension %d: %s", b, m.c_str());
        }
        memset(&tab[b], 0, sizeof(EnsDom));
        tab[b].D = make_dview(dom + b);
        tab[b].p0 = off[b];
        tab[b].p1 = off[b + 1];
    }
    const void *dev = nullptr;
    int rc = lub_upload_table(ctx, 0, tab.data(), tab.size() * sizeof(EnsDom), st, &dev);
    if (rc) return rc;
    E->dom = (const EnsDom *)dev;
    E->nb = nb;
    if (hdom) {
        hdom->resize((size_t)nb);
        for (int b = 0; b < nb; ++b) (*hdom)[b] = tab[b].D;
    }
    return LUB_OK;
}

int check_params(lub_ctx *ctx, const lub_params *p)
{
    if (!p) return lub_set_error(ctx, LUB_ERR_ARG, "params is NULL");
    if (p->precision != LUB_FP64 && p->precision != LUB_MIXED)
        return lub_set_error(ctx, LUB_ERR_ARG, "precision must be LUB_FP64 or LUB_MIXED");
    if (!(p->mu >= 0.0) || !(p->delta_n > 0.0) || !(p->delta_t > 0.0) || !(p->delta_r > 0.0))
        return lub_set_error(ctx, LUB_ERR_ARG, "mu must be >= 0 and the cut-offs > 0");
    if (!(p->h_c >= 0.0) || !(p->eps_c >= 0.0)) return lub_set_error(ctx, LUB_ERR_ARG, "h_c, eps_c must be >= 0");
    if (!(p->list_cutoff >= 0.0) || !isfinite(p->list_cutoff))
        return lub_set_error(ctx, LUB_ERR_ARG, "list_cutoff must be finite and >= 0");
    if (p->max_newton < 1 || p->max_newton > 64) return lub_set_error(ctx, LUB_ERR_ARG, "max_newton must be 1..64");
    if (!(p->newton_tol > 0.0)) return lub_set_error(ctx, LUB_ERR_ARG, "newton_tol must be > 0");
    if (p->warm_start != LUB_WARM_NONE && p->warm_start != LUB_WARM_PREVIOUS && p->warm_start != LUB_WARM_MLP &&
        p->warm_start != LUB_WARM_MLP_ALL)
        return lub_set_error(ctx, LUB_ERR_ARG,
                             "warm_start must be LUB_WARM_NONE, LUB_WARM_PREVIOUS, LUB_WARM_MLP or LUB_WARM_MLP_ALL");
    if (p->model != LUB_MODEL_FULL && p->model != LUB_MODEL_NORMAL)
        return lub_set_error(ctx, LUB_ERR_ARG, "model must be LUB_MODEL_FULL or LUB_MODEL_NORMAL");
    return LUB_OK;
}

int check_pairs(lub_ctx *ctx, const int32_t *pi, const int32_t *pj, const int32_t *d_count, int32_t cap)
{
    if (cap < 0) return lub_set_error(ctx, LUB_ERR_ARG, "capacity < 0");
    if (cap > 0 && (!pi || !pj || !d_count)) return lub_set_error(ctx, LUB_ERR_ARG, "pair arrays or d_count NULL");
    return LUB_OK;
}

}  // namespace

extern "C" {

void lub_default_params(lub_params *p)
{
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->mu = 1.0 / 6.0;
    p->delta_n = 2.0 / 3.0;
    p->delta_t = 0.5;
    p->delta_r = 0.25;
    p->h_c = 0.0;
    p->eps_c = 0.0;
    p->list_cutoff = 1.0;
    p->precision = LUB_MIXED;
    p->fp64_switch = 1e-3;
    p->max_newton = 32;
    p->newton_tol = 1e-4;
    p->warm_start = LUB_WARM_NONE;
}

int lub_ctx_create(lub_ctx **out)
{
    if (!out) return LUB_ERR_ARG;
    *out = nullptr;
    lub_ctx *ctx = new (std::nothrow) lub_ctx();
    if (!ctx) return LUB_ERR_NOMEM;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_flags, 256);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_flags, 0, 256);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        delete ctx;
        return LUB_ERR_CUDA;
    }
    *out = ctx;
    return LUB_OK;
}

int lub_ctx_destroy(lub_ctx *ctx)
{
    if (!ctx) return LUB_ERR_ARG;
    cudaDeviceSynchronize();
    if (ctx->scratch) cudaFree(ctx->scratch);
    if (ctx->mlp_mem) cudaFree(ctx->mlp_mem);
    delete (MlpDevice *)ctx->mlp;
    if (ctx->d_flags) cudaFree(ctx->d_flags);
    for (auto &T : ctx->table)
        if (T.dev) cudaFree(T.dev);
    for (void *r : ctx->retired) cudaFree(r);
    lub_trace_free(ctx);
    delete ctx;
    return LUB_OK;
}

int lub_sync_status(lub_ctx *ctx, void *stream)
{
    if (!ctx) return LUB_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int32_t word = 0;
    int rc = lub_check_cuda(ctx, cudaMemcpyAsync(&word, ctx->d_flags + 1, 4, cudaMemcpyDeviceToHost, st),
                            "copy status");
    if (!rc) rc = lub_check_cuda(ctx, cudaMemsetAsync(ctx->d_flags + 1, 0, 4, st), "clear status");
    if (!rc) rc = lub_check_cuda(ctx, cudaStreamSynchronize(st), "sync");
    if (rc) return rc;
    if (word & 4) return lub_set_error(ctx, LUB_ERR_TIMEOUT, "a bounded wait of a scan look-back timed out");
    if (word & 8) return lub_set_error(ctx, LUB_ERR_TIMEOUT, "a bounded mbarrier wait of the tcgen05 network timed out");
    return LUB_OK;
}

const char *lub_last_error(const lub_ctx *ctx)
{
    if (!ctx) return "no context";
    return ctx->err.c_str();
}

int lub_pairs_build(lub_ctx *ctx, const lub_particles *p, const lub_domain *dom, const lub_params *prm,
                    int32_t *pair_i, int32_t *pair_j, int32_t capacity, int32_t *d_count, int32_t *h_count_or_null,
                    void *stream)
{
    if (!ctx) return LUB_ERR_ARG;
    ctx->err.clear();
    int rc;
    if ((rc = check_particles(ctx, p, false)) || (rc = check_params(ctx, prm))) return rc;
    if (!d_count) return lub_set_error(ctx, LUB_ERR_ARG, "d_count is NULL");
    if (capacity < 0 || (capacity > 0 && (!pair_i || !pair_j)))
        return lub_set_error(ctx, LUB_ERR_ARG, "bad pair arrays or capacity");
    // the sweep indexes its five items per particle in int32
    if (p->n > (INT32_MAX - 1024) / 5)
        return lub_set_error(ctx, LUB_ERR_ARG, "the pair build takes at most %d particles", (INT32_MAX - 1024) / 5);
    cudaStream_t st = (cudaStream_t)stream;
    PView P = make_pview(p);
    DView D;
    Ens E;
    std::vector<DView> hdom;
    if ((rc = prepare_domains(ctx, p, dom, st, &D, &E, &hdom))) return rc;
    float rmax = p->max_semi_axis;
    if (!(rmax > 0.0f)) {
        if ((rc = launch_max_semi_axis(ctx, P, &rmax, st))) return rc;
        if (!(rmax > 0.0f) && p->n > 0)
            return lub_set_error(ctx, LUB_ERR_ARG, "semi-axes must be positive and finite");
        if (!(rmax > 0.0f)) rmax = 1.0f;
    }
    const double range = 2.0 * rmax + prm->list_cutoff;
    const int nd = E.nb ? E.nb : 1;
    for (int b = 0; b < nd; ++b) {
        const DView &Db = E.nb ? hdom[b] : D;
        for (int a = 0; a < 3; ++a)
            if (Db.periodic[a] && !(Db.L[a] > 2.0 * range * (1.0 + 1e-6) + 1e-3))
                return lub_set_error(ctx, LUB_ERR_ARG,
                                     "suspension %d: periodic L[%d] = %g must exceed 2 (2 Rmax + Delta_L) = %g", b, a,
                                     Db.L[a], 2 * range);
    }
    if (E.nb)
        rc = launch_pairs_build_ens(ctx, P, E, hdom.data(), p->batch_offsets, *prm, rmax, pair_i, pair_j, capacity,
                                    d_count, st);
    else
        rc = launch_pairs_build(ctx, P, D, *prm, rmax, pair_i, pair_j, capacity, d_count, st);
    if (rc) return rc;
    if (h_count_or_null) {
        int32_t flags = 0;
        rc = lub_check_cuda(ctx, cudaMemcpyAsync(h_count_or_null, d_count, 4, cudaMemcpyDeviceToHost, st), "copy count");
        if (!rc) rc = lub_check_cuda(ctx, cudaMemcpyAsync(&flags, ctx->d_flags, 4, cudaMemcpyDeviceToHost, st), "copy flags");
        if (!rc) rc = lub_check_cuda(ctx, cudaStreamSynchronize(st), "sync");
        if (rc) return rc;
        if (flags & 4)
            return lub_set_error(ctx, LUB_ERR_TIMEOUT, "a bounded wait of the scan timed out");
        if (flags & 1)
            return lub_set_error(ctx, LUB_ERR_ARG, "a semi-axis exceeds max_semi_axis = %g (or is not finite)", rmax);
        if (flags & 16)
            return lub_set_error(ctx, LUB_ERR_INTERNAL, "the pair sweep met a cell or slot index outside its range");
        if (*h_count_or_null > capacity)
            return lub_set_error(ctx, LUB_ERR_CAPACITY, "%d candidate pairs exceed capacity %d", *h_count_or_null,
                                 capacity);
    }
    return LUB_OK;
}

int lub_closest_points(lub_ctx *ctx, const lub_particles *p, const lub_domain *dom, const lub_params *prm,
                       const int32_t *pair_i, const int32_t *pair_j, const int32_t *d_count, int32_t capacity,
                       double *n, double *gap, uint8_t *status, uint8_t *iters, void *stream)
{
    if (!ctx) return LUB_ERR_ARG;
    ctx->err.clear();
    int rc;
    if ((rc = check_particles(ctx, p, false)) || (rc = check_params(ctx, prm)) ||
        (rc = check_pairs(ctx, pair_i, pair_j, d_count, capacity)))
        return rc;
    if (capacity > 0 && (!n || !gap || !status)) return lub_set_error(ctx, LUB_ERR_ARG, "n, gap or status is NULL");
    DView D;
    Ens E;
    if ((rc = prepare_domains(ctx, p, dom, (cudaStream_t)stream, &D, &E))) return rc;
    return launch_closest(ctx, make_pview(p), D, E, *prm, pair_i, pair_j, d_count, capacity, n, gap, status, iters,
                          (cudaStream_t)stream);
}

int lub_resistance(lub_ctx *ctx, const lub_particles *p, const lub_domain *dom, const lub_params *prm,
                   const int32_t *pair_i, const int32_t *pair_j, const int32_t *d_count, int32_t capacity,
                   const double *n, const double *gap, uint8_t *status, void *FT, void *lever, void *stream)
{
    if (!ctx) return LUB_ERR_ARG;
    ctx->err.clear();
    int rc;
    if ((rc = check_particles(ctx, p, true)) || (rc = check_params(ctx, prm)) ||
        (rc = check_pairs(ctx, pair_i, pair_j, d_count, capacity)))
        return rc;
    if (capacity > 0 && (!n || !gap || !status || !FT || !lever))
        return lub_set_error(ctx, LUB_ERR_ARG, "n, gap, status, FT or lever is NULL");
    DView D;
    Ens E;
    if ((rc = prepare_domains(ctx, p, dom, (cudaStream_t)stream, &D, &E))) return rc;
    return launch_resistance(ctx, make_pview(p), D, E, *prm, pair_i, pair_j, d_count, capacity, n, gap, status, FT,
                             lever, (cudaStream_t)stream);
}

int lub_links(lub_ctx *ctx, const lub_particles *p, const lub_domain *dom, const lub_params *prm,
              const int32_t *pair_i, const int32_t *pair_j, const int32_t *d_count, int32_t capacity,
              double q_bar, double *force, double *torque, int32_t *n_links, void *stream)
{
    if (!ctx) return LUB_ERR_ARG;
    ctx->err.clear();
    int rc;
    if ((rc = check_particles(ctx, p, true)) || (rc = check_params(ctx, prm)) ||
        (rc = check_pairs(ctx, pair_i, pair_j, d_count, capacity)))
        return rc;
    if (capacity > 0 && (!force || !torque)) return lub_set_error(ctx, LUB_ERR_ARG, "force or torque is NULL");
    if (!(q_bar >= 0.0) || !isfinite(q_bar)) return lub_set_error(ctx, LUB_ERR_ARG, "q_bar must be finite and >= 0");
    DView D;
    Ens E;
    if ((rc = prepare_domains(ctx, p, dom, (cudaStream_t)stream, &D, &E))) return rc;
    return launch_links(ctx, make_pview(p), D, E, pair_i, pair_j, d_count, capacity, prm->mu, q_bar, force, torque,
                        n_links, (cudaStream_t)stream);
}

int lub_apply(lub_ctx *ctx, const int32_t *pair_i, const int32_t *pair_j, const int32_t *d_count, int32_t capacity,
              const void *FT, const void *lever, int32_t n, void *force, void *torque, int32_t precision,
              int32_t accumulate, int32_t deterministic, void *stream)
{
    if (!ctx) return LUB_ERR_ARG;
    ctx->err.clear();
    int rc;
    if ((rc = check_pairs(ctx, pair_i, pair_j, d_count, capacity))) return rc;
    if (precision != LUB_FP64 && precision != LUB_MIXED)
        return lub_set_error(ctx, LUB_ERR_ARG, "precision must be LUB_FP64 or LUB_MIXED");
    if (n < 0) return lub_set_error(ctx, LUB_ERR_ARG, "n < 0");
    if (n > 0 && (!force || !torque)) return lub_set_error(ctx, LUB_ERR_ARG, "force or torque is NULL");
    if (capacity > 0 && (!FT || !lever)) return lub_set_error(ctx, LUB_ERR_ARG, "FT or lever is NULL");
    return launch_apply(ctx, pair_i, pair_j, d_count, capacity, FT, lever, n, force, torque, precision, accumulate,
                        deterministic, (cudaStream_t)stream);
}

int lub_resistance_apply(lub_ctx *ctx, const lub_particles *p, const lub_domain *dom, const lub_params *prm,
                         const int32_t *pair_i, const int32_t *pair_j, const int32_t *d_count, int32_t capacity,
                         const double *n, const double *gap, uint8_t *status, void *FT, void *lever, void *force,
                         void *torque, int32_t accumulate, void *stream)
{
    if (!ctx) return LUB_ERR_ARG;
    ctx->err.clear();
    int rc;
    if ((rc = check_particles(ctx, p, true)) || (rc = check_params(ctx, prm)) ||
        (rc = check_pairs(ctx, pair_i, pair_j, d_count, capacity)))
        return rc;
    if (capacity > 0 && (!n || !gap || !status)) return lub_set_error(ctx, LUB_ERR_ARG, "n, gap or status is NULL");
    if (p->n > 0 && (!force || !torque)) return lub_set_error(ctx, LUB_ERR_ARG, "force or torque is NULL");
    DView D;
    Ens E;
    if ((rc = prepare_domains(ctx, p, dom, (cudaStream_t)stream, &D, &E))) return rc;
    return launch_resistance_apply(ctx, make_pview(p), D, E, *prm, pair_i, pair_j, d_count, capacity, n, gap, status,
                                   FT, lever, force, torque, accumulate, (cudaStream_t)stream);
}

int lub_correct(lub_ctx *ctx, const lub_particles *p, const lub_domain *dom, const lub_params *prm,
                const int32_t *pair_i, const int32_t *pair_j, const int32_t *d_count, int32_t capacity, double *n,
                double *gap, uint8_t *status, uint8_t *iters, void *FT, void *lever, void *force, void *torque,
                int32_t accumulate, void *stream)
{
    if (!ctx) return LUB_ERR_ARG;
    ctx->err.clear();
    int rc;
    if ((rc = check_particles(ctx, p, true)) || (rc = check_params(ctx, prm)) ||
        (rc = check_pairs(ctx, pair_i, pair_j, d_count, capacity)))
        return rc;
    if (capacity > 0 && !n) return lub_set_error(ctx, LUB_ERR_ARG, "n is NULL");
    if (p->n > 0 && (!force || !torque)) return lub_set_error(ctx, LUB_ERR_ARG, "force or torque is NULL");
    DView D;
    Ens E;
    if ((rc = prepare_domains(ctx, p, dom, (cudaStream_t)stream, &D, &E))) return rc;
    if (p->n == 0) return LUB_OK;
    return launch_correct(ctx, make_pview(p), D, E, *prm, pair_i, pair_j, d_count, capacity, n, gap, status, iters,
                          FT, lever, force, torque, accumulate, (cudaStream_t)stream);
}

int lub_rigid_step(lub_ctx *ctx, const lub_particles *p, const void *force, const void *torque, int32_t precision,
                   const float *f_ext, const float *t_ext, double density, double dt, void *stream)
{
    if (!ctx) return LUB_ERR_ARG;
    ctx->err.clear();
    int rc;
    if ((rc = check_particles(ctx, p, true))) return rc;
    if (precision != LUB_FP64 && precision != LUB_MIXED)
        return lub_set_error(ctx, LUB_ERR_ARG, "precision must be LUB_FP64 or LUB_MIXED");
    if (!(density > 0.0) || !isfinite(density)) return lub_set_error(ctx, LUB_ERR_ARG, "density must be > 0");
    if (!(dt >= 0.0) || !isfinite(dt)) return lub_set_error(ctx, LUB_ERR_ARG, "dt must be finite and >= 0");
    if (p->n > 0 && (!force || !torque)) return lub_set_error(ctx, LUB_ERR_ARG, "force or torque is NULL");
    return launch_rigid_step(ctx, p, force, torque, precision, f_ext, t_ext, density, dt, (cudaStream_t)stream);
}

int lub_random_motion(lub_ctx *ctx, const lub_particles *p, uint64_t seed, int64_t step, const int64_t *step_dev,
                      int64_t *next_dev, double sigma_r, double sigma_t, void *stream)
{
    if (!ctx) return LUB_ERR_ARG;
    ctx->err.clear();
    int rc;
    if ((rc = check_particles(ctx, p, false))) return rc;
    if (!(sigma_r >= 0.0) || !(sigma_t >= 0.0) || !isfinite(sigma_r) || !isfinite(sigma_t))
        return lub_set_error(ctx, LUB_ERR_ARG, "sigma_r and sigma_t must be finite and >= 0");
    if (step_dev && next_dev && step_dev == next_dev)
        return lub_set_error(ctx, LUB_ERR_ARG, "step_dev and next_dev must be different addresses");
    return launch_random_motion(ctx, p, seed, step, step_dev, next_dev, sigma_r, sigma_t, (cudaStream_t)stream);
}

int lub_carry_normals(lub_ctx *ctx, int32_t n_particles, const int32_t *prev_i, const int32_t *prev_j,
                      const double *prev_n, const int32_t *prev_count, int32_t prev_capacity, const int32_t *pair_i,
                      const int32_t *pair_j, const int32_t *d_count, int32_t capacity, double *n, void *stream)
{
    if (!ctx) return LUB_ERR_ARG;
    ctx->err.clear();
    int rc;
    if (n_particles < 0) return lub_set_error(ctx, LUB_ERR_ARG, "n_particles < 0");
    if ((rc = check_pairs(ctx, pair_i, pair_j, d_count, capacity))) return rc;
    if (prev_capacity < 0 || !prev_count || (prev_capacity > 0 && (!prev_i || !prev_j || !prev_n)))
        return lub_set_error(ctx, LUB_ERR_ARG, "bad previous pair list");
    if (capacity > 0 && !n) return lub_set_error(ctx, LUB_ERR_ARG, "n is NULL");
    return launch_carry_normals(ctx, n_particles, prev_i, prev_j, prev_n, prev_count, prev_capacity, pair_i, pair_j,
                                d_count, capacity, n, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// learned warm start
// ---------------------------------------------------------------------------
int lub_mlp_set(lub_ctx *ctx, const float *params, const float *mean, const float *istd, void *stream)
{
    if (!ctx) return LUB_ERR_ARG;
    ctx->err.clear();
    if (!params || !mean || !istd) return lub_set_error(ctx, LUB_ERR_ARG, "params, mean or istd is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (!ctx->mlp) {
        const size_t bw = (size_t)(8 * 32 + 64 * 32) * sizeof(uint4) + (size_t)(8 * 32) * sizeof(uint2);
        const size_t bf = (size_t)(128 + 128 + 8 + 12 + 12) * sizeof(float);
        const size_t btc = mlp_tc_image_bytes();
        void *mem = nullptr;
        cudaError_t e = cudaMalloc(&mem, ((bw + 255) & ~(size_t)255) + ((bf + 255) & ~(size_t)255) + btc);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return lub_set_error(ctx, LUB_ERR_NOMEM, "cudaMalloc of the network failed");
        }
        MlpDevice *M = new (std::nothrow) MlpDevice();
        if (!M) {
            cudaFree(mem);
            return LUB_ERR_NOMEM;
        }
        char *c = (char *)mem;
        M->F1 = (uint4 *)c;
        M->F2 = M->F1 + 8 * 32;
        M->F3 = (uint2 *)(M->F2 + 64 * 32);
        float *f = (float *)(c + ((bw + 255) & ~(size_t)255));
        M->b1 = f;
        M->b2 = f + 128;
        M->b3 = f + 256;
        M->mean = f + 264;
        M->istd = f + 276;
        M->tc_image = c + ((bw + 255) & ~(size_t)255) + ((bf + 255) & ~(size_t)255);
        ctx->mlp = M;
        ctx->mlp_mem = mem;
    }
    MlpDevice &M = *(MlpDevice *)ctx->mlp;
    int rc = launch_mlp_pack(ctx, params, M, st);
    if (!rc) rc = lub_check_cuda(ctx, cudaMemcpyAsync(M.mean, mean, 12 * sizeof(float), cudaMemcpyDeviceToDevice, st),
                                 "copy mean");
    if (!rc) rc = lub_check_cuda(ctx, cudaMemcpyAsync(M.istd, istd, 12 * sizeof(float), cudaMemcpyDeviceToDevice, st),
                                 "copy istd");
    // the tcgen05 image ends with mean and istd
    char *tail = (char *)M.tc_image + mlp_tc_image_bytes() - 24 * sizeof(float);
    if (!rc) rc = lub_check_cuda(ctx, cudaMemcpyAsync(tail, mean, 12 * sizeof(float), cudaMemcpyDeviceToDevice, st),
                                 "copy mean");
    if (!rc)
        rc = lub_check_cuda(ctx, cudaMemcpyAsync(tail + 12 * sizeof(float), istd, 12 * sizeof(float),
                                                 cudaMemcpyDeviceToDevice, st),
                            "copy istd");
    if (!rc) ctx->mlp_ready = true;
    return rc;
}

int lub_mlp_engine(lub_ctx *ctx, int32_t engine)
{
    if (!ctx) return LUB_ERR_ARG;
    ctx->err.clear();
    if (engine != LUB_MLP_MMA_SYNC && engine != LUB_MLP_TCGEN05)
        return lub_set_error(ctx, LUB_ERR_ARG, "engine must be LUB_MLP_MMA_SYNC or LUB_MLP_TCGEN05");
    ctx->mlp_engine = engine;
    return LUB_OK;
}

int lub_mlp_predict(lub_ctx *ctx, const lub_particles *p, const lub_domain *dom, const int32_t *pair_i,
                    const int32_t *pair_j, const int32_t *d_count, int32_t capacity, float *pq, void *stream)
{
    if (!ctx) return LUB_ERR_ARG;
    ctx->err.clear();
    int rc;
    if ((rc = check_particles(ctx, p, false)) || (rc = check_pairs(ctx, pair_i, pair_j, d_count, capacity))) return rc;
    if (capacity > 0 && !pq) return lub_set_error(ctx, LUB_ERR_ARG, "pq is NULL");
    DView D;
    Ens E;
    if ((rc = prepare_domains(ctx, p, dom, (cudaStream_t)stream, &D, &E))) return rc;
    return launch_mlp_start(ctx, make_pview(p), D, E, pair_i, pair_j, d_count, capacity, nullptr, pq,
                            (cudaStream_t)stream);
}

int lub_mlp_features(lub_ctx *ctx, const lub_particles *p, const lub_domain *dom, const int32_t *pair_i,
                     const int32_t *pair_j, int32_t n, const float *mean, const float *istd, float *feat, void *stream)
{
    if (!ctx) return LUB_ERR_ARG;
    ctx->err.clear();
    int rc;
    if ((rc = check_particles(ctx, p, false)) || (rc = check_domain(ctx, dom))) return rc;
    if (p->batch_offsets) return lub_set_error(ctx, LUB_ERR_ARG, "lub_mlp_features takes one suspension");
    if (n < 0 || (n > 0 && (!pair_i || !pair_j || !feat))) return lub_set_error(ctx, LUB_ERR_ARG, "bad pair arrays");
    if ((mean == nullptr) != (istd == nullptr)) return lub_set_error(ctx, LUB_ERR_ARG, "give both mean and istd or neither");
    return launch_mlp_features(ctx, make_pview(p), make_dview(dom), pair_i, pair_j, n, mean, istd, feat,
                               (cudaStream_t)stream);
}

int lub_mlp_forward_backward(lub_ctx *ctx, const float *params, const float *x, const float *target,
                             const float *weight, int32_t nb, float *grads, float *work, float *loss_rows,
                             void *stream)
{
    if (!ctx) return LUB_ERR_ARG;
    ctx->err.clear();
    if (nb <= 0 || !params || !x || !target || !grads || !work || !loss_rows)
        return lub_set_error(ctx, LUB_ERR_ARG, "bad arguments to lub_mlp_forward_backward");
    return launch_mlp_forward_backward(ctx, params, x, target, weight, nb, grads, work, loss_rows,
                                       (cudaStream_t)stream);
}

int lub_mlp_adam(lub_ctx *ctx, float *params, const float *grads, float *m, float *v, int32_t n, int32_t t, float lr,
                 float beta1, float beta2, float eps, void *stream)
{
    if (!ctx) return LUB_ERR_ARG;
    ctx->err.clear();
    if (n <= 0 || t < 1 || !params || !grads || !m || !v) return lub_set_error(ctx, LUB_ERR_ARG, "bad arguments to lub_mlp_adam");
    return launch_mlp_adam(ctx, params, grads, m, v, n, t, lr, beta1, beta2, eps, (cudaStream_t)stream);
}

}  // extern "C"
