// Launch-shape autotuner: every tunable kernel is a persistent grid-stride
// loop, so its shape (threads per block, blocks per SM) changes only the
// schedule, never a result (apart from the order of atomic additions in
// lub_apply).  lub_autotune times each candidate on the caller's own step and
// keeps the fastest in the context.
#include <string.h>

#include <algorithm>
#include <vector>

#include "lub_internal.cuh"

namespace {

const int kBlocksPerSm[] = {2, 4, 8, 16, 32, 64, 128, 256};

bool valid_block(int id, int block)
{
    return block >= 32 && block % 32 == 0 && block <= kTuneDefaults[id].max_block;
}

// candidate blocks of a kernel: 32 .. its limit, powers of two
std::vector<int> blocks_of(int id)
{
    std::vector<int> v;
    for (int b = 32; b <= kTuneDefaults[id].max_block; b *= 2)
        if (b >= 64 || kTuneDefaults[id].max_block == 32) v.push_back(b);
    return v;
}

}  // namespace

extern "C" {

int lub_get_launch_shape(const lub_ctx *ctx, int32_t kernel, int32_t *block, int32_t *blocks_per_sm)
{
    if (!ctx || kernel < 0 || kernel >= LUB_TUNE_COUNT || !block || !blocks_per_sm) return LUB_ERR_ARG;
    *block = ctx->tune_block[kernel];
    *blocks_per_sm = ctx->tune_per_sm[kernel];
    return LUB_OK;
}

int lub_set_launch_shape(lub_ctx *ctx, int32_t kernel, int32_t block, int32_t blocks_per_sm)
{
    if (!ctx) return LUB_ERR_ARG;
    if (kernel < 0 || kernel >= LUB_TUNE_COUNT) return lub_set_error(ctx, LUB_ERR_ARG, "no tunable kernel %d", kernel);
    if (block == 0 && blocks_per_sm == 0) {
        ctx->tune_block[kernel] = 0;
        ctx->tune_per_sm[kernel] = 0;
        return LUB_OK;
    }
    if (!valid_block(kernel, block) || blocks_per_sm < 1 || blocks_per_sm > 256)
        return lub_set_error(ctx, LUB_ERR_ARG, "shape (%d, %d) not allowed for kernel %d", block, blocks_per_sm,
                             kernel);
    ctx->tune_block[kernel] = block;
    ctx->tune_per_sm[kernel] = blocks_per_sm;
    return LUB_OK;
}

int lub_autotune(lub_ctx *ctx, const lub_particles *p, const lub_domain *dom, const lub_params *prm,
                 int32_t *pair_i, int32_t *pair_j, int32_t capacity, int32_t *d_count, double *n, double *gap,
                 uint8_t *status, uint8_t *iters, void *FT, void *lever, void *force, void *torque, int32_t reps,
                 void *stream)
{
    if (!ctx) return LUB_ERR_ARG;
    if (!p || !prm) return lub_set_error(ctx, LUB_ERR_ARG, "particles or params is NULL");
    if (reps < 1) return lub_set_error(ctx, LUB_ERR_ARG, "reps must be >= 1");
    cudaStream_t st = (cudaStream_t)stream;
    // one step first: the pair list the other calls read, and argument checks
    int32_t h_count = 0;
    int rc = lub_pairs_build(ctx, p, dom, prm, pair_i, pair_j, capacity, d_count, &h_count, stream);
    if (rc) return rc;
    auto run = [&](int id) -> int {
        switch (id) {
        case LUB_TUNE_SWEEP:
            return lub_pairs_build(ctx, p, dom, prm, pair_i, pair_j, capacity, d_count, nullptr, stream);
        case LUB_TUNE_CLOSEST_MIXED:
        case LUB_TUNE_CLOSEST_REFINE:
        case LUB_TUNE_CLOSEST_FP64:
            return lub_closest_points(ctx, p, dom, prm, pair_i, pair_j, d_count, capacity, n, gap, status, iters,
                                      stream);
        case LUB_TUNE_RESISTANCE:
            return lub_resistance(ctx, p, dom, prm, pair_i, pair_j, d_count, capacity, n, gap, status, FT, lever,
                                  stream);
        default:
            return lub_apply(ctx, pair_i, pair_j, d_count, capacity, FT, lever, p->n, force, torque, prm->precision,
                             0, 0, stream);
        }
    };
    // the closest-point kernels of the other precision are not run by this step
    const int ids_mixed[] = {LUB_TUNE_SWEEP, LUB_TUNE_CLOSEST_MIXED, LUB_TUNE_CLOSEST_REFINE, LUB_TUNE_RESISTANCE,
                             LUB_TUNE_APPLY};
    const int ids_fp64[] = {LUB_TUNE_SWEEP, LUB_TUNE_CLOSEST_FP64, LUB_TUNE_RESISTANCE, LUB_TUNE_APPLY};
    const int *ids = prm->precision == LUB_MIXED ? ids_mixed : ids_fp64;
    const int nid = prm->precision == LUB_MIXED ? 5 : 4;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((rc = lub_check_cuda(ctx, cudaEventCreate(&e0), "event")) ||
        (rc = lub_check_cuda(ctx, cudaEventCreate(&e1), "event")))
        return rc;
    // valid closest-point and resistance outputs for the later candidates
    if (!rc) rc = run(LUB_TUNE_CLOSEST_FP64);
    if (!rc) rc = run(LUB_TUNE_RESISTANCE);
    for (int q = 0; q < nid && !rc; ++q) {
        const int id = ids[q];
        float best = 1e30f;
        int bb = 0, bp = 0;
        for (int block : blocks_of(id)) {
            for (int per_sm : kBlocksPerSm) {
                if (block * per_sm > 32768) continue;  // 16 waves of resident threads: as good as any larger grid
                // the sweep runs one thread per item: its grid follows from the block
                if (id == LUB_TUNE_SWEEP && per_sm != kBlocksPerSm[0]) continue;
                ctx->tune_block[id] = block;
                ctx->tune_per_sm[id] = per_sm;
                if ((rc = run(id))) break;  // warm-up
                std::vector<float> t;
                for (int r = 0; r < reps && !rc; ++r) {
                    rc = lub_check_cuda(ctx, cudaEventRecord(e0, st), "event record");
                    if (!rc) rc = run(id);
                    if (!rc) rc = lub_check_cuda(ctx, cudaEventRecord(e1, st), "event record");
                    if (!rc) rc = lub_check_cuda(ctx, cudaEventSynchronize(e1), "event sync");
                    float ms = 0.f;
                    if (!rc) rc = lub_check_cuda(ctx, cudaEventElapsedTime(&ms, e0, e1), "event time");
                    t.push_back(ms);
                }
                if (rc) break;
                std::sort(t.begin(), t.end());
                const float med = t[t.size() / 2];
                if (med < best) {
                    best = med;
                    bb = block;
                    bp = per_sm;
                }
            }
            if (rc) break;
        }
        ctx->tune_block[id] = bb;
        ctx->tune_per_sm[id] = bp;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        for (int id = 0; id < LUB_TUNE_COUNT; ++id) ctx->tune_block[id] = ctx->tune_per_sm[id] = 0;
        return rc;
    }
    // leave the outputs of one full step with the chosen shapes
    if (!rc) rc = run(LUB_TUNE_SWEEP);
    if (!rc) rc = run(LUB_TUNE_CLOSEST_FP64);
    if (!rc) rc = run(LUB_TUNE_RESISTANCE);
    if (!rc) rc = run(LUB_TUNE_APPLY);
    if (!rc) rc = lub_check_cuda(ctx, cudaStreamSynchronize(st), "sync");
    return rc;
}

}  // extern "C"
