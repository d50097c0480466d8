// Internal declarations of the learned warm start (mlp.cu).
#pragma once

#include <cuda_bf16.h>

#include "lub_internal.cuh"

// BF16 inference weights, stored in the B-fragment order of mma.m16n8k16 (one
// 16-byte load per lane gives the fragments of two adjacent 8-column n-tiles),
// and FP32 biases / feature standardisation; owned by a context.
//   F1 [8 n-tile pairs][32 lanes]             layer 1, inputs padded 12 -> 16
//   F2 [8 n-tile pairs][8 k-tiles][32 lanes]  layer 2
//   F3 [8 k-tiles][32 lanes]                  layer 3, outputs padded 4 -> 8
struct MlpDevice {
    uint4 *F1;
    uint4 *F2;
    uint2 *F3;
    float *b1, *b2, *b3;  // [128], [128], [8]
    float *mean, *istd;   // [12] each
    void *tc_image;       // the tcgen05 kernel's weights: an image of its shared-memory block
};

static_assert(LUB_MLP_PARAMS == 128 * 12 + 128 + 128 * 128 + 128 + 4 * 128 + 4, "parameter count");
static_assert(LUB_MLP_WORK_PER_SAMPLE == 6 * 128 + 2 * 4, "training scratch per sample");

int launch_mlp_start(lub_ctx *ctx, const PView &P, const DView &D, const Ens &E, const int32_t *pi, const int32_t *pj,
                     const int32_t *d_count, int32_t cap, double *n0, float *pq, cudaStream_t st);
size_t mlp_start_smem();
int launch_mlp_features(lub_ctx *ctx, const PView &P, const DView &D, const int32_t *pi, const int32_t *pj, int n,
                        const float *mean, const float *istd, float *feat, cudaStream_t st);
int launch_mlp_forward_backward(lub_ctx *ctx, const float *params, const float *x, const float *tgt,
                                const float *wgt, int M, float *grads, float *work, float *loss_rows, cudaStream_t st);
int launch_mlp_adam(lub_ctx *ctx, float *params, const float *grads, float *m, float *v, int n, int t, float lr,
                    float b1, float b2, float eps, cudaStream_t st);
int launch_mlp_pack(lub_ctx *ctx, const float *params, const MlpDevice &M, cudaStream_t st);
size_t mlp_tc_image_bytes();
