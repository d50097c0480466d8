"""GB300 lubrication corrections for near-contact spheroids (arXiv:1308.6482).

A thin Python binding of the C ABI in ``include/lub.h`` (``liblub.so``,
hand-written CUDA for sm_103a).  The functions named ``lub_*`` take torch
CUDA tensors (or raw device pointers) and only marshal arguments; every step
of the computation runs in the library's kernels.  There is no CPU fallback:
if ``liblub.so`` has not been built, importing the binding succeeds but the
first call raises.

``Pipeline`` allocates the per-pair and per-particle buffers with torch and
runs the four calls of one correction step on the current CUDA stream.  With
particles made by ``make_ensemble`` (many independent suspensions back to
back) the same four calls process every suspension in one launch per stage.
"""
from ._lib import (LUB_ERR_ARG, LUB_ERR_CAPACITY, LUB_ERR_CUDA, LUB_ERR_INTERNAL, LUB_ERR_LIMIT, LUB_ERR_NOMEM, LUB_ERR_TIMEOUT,
                   LUB_FP64, LUB_MIXED, LUB_MLP_MMA_SYNC, LUB_MLP_PARAMS, LUB_MLP_TCGEN05, LUB_MODEL_FULL,
                   LUB_MODEL_NORMAL, LUB_OK, LUB_PROBE_FP32, LUB_PROBE_FP64, LUB_ST_DEGENERATE, LUB_ST_FP64,
                   LUB_ST_NOCONV, LUB_ST_OVERLAP, LUB_TRACE_APPLY, LUB_TRACE_CLOSEST, LUB_TRACE_COUNT,
                   LUB_TRACE_RESISTANCE, LUB_TRACE_SWEEP, LUB_TUNE_APPLY, LUB_TUNE_CLOSEST_FP64,
                   LUB_TUNE_CLOSEST_MIXED, LUB_TUNE_CLOSEST_REFINE, LUB_TUNE_COUNT, LUB_TUNE_RESISTANCE,
                   LUB_TUNE_SWEEP, LUB_WARM_MLP, LUB_WARM_MLP_ALL, LUB_WARM_NONE, LUB_WARM_PREVIOUS, TRACE_NAMES,
                   TUNE_NAMES, Context, DeviceParticles, LubError, Pipeline, default_params, library_path,
                   load_library, lub_apply, lub_autotune, lub_carry_normals, lub_closest_points, lub_correct,
                   lub_ctx_create, lub_ctx_destroy, lub_default_params, lub_get_launch_shape, lub_last_error,
                   lub_links, lub_mlp_adam, lub_mlp_engine, lub_mlp_features, lub_mlp_forward_backward,
                   lub_mlp_predict, lub_mlp_set, lub_pairs_build, lub_pairs_build_static, lub_probe_peak, lub_random_motion,
                   lub_resistance, lub_resistance_apply, lub_rigid_step, lub_set_launch_shape, lub_sync_status, lub_trace_enable,
                   lub_trace_read, make_domain, make_ensemble)

__all__ = [n for n in dir() if not n.startswith("_")]
