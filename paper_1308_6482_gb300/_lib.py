"""ctypes binding of liblub (include/lub.h).  Argument marshalling only."""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# LUB_LIBRARY selects another build of the library (the tests of the bounded
# waits load the test build, liblub_testing.so, in a process of their own)
_SO = os.environ.get("LUB_LIBRARY") or os.path.join(_HERE, "liblub.so")

LUB_OK = 0
LUB_ERR_ARG = -1
LUB_ERR_CAPACITY = -2
LUB_ERR_CUDA = -3
LUB_ERR_TIMEOUT = -4
LUB_ERR_NOMEM = -5
LUB_ERR_LIMIT = -6
LUB_ERR_INTERNAL = -7
LUB_STATIC_MAX_PARTICLES = 65536
LUB_STATIC_MAX_CELLS = 262144
LUB_FP64 = 0
LUB_MIXED = 1
LUB_WARM_NONE = 0
LUB_WARM_PREVIOUS = 1
LUB_WARM_MLP = 2
LUB_WARM_MLP_ALL = 3
LUB_MLP_MMA_SYNC = 0
LUB_MLP_TCGEN05 = 1
LUB_MODEL_FULL = 0
LUB_MODEL_NORMAL = 1
LUB_MLP_PARAMS = 18692
LUB_MLP_WORK_PER_SAMPLE = 776
LUB_ST_OVERLAP = 1
LUB_ST_NOCONV = 2
LUB_ST_DEGENERATE = 4
LUB_ST_FP64 = 8
LUB_TUNE_CLOSEST_MIXED = 0
LUB_TUNE_CLOSEST_REFINE = 1
LUB_TUNE_CLOSEST_FP64 = 2
LUB_TUNE_RESISTANCE = 3
LUB_TUNE_APPLY = 4
LUB_TUNE_SWEEP = 5
LUB_TUNE_COUNT = 6
LUB_TRACE_SWEEP = 0
LUB_TRACE_CLOSEST = 1
LUB_TRACE_RESISTANCE = 2
LUB_TRACE_APPLY = 3
LUB_TRACE_COUNT = 4
TRACE_NAMES = ("sweep", "closest", "resistance", "apply")
LUB_PROBE_FP32 = 0
LUB_PROBE_FP64 = 1
TUNE_NAMES = ("closest_mixed", "closest_refine", "closest_fp64", "resistance", "apply", "sweep")

_P_FIELDS = ("x", "y", "z", "qw", "qx", "qy", "qz", "r_par", "r_perp", "vx", "vy", "vz", "wx", "wy", "wz")


class LubError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("liblub error %d: %s" % (code, msg))
        self.code = code


class lub_particles(ctypes.Structure):
    _fields_ = [(f, ctypes.c_void_p) for f in _P_FIELDS] + [("n", ctypes.c_int32),
                                                             ("max_semi_axis", ctypes.c_float),
                                                             ("batch_offsets", ctypes.c_void_p),
                                                             ("n_batches", ctypes.c_int32)]


class lub_domain(ctypes.Structure):
    _fields_ = [("L", ctypes.c_double * 3), ("periodic", ctypes.c_int32 * 3), ("n_walls", ctypes.c_int32),
                ("wall_z", ctypes.c_double * 2), ("wall_dir", ctypes.c_int32 * 2)]


class lub_params(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_double), ("delta_n", ctypes.c_double), ("delta_t", ctypes.c_double),
                ("delta_r", ctypes.c_double), ("h_c", ctypes.c_double), ("eps_c", ctypes.c_double),
                ("list_cutoff", ctypes.c_double), ("precision", ctypes.c_int32), ("fp64_switch", ctypes.c_double),
                ("max_newton", ctypes.c_int32), ("newton_tol", ctypes.c_double), ("warm_start", ctypes.c_int32),
                ("model", ctypes.c_int32)]


# every exported symbol of include/lub.h
EXPORTS = ("lub_default_params", "lub_ctx_create", "lub_ctx_destroy", "lub_last_error", "lub_pairs_build",
           "lub_closest_points", "lub_resistance", "lub_apply", "lub_pairs_build_static", "lub_mlp_set",
           "lub_mlp_predict", "lub_mlp_features", "lub_mlp_forward_backward", "lub_mlp_adam", "lub_autotune",
           "lub_get_launch_shape", "lub_set_launch_shape", "lub_carry_normals", "lub_correct",
           "lub_resistance_apply", "lub_rigid_step", "lub_mlp_engine", "lub_links", "lub_trace_enable",
           "lub_trace_read", "lub_probe_peak", "lub_random_motion", "lub_sync_status")

_lib = None


def library_path():
    return _SO


def load_library():
    """Load liblub.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_SO):
        raise RuntimeError("liblub.so not found at %s: build it with paper_1308_6482_gb300.build.build() "
                           "(nvcc, sm_103a); there is no CPU fallback" % _SO)
    lib = ctypes.CDLL(_SO)
    P = ctypes.POINTER
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    lib.lub_default_params.restype = None
    lib.lub_default_params.argtypes = [P(lub_params)]
    lib.lub_ctx_create.restype = ctypes.c_int
    lib.lub_ctx_create.argtypes = [P(vp)]
    lib.lub_ctx_destroy.restype = ctypes.c_int
    lib.lub_ctx_destroy.argtypes = [vp]
    lib.lub_last_error.restype = ctypes.c_char_p
    lib.lub_last_error.argtypes = [vp]
    lib.lub_pairs_build.restype = ctypes.c_int
    lib.lub_pairs_build.argtypes = [vp, P(lub_particles), P(lub_domain), P(lub_params), vp, vp, i32, vp,
                                    P(i32), vp]
    lib.lub_closest_points.restype = ctypes.c_int
    lib.lub_closest_points.argtypes = [vp, P(lub_particles), P(lub_domain), P(lub_params), vp, vp, vp, i32, vp,
                                       vp, vp, vp, vp]
    lib.lub_resistance.restype = ctypes.c_int
    lib.lub_links.restype = i32
    lib.lub_links.argtypes = [vp, P(lub_particles), P(lub_domain), P(lub_params), vp, vp, vp, i32, ctypes.c_double,
                              vp, vp, vp, vp]
    lib.lub_resistance.argtypes = [vp, P(lub_particles), P(lub_domain), P(lub_params), vp, vp, vp, i32, vp, vp,
                                   vp, vp, vp, vp]
    lib.lub_apply.restype = ctypes.c_int
    lib.lub_apply.argtypes = [vp, vp, vp, vp, i32, vp, vp, i32, vp, vp, i32, i32, i32, vp]
    f32 = ctypes.c_float
    lib.lub_mlp_set.restype = ctypes.c_int
    lib.lub_mlp_set.argtypes = [vp, vp, vp, vp, vp]
    lib.lub_mlp_predict.restype = ctypes.c_int
    lib.lub_mlp_predict.argtypes = [vp, P(lub_particles), P(lub_domain), vp, vp, vp, i32, vp, vp]
    lib.lub_mlp_features.restype = ctypes.c_int
    lib.lub_mlp_features.argtypes = [vp, P(lub_particles), P(lub_domain), vp, vp, i32, vp, vp, vp, vp]
    lib.lub_mlp_forward_backward.restype = ctypes.c_int
    lib.lub_mlp_forward_backward.argtypes = [vp, vp, vp, vp, vp, i32, vp, vp, vp, vp]
    lib.lub_mlp_adam.restype = ctypes.c_int
    lib.lub_mlp_adam.argtypes = [vp, vp, vp, vp, vp, i32, i32, f32, f32, f32, f32, vp]
    lib.lub_autotune.restype = ctypes.c_int
    lib.lub_autotune.argtypes = [vp, P(lub_particles), P(lub_domain), P(lub_params), vp, vp, i32, vp, vp, vp, vp, vp,
                                 vp, vp, vp, vp, i32, vp]
    lib.lub_mlp_engine.restype = ctypes.c_int
    lib.lub_mlp_engine.argtypes = [vp, i32]
    lib.lub_rigid_step.restype = ctypes.c_int
    lib.lub_rigid_step.argtypes = [vp, P(lub_particles), vp, vp, i32, vp, vp, ctypes.c_double, ctypes.c_double, vp]
    lib.lub_resistance_apply.restype = ctypes.c_int
    lib.lub_resistance_apply.argtypes = [vp, P(lub_particles), P(lub_domain), P(lub_params), vp, vp, vp, i32, vp, vp,
                                         vp, vp, vp, vp, vp, i32, vp]
    lib.lub_correct.restype = ctypes.c_int
    lib.lub_correct.argtypes = [vp, P(lub_particles), P(lub_domain), P(lub_params), vp, vp, vp, i32, vp, vp, vp, vp,
                                vp, vp, vp, vp, i32, vp]
    lib.lub_carry_normals.restype = ctypes.c_int
    lib.lub_carry_normals.argtypes = [vp, i32, vp, vp, vp, vp, i32, vp, vp, vp, i32, vp, vp]
    lib.lub_get_launch_shape.restype = ctypes.c_int
    lib.lub_get_launch_shape.argtypes = [vp, i32, P(i32), P(i32)]
    lib.lub_set_launch_shape.restype = ctypes.c_int
    lib.lub_set_launch_shape.argtypes = [vp, i32, i32, i32]
    lib.lub_pairs_build_static.restype = ctypes.c_int
    lib.lub_pairs_build_static.argtypes = [P(lub_particles), P(lub_domain), P(lub_params), vp, vp, i32, vp, vp]
    lib.lub_trace_enable.restype = ctypes.c_int
    lib.lub_trace_enable.argtypes = [vp, i32]
    lib.lub_trace_read.restype = ctypes.c_int
    lib.lub_trace_read.argtypes = [vp, i32, P(ctypes.c_double), P(ctypes.c_int64)]
    lib.lub_sync_status.restype = ctypes.c_int
    lib.lub_sync_status.argtypes = [vp, vp]
    lib.lub_random_motion.restype = ctypes.c_int
    lib.lub_random_motion.argtypes = [vp, P(lub_particles), ctypes.c_uint64, ctypes.c_int64, vp, vp,
                                      ctypes.c_double, ctypes.c_double, vp]
    lib.lub_probe_peak.restype = ctypes.c_int
    lib.lub_probe_peak.argtypes = [vp, i32, P(ctypes.c_double), vp]
    _lib = lib
    return lib


def _ptr(t):
    """Device (or host) pointer of a tensor / numpy array / int / None."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    raise TypeError(type(t))


def _dom(domain):
    """A lub_domain by reference, or an ensemble's array of them (decays to a pointer)."""
    return domain if isinstance(domain, ctypes.Array) else ctypes.byref(domain)


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(ctx, rc):
    if rc != LUB_OK:
        msg = load_library().lub_last_error(ctx).decode()
        raise LubError(rc, msg)
    return rc


# ---------------------------------------------------------------------------
# the C entry points, same names
# ---------------------------------------------------------------------------
def lub_default_params():
    p = lub_params()
    load_library().lub_default_params(ctypes.byref(p))
    return p


def lub_ctx_create():
    h = ctypes.c_void_p()
    rc = load_library().lub_ctx_create(ctypes.byref(h))
    if rc != LUB_OK:
        raise LubError(rc, "lub_ctx_create failed")
    return h.value


def lub_ctx_destroy(ctx):
    return load_library().lub_ctx_destroy(ctx)


def lub_last_error(ctx):
    return load_library().lub_last_error(ctx).decode()


def lub_pairs_build(ctx, particles, domain, params, pair_i, pair_j, capacity, d_count, h_count=None,
                    stream=None, check=True):
    hc = ctypes.c_int32(0)
    rc = load_library().lub_pairs_build(ctx, ctypes.byref(particles), _dom(domain), ctypes.byref(params),
                                        _ptr(pair_i), _ptr(pair_j), int(capacity), _ptr(d_count),
                                        ctypes.byref(hc) if h_count else None, _stream(stream))
    if check and rc not in (LUB_OK, LUB_ERR_CAPACITY):
        _check(ctx, rc)
    return rc, (hc.value if h_count else None)


def lub_pairs_build_static(particles, domain, params, pair_i, pair_j, capacity, d_count, stream=None):
    """Pair build on the library's static scratch (no allocation); returns the code."""
    return load_library().lub_pairs_build_static(ctypes.byref(particles), _dom(domain),
                                                 ctypes.byref(params), _ptr(pair_i), _ptr(pair_j), int(capacity),
                                                 _ptr(d_count), _stream(stream))


def lub_mlp_set(ctx, params, mean, istd, stream=None):
    return _check(ctx, load_library().lub_mlp_set(ctx, _ptr(params), _ptr(mean), _ptr(istd), _stream(stream)))


def lub_mlp_predict(ctx, particles, domain, pair_i, pair_j, d_count, capacity, pq, stream=None):
    return _check(ctx, load_library().lub_mlp_predict(ctx, ctypes.byref(particles), _dom(domain),
                                                      _ptr(pair_i), _ptr(pair_j), _ptr(d_count), int(capacity),
                                                      _ptr(pq), _stream(stream)))


def lub_mlp_features(ctx, particles, domain, pair_i, pair_j, n, mean, istd, feat, stream=None):
    return _check(ctx, load_library().lub_mlp_features(ctx, ctypes.byref(particles), _dom(domain),
                                                       _ptr(pair_i), _ptr(pair_j), int(n), _ptr(mean), _ptr(istd),
                                                       _ptr(feat), _stream(stream)))


def lub_mlp_forward_backward(ctx, params, x, target, weight, nb, grads, work, loss_rows, stream=None):
    return _check(ctx, load_library().lub_mlp_forward_backward(ctx, _ptr(params), _ptr(x), _ptr(target),
                                                               _ptr(weight), int(nb),
                                                               _ptr(grads), _ptr(work), _ptr(loss_rows),
                                                               _stream(stream)))


def lub_mlp_adam(ctx, params, grads, m, v, n, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    return _check(ctx, load_library().lub_mlp_adam(ctx, _ptr(params), _ptr(grads), _ptr(m), _ptr(v), int(n), int(t),
                                                   float(lr), float(beta1), float(beta2), float(eps),
                                                   _stream(stream)))


def lub_closest_points(ctx, particles, domain, params, pair_i, pair_j, d_count, capacity, n, gap, status,
                       iters=None, stream=None):
    return _check(ctx, load_library().lub_closest_points(
        ctx, ctypes.byref(particles), _dom(domain), ctypes.byref(params), _ptr(pair_i), _ptr(pair_j),
        _ptr(d_count), int(capacity), _ptr(n), _ptr(gap), _ptr(status), _ptr(iters), _stream(stream)))


def lub_resistance(ctx, particles, domain, params, pair_i, pair_j, d_count, capacity, n, gap, status, FT, lever,
                   stream=None):
    return _check(ctx, load_library().lub_resistance(
        ctx, ctypes.byref(particles), _dom(domain), ctypes.byref(params), _ptr(pair_i), _ptr(pair_j),
        _ptr(d_count), int(capacity), _ptr(n), _ptr(gap), _ptr(status), _ptr(FT), _ptr(lever), _stream(stream)))


def lub_links(ctx, particles, domain, params, pair_i, pair_j, d_count, capacity, q_bar, force, torque, n_links=None,
              stream=None):
    return _check(ctx, load_library().lub_links(
        ctx, ctypes.byref(particles), _dom(domain), ctypes.byref(params), _ptr(pair_i), _ptr(pair_j),
        _ptr(d_count), int(capacity), float(q_bar), _ptr(force), _ptr(torque), _ptr(n_links), _stream(stream)))


def lub_apply(ctx, pair_i, pair_j, d_count, capacity, FT, lever, n, force, torque, precision, accumulate=0,
              deterministic=0, stream=None):
    return _check(ctx, load_library().lub_apply(
        ctx, _ptr(pair_i), _ptr(pair_j), _ptr(d_count), int(capacity), _ptr(FT), _ptr(lever), int(n), _ptr(force),
        _ptr(torque), int(precision), int(accumulate), int(deterministic), _stream(stream)))


def lub_autotune(ctx, particles, domain, params, pair_i, pair_j, capacity, d_count, n, gap, status, iters, FT,
                 lever, force, torque, reps=3, stream=None):
    return _check(ctx, load_library().lub_autotune(
        ctx, ctypes.byref(particles), _dom(domain), ctypes.byref(params), _ptr(pair_i), _ptr(pair_j), int(capacity),
        _ptr(d_count), _ptr(n), _ptr(gap), _ptr(status), _ptr(iters), _ptr(FT), _ptr(lever), _ptr(force),
        _ptr(torque), int(reps), _stream(stream)))


def lub_mlp_engine(ctx, engine):
    if isinstance(engine, str):
        engine = {"mma_sync": LUB_MLP_MMA_SYNC, "tcgen05": LUB_MLP_TCGEN05}[engine]
    return _check(ctx, load_library().lub_mlp_engine(ctx, int(engine)))


def lub_rigid_step(ctx, particles, force, torque, precision, f_ext, t_ext, density, dt, stream=None):
    return _check(ctx, load_library().lub_rigid_step(ctx, ctypes.byref(particles), _ptr(force), _ptr(torque),
                                                     int(precision), _ptr(f_ext), _ptr(t_ext), float(density),
                                                     float(dt), _stream(stream)))


def lub_resistance_apply(ctx, particles, domain, params, pair_i, pair_j, d_count, capacity, n, gap, status, FT,
                         lever, force, torque, accumulate=0, stream=None):
    return _check(ctx, load_library().lub_resistance_apply(
        ctx, ctypes.byref(particles), _dom(domain), ctypes.byref(params), _ptr(pair_i), _ptr(pair_j), _ptr(d_count),
        int(capacity), _ptr(n), _ptr(gap), _ptr(status), _ptr(FT), _ptr(lever), _ptr(force), _ptr(torque),
        int(accumulate), _stream(stream)))


def lub_correct(ctx, particles, domain, params, pair_i, pair_j, d_count, capacity, n, gap, status, iters, FT, lever,
                force, torque, accumulate=0, stream=None):
    return _check(ctx, load_library().lub_correct(
        ctx, ctypes.byref(particles), _dom(domain), ctypes.byref(params), _ptr(pair_i), _ptr(pair_j), _ptr(d_count),
        int(capacity), _ptr(n), _ptr(gap), _ptr(status), _ptr(iters), _ptr(FT), _ptr(lever), _ptr(force),
        _ptr(torque), int(accumulate), _stream(stream)))


def lub_carry_normals(ctx, n_particles, prev_i, prev_j, prev_n, prev_count, prev_capacity, pair_i, pair_j, d_count,
                      capacity, n, stream=None):
    return _check(ctx, load_library().lub_carry_normals(
        ctx, int(n_particles), _ptr(prev_i), _ptr(prev_j), _ptr(prev_n), _ptr(prev_count), int(prev_capacity),
        _ptr(pair_i),
        _ptr(pair_j), _ptr(d_count), int(capacity), _ptr(n), _stream(stream)))


def lub_get_launch_shape(ctx, kernel):
    b, p = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(ctx, load_library().lub_get_launch_shape(ctx, int(kernel), ctypes.byref(b), ctypes.byref(p)))
    return b.value, p.value


def lub_set_launch_shape(ctx, kernel, block, blocks_per_sm):
    return _check(ctx, load_library().lub_set_launch_shape(ctx, int(kernel), int(block), int(blocks_per_sm)))


def lub_sync_status(ctx, stream=None):
    """Raises LubError(LUB_ERR_TIMEOUT) if a bounded device wait timed out since the last check."""
    return _check(ctx, load_library().lub_sync_status(ctx, _stream(stream)))


def lub_trace_enable(ctx, on):
    return _check(ctx, load_library().lub_trace_enable(ctx, int(bool(on))))


def lub_trace_read(ctx, kernel):
    """(total milliseconds, launches) of traced kernel `kernel` since the last read."""
    ms, n = ctypes.c_double(0.0), ctypes.c_int64(0)
    _check(ctx, load_library().lub_trace_read(ctx, int(kernel), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def lub_random_motion(ctx, particles, seed, step, sigma_r, sigma_t, step_dev=None, next_dev=None, stream=None):
    return _check(ctx, load_library().lub_random_motion(ctx, ctypes.byref(particles), int(seed) & ((1 << 64) - 1),
                                                        int(step), _ptr(step_dev), _ptr(next_dev), float(sigma_r),
                                                        float(sigma_t), _stream(stream)))


def lub_probe_peak(ctx, pipe, stream=None):
    """Sustained FMA throughput of the FP32 (pipe 0) or FP64 (pipe 1) pipe, TFLOP/s."""
    t = ctypes.c_double(0.0)
    _check(ctx, load_library().lub_probe_peak(ctx, int(pipe), ctypes.byref(t), _stream(stream)))
    return t.value


# ---------------------------------------------------------------------------
# conveniences: device particles, domain, params, a context, one step
# ---------------------------------------------------------------------------
def default_params(**kw):
    p = lub_default_params()
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": LUB_FP64, "mixed": LUB_MIXED}[v]
        if k == "warm_start" and isinstance(v, str):
            v = {"none": LUB_WARM_NONE, "previous": LUB_WARM_PREVIOUS, "mlp": LUB_WARM_MLP,
                 "mlp_all": LUB_WARM_MLP_ALL}[v]
        if k == "model" and isinstance(v, str):
            v = {"full": LUB_MODEL_FULL, "normal": LUB_MODEL_NORMAL}[v]
        setattr(p, k, v)
    return p


def make_domain(dom):
    """lub_domain of a domain dict; for a list of dicts (an ensemble), an array of them."""
    if isinstance(dom, (list, tuple)):
        arr = (lub_domain * len(dom))()
        for b, one in enumerate(dom):
            arr[b] = make_domain(one)
        return arr
    d = lub_domain()
    for k in range(3):
        d.L[k] = float(dom["L"][k])
        d.periodic[k] = int(bool(dom["periodic"][k]))
    walls = dom.get("walls", [])
    d.n_walls = len(walls)
    for w, (z, s) in enumerate(walls):
        d.wall_z[w] = float(z)
        d.wall_dir[w] = int(s)
    return d


def make_ensemble(suspensions):
    """Concatenate independent suspensions [(parts, dom), ...] for ensemble mode.

    Returns (parts, doms, offsets): the particle arrays back to back, the list
    of domain dicts, and the host offsets [n_batches + 1] (suspension b owns
    particles offsets[b] .. offsets[b+1]-1)."""
    offsets = np.zeros(len(suspensions) + 1, np.int32)
    for b, (p, _) in enumerate(suspensions):
        offsets[b + 1] = offsets[b] + len(p["x"])
    keys = [k for k in _P_FIELDS if all(k in p for p, _ in suspensions)]
    parts = {k: np.concatenate([np.asarray(p[k]) for p, _ in suspensions]) for k in keys}
    return parts, [d for _, d in suspensions], offsets


def _packed_layout(n):
    """Byte offsets of the 15 particle arrays in one buffer: the three float64
    centre arrays first, then the float32 ones, each 256-byte aligned."""
    lay, off = {}, 0
    for f in _P_FIELDS:
        dt = np.dtype(np.float64) if f in ("x", "y", "z") else np.dtype(np.float32)
        lay[f] = (off, dt)
        off += (n * dt.itemsize + 255) // 256 * 256
    return lay, max(off, 256)


class DeviceParticles:
    """Particle arrays on the GPU (float64 centres, float32 the rest)."""

    def __init__(self, parts, device="cuda", max_semi_axis=None, batch_offsets=None, packed=False):
        """packed=True lays the 15 arrays out as views of one device buffer
        (self.blob; layout self.layout), so one copy moves a whole pose and
        velocity update: see host_blob()."""
        import torch
        n = len(parts["x"])
        self.n = n
        # ensemble mode: host offsets [n_batches + 1], kept alive with the struct
        self.offsets = None if batch_offsets is None else np.ascontiguousarray(batch_offsets, np.int32)
        self.t = {}
        self.blob = None
        self.layout = None
        if packed:
            self.layout, total = _packed_layout(n)
            self.blob = torch.empty(total, dtype=torch.uint8, device=device)
            for f in _P_FIELDS:
                off, dt = self.layout[f]
                self.t[f] = self.blob[off:off + n * dt.itemsize].view(torch.float64 if dt == np.float64
                                                                        else torch.float32)
            self.blob.copy_(torch.as_tensor(self.host_blob(parts)))
        for f in _P_FIELDS:
            if packed:
                break
            a = parts.get(f)
            if a is None:
                a = np.zeros(n)
            dt = torch.float64 if f in ("x", "y", "z") else torch.float32
            self.t[f] = torch.as_tensor(np.ascontiguousarray(a), dtype=dt).to(device)
        if max_semi_axis is None:
            max_semi_axis = float(max(np.max(parts["r_par"]), np.max(parts["r_perp"]))) if n else 1.0
        self.max_semi_axis = float(max_semi_axis)
        self.refresh()

    def host_blob(self, parts, out=None):
        """The packed layout of `parts` as host bytes (into `out`, e.g. a pinned
        uint8 tensor, if given)."""
        import torch
        _, total = _packed_layout(self.n)
        buf = np.zeros(total, np.uint8) if out is None else out.numpy()
        for f in _P_FIELDS:
            off, dt = self.layout[f]
            a = parts.get(f)
            a = np.zeros(self.n, dt) if a is None else np.ascontiguousarray(a, dt)
            buf[off:off + self.n * dt.itemsize] = a.view(np.uint8)
        return out if out is not None else torch.as_tensor(buf)

    def refresh(self):
        off = self.offsets
        self.c = lub_particles(*[self.t[f].data_ptr() for f in _P_FIELDS], self.n, self.max_semi_axis,
                               None if off is None else off.ctypes.data, 0 if off is None else len(off) - 1)


class Context:
    def __init__(self):
        self.h = lub_ctx_create()

    def close(self):
        if self.h:
            lub_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Pipeline:
    """Buffers and the four calls of one correction step for one suspension."""

    def __init__(self, parts, dom, params=None, capacity=None, device="cuda", ctx=None):
        import torch
        self.torch = torch
        self.P = parts if isinstance(parts, DeviceParticles) else DeviceParticles(parts, device)
        self.D = make_domain(dom)
        self.prm = params if params is not None else default_params()
        self.ctx = ctx or Context()
        self.n = self.P.n
        if capacity is None:
            capacity = max(1024, 16 * self.n)
        self._alloc(capacity, device)

    def _alloc(self, cap, device):
        torch = self.torch
        self.cap = int(cap)
        fdt = torch.float32 if self.prm.precision == LUB_MIXED else torch.float64
        self.pair_i = torch.empty(self.cap, dtype=torch.int32, device=device)
        self.pair_j = torch.empty(self.cap, dtype=torch.int32, device=device)
        self.d_count = torch.zeros(1, dtype=torch.int32, device=device)
        self.nrm = torch.zeros(3 * self.cap, dtype=torch.float64, device=device)
        self.gap = torch.empty(self.cap, dtype=torch.float64, device=device)
        self.status = torch.empty(self.cap, dtype=torch.uint8, device=device)
        self.iters = torch.empty(self.cap, dtype=torch.uint8, device=device)
        self.FT = torch.empty(6 * self.cap, dtype=fdt, device=device)
        self.lever = torch.empty(6 * self.cap, dtype=fdt, device=device)
        # force and torque: two views of one buffer, so one copy reads both back
        self.ft_particles = torch.empty(6 * max(self.n, 1), dtype=fdt, device=device)
        self.force = self.ft_particles[:3 * max(self.n, 1)]
        self.torque = self.ft_particles[3 * max(self.n, 1):]

    def build_pairs(self, sync_count=True, grow=True, stream=None):
        h = self.ctx.h
        rc, cnt = lub_pairs_build(h, self.P.c, self.D, self.prm, self.pair_i, self.pair_j, self.cap, self.d_count,
                                  h_count=sync_count, stream=stream)
        if rc == LUB_ERR_CAPACITY and grow:
            self._alloc(int(cnt * 1.25) + 1024, self.pair_i.device)
            rc, cnt = lub_pairs_build(h, self.P.c, self.D, self.prm, self.pair_i, self.pair_j, self.cap,
                                      self.d_count, h_count=True, stream=stream)
        if rc != LUB_OK:
            _check(h, rc)
        return cnt

    def set_pairs(self, pi, pj):
        torch = self.torch
        m = len(pi)
        if m > self.cap:
            self._alloc(m, self.pair_i.device)
        self.pair_i[:m] = torch.as_tensor(np.asarray(pi, np.int32), device=self.pair_i.device)
        self.pair_j[:m] = torch.as_tensor(np.asarray(pj, np.int32), device=self.pair_i.device)
        self.d_count.fill_(m)
        return m

    def closest(self, stream=None):
        lub_closest_points(self.ctx.h, self.P.c, self.D, self.prm, self.pair_i, self.pair_j, self.d_count, self.cap,
                           self.nrm, self.gap, self.status, self.iters, stream=stream)

    def resistance(self, stream=None):
        lub_resistance(self.ctx.h, self.P.c, self.D, self.prm, self.pair_i, self.pair_j, self.d_count, self.cap,
                       self.nrm, self.gap, self.status, self.FT, self.lever, stream=stream)

    def links(self, q_bar=0.6, stream=None):
        """Link-based lubrication of Ding and Aidun on this step's pair list
        (lub_links): per-pair force on i [3][cap], torques on i and j [6][cap]
        and link counts [cap], double and int32 device tensors."""
        import torch
        dev = self.pair_i.device
        if getattr(self, "_links_cap", None) != self.cap:
            self.link_force = torch.zeros(3 * self.cap, dtype=torch.float64, device=dev)
            self.link_torque = torch.zeros(6 * self.cap, dtype=torch.float64, device=dev)
            self.link_count = torch.zeros(self.cap, dtype=torch.int32, device=dev)
            self._links_cap = self.cap
        lub_links(self.ctx.h, self.P.c, self.D, self.prm, self.pair_i, self.pair_j, self.d_count, self.cap, q_bar,
                  self.link_force, self.link_torque, self.link_count, stream=stream)
        return self.link_force, self.link_torque, self.link_count

    def apply(self, deterministic=0, accumulate=0, stream=None):
        lub_apply(self.ctx.h, self.pair_i, self.pair_j, self.d_count, self.cap, self.FT, self.lever, self.n,
                  self.force, self.torque, self.prm.precision, accumulate, deterministic, stream=stream)

    def rigid_step(self, density, dt, f_ext=None, t_ext=None, stream=None):
        """One particle sub-step with this step's lubrication force and torque
        (lub_rigid_step); moves the particles in place."""
        lub_rigid_step(self.ctx.h, self.P.c, self.force, self.torque, self.prm.precision, f_ext, t_ext, density, dt,
                       stream)

    def substeps(self, n_sub, density, dt, f_ext=None, t_ext=None, form="merged", stream=None):
        """One lattice-Boltzmann step of particle motion: the pair list built
        once, then n_sub sub-steps of (closest points, resistance + scatter,
        rigid update) at dt each."""
        self.build_pairs(sync_count=False, grow=False, stream=stream)
        for _ in range(n_sub):
            self.step(build=False, form=form, stream=stream)
            self.rigid_step(density, dt, f_ext, t_ext, stream)

    def keep_previous(self, stream=None):
        """Copy this step's pair list and normals aside for the temporal warm start."""
        torch = self.torch
        cur = torch.cuda.current_stream() if stream is None else stream
        with torch.cuda.stream(cur):
            if getattr(self, "prev_cap", None) != self.cap:
                self.prev_i = torch.empty_like(self.pair_i)
                self.prev_j = torch.empty_like(self.pair_j)
                self.prev_n = torch.empty_like(self.nrm)
                self.prev_count = torch.zeros_like(self.d_count)
                self.prev_cap = self.cap
            self.prev_i.copy_(self.pair_i)
            self.prev_j.copy_(self.pair_j)
            self.prev_n.copy_(self.nrm)
            self.prev_count.copy_(self.d_count)

    def carry(self, stream=None):
        """Start normals from the previous step's list (lub_carry_normals)."""
        lub_carry_normals(self.ctx.h, self.n, self.prev_i, self.prev_j, self.prev_n, self.prev_count, self.prev_cap,
                          self.pair_i, self.pair_j, self.d_count, self.cap, self.nrm, stream)

    def autotune(self, reps=3, stream=None):
        """Pick the launch shapes of this step's kernels (lub_autotune); returns them by name."""
        lub_autotune(self.ctx.h, self.P.c, self.D, self.prm, self.pair_i, self.pair_j, self.cap, self.d_count,
                     self.nrm, self.gap, self.status, self.iters, self.FT, self.lever, self.force, self.torque, reps,
                     stream)
        return {TUNE_NAMES[k]: lub_get_launch_shape(self.ctx.h, k) for k in range(LUB_TUNE_COUNT)}

    def correct(self, per_pair=True, pair_forces=True, stream=None):
        """Closest points, resistance and scatter in one call (lub_correct);
        per_pair=False skips the per-pair outputs other than the normals,
        pair_forces=False only the per-pair forces and lever arms (FT,
        lever): the per-particle sums are the step's result either way."""
        o = (lambda t: t) if per_pair else (lambda t: None)
        f = (lambda t: t) if (per_pair and pair_forces) else (lambda t: None)
        lub_correct(self.ctx.h, self.P.c, self.D, self.prm, self.pair_i, self.pair_j, self.d_count, self.cap, self.nrm,
                    o(self.gap), o(self.status), o(self.iters), f(self.FT), f(self.lever), self.force, self.torque, 0,
                    stream)

    def resistance_apply(self, per_pair=True, stream=None):
        """Resistance and the atomic scatter in one pass (lub_resistance_apply)."""
        o = (lambda t: t) if per_pair else (lambda t: None)
        lub_resistance_apply(self.ctx.h, self.P.c, self.D, self.prm, self.pair_i, self.pair_j, self.d_count,
                             self.cap, self.nrm, self.gap, self.status, o(self.FT), o(self.lever), self.force,
                             self.torque, 0, stream)

    def step(self, build=True, deterministic=0, sync_count=False, fused=False, per_pair=True, form=None,
             pair_forces=True, stream=None):
        """One correction step: the pair build, then the per-pair work in one
        of three forms: "calls" (closest points, resistance, apply), "merged"
        (closest points, then resistance + scatter in one pass) or "fused"
        (one lub_correct call: in FP64 all three in one pass, in mixed
        precision the merged kernels on one set of particle records;
        fused=True is the same).  deterministic needs
        "calls".  With warm_start = LUB_WARM_PREVIOUS the normals are carried
        over from the step before (keep_previous is called at the end of
        every step).  pair_forces=False: the fused form writes no per-pair
        forces and lever arms (the other forms always do)."""
        form = form or ("fused" if fused else "calls")
        if deterministic:
            form = "calls"
        temporal = self.prm.warm_start == LUB_WARM_PREVIOUS
        if build:
            self.build_pairs(sync_count=sync_count, grow=sync_count, stream=stream)
        if temporal and getattr(self, "prev_cap", None) == self.cap:
            self.carry(stream)
        if form == "fused":
            self.correct(per_pair=per_pair, pair_forces=pair_forces, stream=stream)
        elif form == "merged":
            self.closest(stream)
            self.resistance_apply(per_pair=per_pair, stream=stream)
        else:
            self.closest(stream)
            self.resistance(stream)
            self.apply(deterministic=deterministic, stream=stream)
        if temporal:
            self.keep_previous(stream)

    # host views (synchronising)
    def count(self):
        return int(self.d_count.item())

    def results(self):
        m = min(self.count(), self.cap)
        c = self.cap
        g = lambda t: t.cpu().numpy()
        nrm = g(self.nrm).reshape(3, c)[:, :m].T
        FT = g(self.FT).reshape(6, c)[:, :m].T
        lever = g(self.lever).reshape(6, c)[:, :m].T
        n = self.n
        return dict(pi=g(self.pair_i)[:m], pj=g(self.pair_j)[:m], n=nrm, h=g(self.gap)[:m],
                    status=g(self.status)[:m], iters=g(self.iters)[:m], FT=FT, lever=lever,
                    force=g(self.force)[:3 * n].reshape(3, n).T, torque=g(self.torque)[:3 * n].reshape(3, n).T)
