"""Seeded synthetic inputs shaped like the paper's suspensions.

This module generates inputs only and serves both the CUDA path and the
oracle.  It holds none of the lubrication method's arithmetic: it draws
poses, shapes, gaps and velocities, and places particles (uniformly, or in
contact with a parent at a drawn surface gap).  A drawn gap is a property of
the input distribution; tests always take expected gaps and forces from the
oracle.

Particle dicts have the keys ``x y z`` (float64), ``qw qx qy qz`` (float32,
scalar-first quaternion, body z = axis of rotational symmetry), ``r_par``
(semi-axis along the symmetry axis) and ``r_perp`` (float32), and ``vx vy vz
wx wy wz`` (float32).  Domains are dicts ``L`` (3), ``periodic`` (3 bools),
``walls`` (list of ``(z, dir)``).

Workloads (lattice units; shapes and fractions of the paper's suspensions,
Sec. IV):
  * ``config_prolate_wall``: 64 prolates (6,3,3) in a 42^3 box (periodic in
    x, y) over a plane wall at z = 0, Phi ~ 0.195.
  * ``config_mixed_suspension``: 32,768 particles, half spheres r = 4.5 and
    half oblates (6,6,3), periodic 357^3 box, Phi = 0.3; most particles are
    attached to an earlier one at a gap drawn log-uniform in [1e-4, 1].
  * ``pair_stream``: independent pairs at gaps drawn log-uniform (optionally
    scaled by the smaller semi-axis), each pair far from all others.
  * ``ensemble``: 256 periodic suspensions of spheroids (aspect ratio
    log-uniform in [1/3, 3]) at volume fractions uniform in [0.1, 0.5], sized
    for pair counts log-uniform in [1e3, 2e5]: growth packings tiled k^3.
  * ``large_config``: 2^20 such spheroids at Phi = 0.5 in a 1024^3 cube
    between two walls: a growth packing of a slab, tiled 8 x 8.

Dense suspensions come from ``grow``, the growth method of the paper's
Sec. IV (random placement at 30 % of the sizes, growth with overlap
repulsion and damped motion to slightly beyond full size, sizes reset);
random sequential placement (``suspension``) jams near Phi = 0.4.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen_core.c")
_SO = os.path.join(_HERE, "libgen.so")
_lib = None

VEL_SIGMA = 1e-3  # velocities and angular velocities ~ N(0, 1e-3^2) per component


def build(force=False):
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    try:  # OpenMP for the growth sweeps (results do not depend on the thread count)
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"],
                              stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P = ctypes.POINTER
        lib.gen_rsa.restype = ctypes.c_int64
        lib.gen_rsa.argtypes = [ctypes.c_int64, P(ctypes.c_double), P(ctypes.c_int32), ctypes.c_int32,
                                P(ctypes.c_double), P(ctypes.c_int32), P(ctypes.c_float),
                                P(ctypes.c_float), ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_int64, ctypes.c_uint64,
                                P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double),
                                P(ctypes.c_float)]
        lib.gen_grow.restype = ctypes.c_int64
        lib.gen_grow.argtypes = [ctypes.c_int64, P(ctypes.c_double), P(ctypes.c_int32), ctypes.c_int32,
                                 P(ctypes.c_double), P(ctypes.c_int32), P(ctypes.c_float), P(ctypes.c_float),
                                 ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                 ctypes.c_uint64, P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double),
                                 P(ctypes.c_float), P(ctypes.c_int64)]
        _lib = lib
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def random_quaternions(n, rng):
    """Uniform random rotations (Shoemake), float32 (w, x, y, z)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1 - u1), np.sqrt(u1)
    q = np.stack([b * np.cos(2 * np.pi * u3), a * np.sin(2 * np.pi * u2),
                  a * np.cos(2 * np.pi * u2), b * np.sin(2 * np.pi * u3)], axis=1)
    return q.astype(np.float32)


def _rotmat(q):
    """Rotation matrices [n,3,3] of normalised quaternions [n,4] (float64 math)."""
    q = np.asarray(q, np.float64)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    t = 2.0 / (w * w + x * x + y * y + z * z)
    R = np.empty((len(q), 3, 3))
    R[:, 0, 0] = 1 - t * (y * y + z * z)
    R[:, 0, 1] = t * (x * y - w * z)
    R[:, 0, 2] = t * (x * z + w * y)
    R[:, 1, 0] = t * (x * y + w * z)
    R[:, 1, 1] = 1 - t * (x * x + z * z)
    R[:, 1, 2] = t * (y * z - w * x)
    R[:, 2, 0] = t * (x * z - w * y)
    R[:, 2, 1] = t * (y * z + w * x)
    R[:, 2, 2] = 1 - t * (x * x + y * y)
    return R


def _surface_point_with_normal(R, rpar, rperp, n):
    """Offset from the centre of the surface point whose outward normal is n."""
    D = np.stack([rperp ** 2, rperp ** 2, rpar ** 2], axis=1).astype(np.float64)
    nb = np.einsum("kji,kj->ki", R, n)  # body components
    s = np.sqrt(np.sum(D * nb * nb, axis=1))
    yb = D * nb / s[:, None]
    return np.einsum("kij,kj->ki", R, yb)


def _unit_vectors(n, rng):
    z = 2 * rng.random(n) - 1
    ph = 2 * np.pi * rng.random(n)
    s = np.sqrt(1 - z * z)
    return np.stack([s * np.cos(ph), s * np.sin(ph), z], axis=1)


def velocities(parts, rng, sigma=VEL_SIGMA):
    n = len(parts["x"])
    for k in ("vx", "vy", "vz", "wx", "wy", "wz"):
        parts[k] = (sigma * rng.standard_normal(n)).astype(np.float32)
    return parts


def suspension(shapes, L, periodic=(True, True, True), walls=(), attach_prob=0.0,
               gap_range=(1e-4, 1.0), wall_min=0.0, seed=1, max_attempts=100000):
    """Random sequential placement of the given shapes ([(r_par, r_perp)] per particle)."""
    lib = _load()
    shapes = np.asarray(shapes, np.float32)
    N = len(shapes)
    r_par = np.ascontiguousarray(shapes[:, 0])
    r_perp = np.ascontiguousarray(shapes[:, 1])
    Lc = np.asarray(L, np.float64)
    per = np.asarray([int(bool(p)) for p in periodic], np.int32)
    wz = np.zeros(2)
    wd = np.zeros(2, np.int32)
    for w, (zz, dd) in enumerate(walls):
        wz[w], wd[w] = zz, dd
    x = np.zeros(N)
    y = np.zeros(N)
    z = np.zeros(N)
    q = np.zeros((N, 4), np.float32)
    placed = lib.gen_rsa(N, _ptr(Lc, ctypes.c_double), _ptr(per, ctypes.c_int32), len(walls),
                         _ptr(wz, ctypes.c_double), _ptr(wd, ctypes.c_int32),
                         _ptr(r_par, ctypes.c_float), _ptr(r_perp, ctypes.c_float),
                         float(attach_prob), float(gap_range[0]), float(gap_range[1]),
                         float(wall_min), int(max_attempts), int(seed) & ((1 << 64) - 1),
                         _ptr(x, ctypes.c_double), _ptr(y, ctypes.c_double),
                         _ptr(z, ctypes.c_double), _ptr(q, ctypes.c_float))
    if placed != N:
        raise RuntimeError("placement stalled after %d of %d particles" % (placed, N))
    parts = dict(x=x, y=y, z=z, qw=q[:, 0].copy(), qx=q[:, 1].copy(), qy=q[:, 2].copy(),
                 qz=q[:, 3].copy(), r_par=r_par.copy(), r_perp=r_perp.copy())
    velocities(parts, np.random.default_rng(seed + 7919))
    dom = dict(L=tuple(float(v) for v in L), periodic=tuple(bool(p) for p in periodic),
               walls=[(float(a), int(b)) for a, b in walls])
    return parts, dom


def grow(shapes, L, periodic=(True, True, True), walls=(), seed=1, s0=0.3, s_over=1.02, g0=0.01,
         max_sweeps=20000):
    """Growth packing (the paper's initialisation of dense suspensions, Sec. IV):
    random placement at s0 of the linear sizes, growth with overlap repulsion
    and overdamped motion to s_over, sizes reset to 1.  Every gap ends at
    least about (s_over - 1) times the particle sizes.  Returns (parts, dom);
    Returns (parts, dom, sweeps)."""
    lib = _load()
    shapes = np.asarray(shapes, np.float32)
    N = len(shapes)
    r_par = np.ascontiguousarray(shapes[:, 0])
    r_perp = np.ascontiguousarray(shapes[:, 1])
    Lc = np.asarray(L, np.float64)
    per = np.asarray([int(bool(p)) for p in periodic], np.int32)
    wz = np.zeros(2)
    wd = np.zeros(2, np.int32)
    for w, (zz, dd) in enumerate(walls):
        wz[w], wd[w] = zz, dd
    x, y, z = np.zeros(N), np.zeros(N), np.zeros(N)
    q = np.zeros((N, 4), np.float32)
    sweeps = np.zeros(1, np.int64)
    rc = lib.gen_grow(N, _ptr(Lc, ctypes.c_double), _ptr(per, ctypes.c_int32), len(walls),
                      _ptr(wz, ctypes.c_double), _ptr(wd, ctypes.c_int32), _ptr(r_par, ctypes.c_float),
                      _ptr(r_perp, ctypes.c_float), float(s0), float(s_over), float(g0), int(max_sweeps),
                      int(seed) & ((1 << 64) - 1), _ptr(x, ctypes.c_double), _ptr(y, ctypes.c_double),
                      _ptr(z, ctypes.c_double), _ptr(q, ctypes.c_float), _ptr(sweeps, ctypes.c_int64))
    if rc == -1:
        raise RuntimeError("placement at %g of the sizes stalled" % s0)
    if rc < -1:
        raise RuntimeError("growth stalled: %d contacts still overlap after %d sweeps" % (-2 - rc, sweeps[0]))
    parts = dict(x=x, y=y, z=z, qw=q[:, 0].copy(), qx=q[:, 1].copy(), qy=q[:, 2].copy(),
                 qz=q[:, 3].copy(), r_par=r_par.copy(), r_perp=r_perp.copy())
    velocities(parts, np.random.default_rng(seed + 7919))
    dom = dict(L=tuple(float(v) for v in L), periodic=tuple(bool(p) for p in periodic),
               walls=[(float(a), int(b)) for a, b in walls])
    return parts, dom, int(sweeps[0])


def config_prolate_wall(seed=1, N=64, L=42.0):
    """64 prolates (R_par=6, R_perp=3) in an L^3 box, periodic in x, y, wall at z=0."""
    shapes = np.tile([[6.0, 3.0]], (N, 1))
    return suspension(shapes, (L, L, L), periodic=(True, True, False), walls=[(0.0, 1)],
                      attach_prob=0.0, seed=seed)


def mixed_shapes(N, rng):
    """Half spheres r=4.5, half oblates (R_perp=6, R_par=3), shuffled."""
    sh = np.empty((N, 2), np.float32)
    sh[: N // 2] = (4.5, 4.5)
    sh[N // 2:] = (3.0, 6.0)
    rng.shuffle(sh)
    return sh


def config_mixed_suspension(N=32768, phi=0.3, seed=2, attach_prob=0.9, gap_range=(1e-4, 1.0)):
    """Mixed spheres/oblates at volume fraction phi in a periodic cube."""
    rng = np.random.default_rng(seed)
    sh = mixed_shapes(N, rng)
    vol = float(np.sum(4.0 / 3.0 * np.pi * sh[:, 0].astype(np.float64) * sh[:, 1] ** 2))
    L = (vol / phi) ** (1.0 / 3.0)
    return suspension(sh, (L, L, L), attach_prob=attach_prob, gap_range=gap_range, seed=seed)


def pair_stream(P, seed=3, kind="mixed", gap_range=(1e-4, 1.0), gap_scale="absolute", spacing=None):
    """P independent pairs (2k, 2k+1), each at a drawn gap, far from all others.

    kind: 'mixed'   spheres r=4.5 / oblates (6,6,3), 50 % each, random per particle;
          'aspect'  aspect ratio log-uniform in [1/3, 3], equivalent radius 4.5;
          'spheres' radii uniform in [2, 8].
    gap_scale: 'absolute' (gap in lattice units) or 'min_axis' (gap times the
    smaller semi-axis of the two particles).
    Returns (parts, dom, pi, pj)."""
    rng = np.random.default_rng(seed)
    n = 2 * P
    if kind == "mixed":
        sh = np.where(rng.random(n)[:, None] < 0.5, [[4.5, 4.5]], [[3.0, 6.0]]).astype(np.float32)
    elif kind == "aspect":
        lam = np.exp(rng.uniform(np.log(1 / 3), np.log(3.0), n))
        rperp = 4.5 * lam ** (-1.0 / 3.0)
        rpar = 4.5 * lam ** (2.0 / 3.0)
        sh = np.stack([rpar, rperp], 1).astype(np.float32)
    elif kind == "spheres":
        r = rng.uniform(2.0, 8.0, n)
        sh = np.stack([r, r], 1).astype(np.float32)
    else:
        raise ValueError(kind)
    q = random_quaternions(n, rng)
    R = _rotmat(q)
    rpar = sh[:, 0].astype(np.float64)
    rperp = sh[:, 1].astype(np.float64)
    nrm = _unit_vectors(P, rng)
    g = np.exp(rng.uniform(np.log(gap_range[0]), np.log(gap_range[1]), P))
    if gap_scale == "min_axis":
        g = g * np.minimum(sh[0::2].min(1), sh[1::2].min(1))
    a, b = np.arange(0, n, 2), np.arange(1, n, 2)
    if spacing is None:
        spacing = 2.0 * float(sh.max()) * 2.0 + 4.0
    side = int(np.ceil(P ** (1.0 / 3.0)))
    idx = np.arange(P)
    grid = np.stack([idx % side, (idx // side) % side, idx // (side * side)], 1).astype(np.float64)
    ra = (grid + 0.5) * spacing + rng.uniform(-1, 1, (P, 3))
    ya = ra + _surface_point_with_normal(R[a], rpar[a], rperp[a], nrm)
    rb = ya + g[:, None] * nrm - _surface_point_with_normal(R[b], rpar[b], rperp[b], -nrm)
    pos = np.empty((n, 3))
    pos[a] = ra
    pos[b] = rb
    Lb = float(side * spacing)
    parts = dict(x=pos[:, 0].copy(), y=pos[:, 1].copy(), z=pos[:, 2].copy(),
                 qw=q[:, 0].copy(), qx=q[:, 1].copy(), qy=q[:, 2].copy(), qz=q[:, 3].copy(),
                 r_par=sh[:, 0].copy(), r_perp=sh[:, 1].copy())
    velocities(parts, rng)
    dom = dict(L=(Lb, Lb, Lb), periodic=(False, False, False), walls=[])
    return parts, dom, a.astype(np.int32), b.astype(np.int32)


def aspect_shapes(N, rng, r_eq=4.5):
    """Spheroids with aspect ratio log-uniform in [1/3, 3] and equivalent radius
    r_eq (R_par R_perp^2 = r_eq^3)."""
    lam = np.exp(rng.uniform(np.log(1 / 3), np.log(3.0), N))
    return np.stack([r_eq * lam ** (2.0 / 3.0), r_eq * lam ** (-1.0 / 3.0)], 1).astype(np.float32)


def tile_periodic(parts, dom, k, rng, axes=(0, 1, 2)):
    """k copies per listed (periodic) axis of a suspension side by side: again
    a suspension, periodic along those axes and k^len(axes) times the size,
    whose pairs across copy boundaries are the periodic-image pairs of the
    original.  Velocities are drawn afresh."""
    if k == 1:
        return parts, dom
    L = np.asarray(dom["L"], np.float64)
    for a in axes:
        assert dom["periodic"][a], "tiling needs a periodic axis"
    reps = [k if a in axes else 1 for a in range(3)]
    sh = np.stack(np.meshgrid(*[np.arange(r) for r in reps], indexing="ij"), -1).reshape(-1, 3)
    out = {}
    for a, key in enumerate(("x", "y", "z")):
        out[key] = (np.asarray(parts[key])[None, :] + (sh[:, a] * L[a])[:, None]).reshape(-1)
    for key in ("qw", "qx", "qy", "qz", "r_par", "r_perp"):
        out[key] = np.tile(np.asarray(parts[key]), len(sh))
    velocities(out, rng)
    d = dict(dom)
    d["L"] = tuple(float(v) * reps[a] for a, v in enumerate(L))
    return out, d


def large_config(N=1 << 20, phi=0.5, seed=6, k=8, L=1024.0, base_only=False):
    """Large dense run: N spheroids (aspect ratio log-uniform in [1/3, 3]) at
    volume fraction phi in an L^3 cube periodic in x, y between plane walls
    at z = 0 and z = L; the equivalent radius fills the cube at phi
    (4.96 for 2^20 particles in 1024^3 at 0.5).  A growth packing of N / k^2
    particles in a slab of L/k x L/k x L (walls included), tiled k x k in x
    and y.  base_only: the slab itself (periodic in x, y with period L/k),
    whose pairs are the large run's pairs up to the tiling."""
    rng = np.random.default_rng(seed)
    r_eq = (phi * L ** 3 / (N * 4.0 / 3.0 * np.pi)) ** (1.0 / 3.0)
    n0 = N // (k * k)
    sh = aspect_shapes(n0, rng, r_eq)
    base, dom, _ = grow(sh, (L / k, L / k, L), periodic=(True, True, False), walls=[(0.0, 1), (L, -1)], seed=seed)
    if base_only:
        return base, dom
    return tile_periodic(base, dom, k, rng, axes=(0, 1))


# candidate pairs per particle of growth packings of these spheroids (list
# cut-off 1, equivalent radius 4.5) at volume fraction phi, fitted on 800-
# particle packings at phi = 0.1 .. 0.5 (0.80, 1.58, 2.45, 3.32, 4.26)
def _pairs_per_particle(phi):
    return 8.65 * phi - 0.065


def ensemble_member(args):
    """One suspension of the ensemble workload: (seed, phi, target pairs) ->
    (parts, dom), a growth packing of 128..1024 spheroids tiled k^3 times."""
    seed, phi, target = args
    rng = np.random.default_rng(seed)
    n_all = target / _pairs_per_particle(phi)
    k = max(1, int(np.ceil((n_all / 1024.0) ** (1.0 / 3.0))))
    n0 = int(max(128, round(n_all / k ** 3)))
    sh = aspect_shapes(n0, rng)
    vol = float(np.sum(4.0 / 3.0 * np.pi * sh[:, 0].astype(np.float64) * sh[:, 1] ** 2))
    L = (vol / phi) ** (1.0 / 3.0)
    parts, dom, _ = grow(sh, (L, L, L), seed=seed)
    return tile_periodic(parts, dom, k, rng)


def _pool_member(args):
    # one thread per pool process (set before the generator library loads)
    os.environ["OMP_NUM_THREADS"] = "1"
    return ensemble_member(args)


def ensemble(n_susp=256, seed=4, phi_range=(0.1, 0.5), pairs_range=(1e3, 2e5), processes=None):
    """Independent periodic suspensions of mixed spheroids (aspect ratio
    log-uniform in [1/3, 3]) at volume fractions uniform in phi_range, sized
    for pair counts log-uniform in pairs_range.  Returns ([(parts, dom)], meta).
    Built in a spawn process pool (safe after CUDA has started)."""
    import multiprocessing as mp
    rng = np.random.default_rng(seed)
    phi = rng.uniform(phi_range[0], phi_range[1], n_susp)
    target = np.exp(rng.uniform(np.log(pairs_range[0]), np.log(pairs_range[1]), n_susp))
    jobs = [(int(seed) * 100003 + b, float(phi[b]), float(target[b])) for b in range(n_susp)]
    procs = processes if processes is not None else min(16, os.cpu_count() or 1)
    if procs > 1:
        with mp.get_context("spawn").Pool(procs) as pool:
            sus = pool.map(_pool_member, jobs, chunksize=1)
    else:
        sus = [ensemble_member(j) for j in jobs]
    return sus, dict(phi=phi, target_pairs=target)


def subset(parts, idx):
    return {k: np.asarray(v)[idx].copy() for k, v in parts.items()}
