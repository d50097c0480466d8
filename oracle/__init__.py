"""Plain FP64 CPU oracle for the lubrication correction of arXiv:1308.6482.

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  It
shares no code with the CUDA library (``paper_1308_6482_gb300``) and neither
imports the other.  The arithmetic lives in ``lub_oracle.c`` (plain C, double
precision, paper order); this module only marshals numpy arrays.

Particles are given as a dict of 1-D arrays with the keys
``x y z qw qx qy qz r_par r_perp vx vy vz wx wy wz`` (any float dtype; they
are converted exactly to float64).  The domain is a dict with ``L`` (3),
``periodic`` (3 bools), ``walls`` (list of ``(z, dir)`` with ``dir=+1`` for a
wall whose fluid side is +z).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lub_oracle.c")
_SO = os.path.join(_HERE, "liborc.so")

ST_OVERLAP = 1
ST_NOCONV = 2
ST_DEGENERATE = 4

# cut-offs of Eq. results:cutoffs and mu = rho nu = 1/6 (tau = 1)
DEFAULT_PARAMS = dict(mu=1.0 / 6.0, delta_n=2.0 / 3.0, delta_t=0.5, delta_r=0.25,
                      h_c=0.0, eps_c=0.0, list_cutoff=1.0, model=0.0)

_FIELDS = ("x", "y", "z", "qw", "qx", "qy", "qz", "r_par", "r_perp",
           "vx", "vy", "vz", "wx", "wy", "wz")


def build(force=False):
    """Compile the oracle with gcc (plain -O2, no fast-math, no FMA contraction)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


class _Particles(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64)] + [(f, ctypes.POINTER(ctypes.c_double)) for f in _FIELDS]


class _Domain(ctypes.Structure):
    _fields_ = [("L", ctypes.c_double * 3), ("periodic", ctypes.c_int32 * 3),
                ("n_walls", ctypes.c_int32), ("wall_z", ctypes.c_double * 2),
                ("wall_dir", ctypes.c_int32 * 2)]


class _Params(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("mu", "delta_n", "delta_t", "delta_r", "h_c", "eps_c", "list_cutoff", "model")]


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P = ctypes.POINTER
        dp, ip = P(ctypes.c_double), P(ctypes.c_int32)
        lib.orc_candidates.restype = ctypes.c_int64
        lib.orc_candidates.argtypes = [P(_Particles), P(_Domain), ctypes.c_double, ip, ip, ctypes.c_int64]
        lib.orc_closest.restype = None
        lib.orc_closest.argtypes = [P(_Particles), P(_Domain), ctypes.c_int64, ip, ip, dp, dp, dp, dp, ip]
        lib.orc_pair_force.restype = None
        lib.orc_pair_force.argtypes = [P(_Particles), P(_Domain), P(_Params), ctypes.c_int64, ip, ip,
                                       dp, dp, dp, dp, dp, dp, dp, dp, ip]
        lib.orc_apply.restype = None
        lib.orc_apply.argtypes = [ctypes.c_int64, ctypes.c_int64, ip, ip, dp, dp, dp, dp]
        lib.orc_surface_geometry.restype = None
        lib.orc_surface_geometry.argtypes = [P(_Particles), ctypes.c_int64, dp, dp, dp]
        lib.orc_links.restype = None
        lib.orc_links.argtypes = [P(_Particles), P(_Domain), ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                  ip, ip, dp, dp, ip]
        lib.orc_g.restype = ctypes.c_double
        lib.orc_g.argtypes = [P(_Particles), P(_Domain), ctypes.c_int32, ctypes.c_int32, dp]
        lib.orc_surface_pq.restype = None
        lib.orc_surface_pq.argtypes = [P(_Particles), ctypes.c_int64, dp, dp]
        lib.orc_mlp_features.restype = None
        lib.orc_mlp_features.argtypes = [P(_Particles), P(_Domain), ctypes.c_int64, ip, ip, dp]
        lib.orc_pq_labels.restype = None
        lib.orc_pq_labels.argtypes = [P(_Particles), ctypes.c_int64, ip, ip, dp, dp, dp]
        lib.orc_mlp_loss_grad.restype = ctypes.c_double
        lib.orc_mlp_loss_grad.argtypes = [ctypes.c_int64] + [dp] * 16
        lib.orc_mlp_baseline.restype = None
        lib.orc_mlp_baseline.argtypes = [P(_Particles), P(_Domain), ctypes.c_int64, ip, ip, dp]
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


class Particles:
    """FP64 copies of the particle arrays, kept alive for the C calls."""

    def __init__(self, parts):
        n = len(parts["x"])
        self.arrays = {}
        for f in _FIELDS:
            a = parts.get(f)
            if a is None:
                a = np.zeros(n)
            a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
            assert a.shape == (n,), (f, a.shape)
            self.arrays[f] = a
        self.n = n
        self.c = _Particles(n, *[_dp(self.arrays[f]) for f in _FIELDS])


def _domain(dom):
    walls = dom.get("walls", [])
    assert len(walls) <= 2
    d = _Domain()
    for k in range(3):
        d.L[k] = float(dom["L"][k])
        d.periodic[k] = int(bool(dom["periodic"][k]))
    d.n_walls = len(walls)
    for w, (z, s) in enumerate(walls):
        d.wall_z[w] = float(z)
        d.wall_dir[w] = int(s)
    return d


def _params(prm):
    p = dict(DEFAULT_PARAMS)
    if prm:
        p.update({k: v for k, v in prm.items() if k in DEFAULT_PARAMS})
    return _Params(*[float(p[k]) for k in
                     ("mu", "delta_n", "delta_t", "delta_r", "h_c", "eps_c", "list_cutoff", "model")])


def _as_particles(parts):
    return parts if isinstance(parts, Particles) else Particles(parts)


def candidates(parts, dom, list_cutoff=1.0):
    """Candidate pairs by the paper's pre-filters (Sec. III A); (pi, pj) int32.

    Particle pairs in (i, j) order with i < j, then wall pairs (j = -1 - w)
    in (i, w) order."""
    lib = _load()
    P = _as_particles(parts)
    D = _domain(dom)
    cnt = lib.orc_candidates(ctypes.byref(P.c), ctypes.byref(D), float(list_cutoff), None, None, 0)
    pi = np.zeros(max(cnt, 1), np.int32)
    pj = np.zeros(max(cnt, 1), np.int32)
    lib.orc_candidates(ctypes.byref(P.c), ctypes.byref(D), float(list_cutoff), _ip(pi), _ip(pj), cnt)
    return pi[:cnt], pj[:cnt]


def closest(parts, dom, pi, pj):
    """Points of closest approach: dict(n, h, yi, yj, status)."""
    lib = _load()
    P = _as_particles(parts)
    D = _domain(dom)
    pi = np.ascontiguousarray(pi, np.int32)
    pj = np.ascontiguousarray(pj, np.int32)
    m = len(pi)
    n = np.zeros((m, 3))
    h = np.zeros(m)
    yi = np.zeros((m, 3))
    yj = np.zeros((m, 3))
    st = np.zeros(m, np.int32)
    if m:
        lib.orc_closest(ctypes.byref(P.c), ctypes.byref(D), m, _ip(pi), _ip(pj), _dp(n), _dp(h),
                        _dp(yi), _dp(yj), _ip(st))
    return dict(n=n, h=h, yi=yi, yj=yj, status=st)


def pair_force(parts, dom, prm, pi, pj, cp, want_k=False, want_geom=False):
    """Per-pair F_i, T_i (lab, T about y*_i) and lever arms; optionally K~ and geometry.

    Returns dict(FT [m,6], lever [m,6], Kt [m,6,6], geom [m,40], status).

    geom: S1 S2 S1' S2' G0 G2 G0' G2' phi lam1 lam2 chi kappa0..3 x1[3] x2[3] x3[3]
    H33 h_eff u[6] (local relative surface velocity)."""
    lib = _load()
    P = _as_particles(parts)
    D = _domain(dom)
    p = _params(prm)
    pi = np.ascontiguousarray(pi, np.int32)
    pj = np.ascontiguousarray(pj, np.int32)
    m = len(pi)
    FT = np.zeros((m, 6))
    lever = np.zeros((m, 6))
    Kt = np.zeros((m, 36)) if want_k else None
    geom = np.zeros((m, 40)) if want_geom else None
    st = np.array(cp["status"], np.int32, copy=True)
    if m:
        lib.orc_pair_force(ctypes.byref(P.c), ctypes.byref(D), ctypes.byref(p), m, _ip(pi), _ip(pj),
                           _dp(np.ascontiguousarray(cp["n"], np.float64)),
                           _dp(np.ascontiguousarray(cp["h"], np.float64)),
                           _dp(np.ascontiguousarray(cp["yi"], np.float64)),
                           _dp(np.ascontiguousarray(cp["yj"], np.float64)),
                           _dp(FT), _dp(lever), _dp(Kt) if want_k else None,
                           _dp(geom) if want_geom else None, _ip(st))
    out = dict(FT=FT, lever=lever, status=st)
    if want_k:
        out["Kt"] = Kt.reshape(m, 6, 6)
    if want_geom:
        out["geom"] = geom
    return out


def apply(nparticles, pi, pj, FT, lever):
    """Per-particle force and torque [n,3] each (Newton's third law for j)."""
    lib = _load()
    pi = np.ascontiguousarray(pi, np.int32)
    pj = np.ascontiguousarray(pj, np.int32)
    FT = np.ascontiguousarray(FT, np.float64)
    lever = np.ascontiguousarray(lever, np.float64)
    f = np.zeros((nparticles, 3))
    t = np.zeros((nparticles, 3))
    lib.orc_apply(nparticles, len(pi), _ip(pi), _ip(pj), _dp(FT), _dp(lever), _dp(f), _dp(t))
    return f, t


def links(parts, dom, pi, pj, mu=1.0 / 6.0, qbar=0.6):
    """Link-based lubrication of Ding and Aidun (Eq. methods:dlub) per pair:
    dict(F [m,3] force on i, T [m,6] torques on i and j about their centres,
    links [m] contributing links).  See orc_links for the readings."""
    lib = _load()
    P = _as_particles(parts)
    D = _domain(dom)
    pi = np.ascontiguousarray(pi, np.int32)
    pj = np.ascontiguousarray(pj, np.int32)
    m = len(pi)
    F = np.zeros((m, 3))
    T = np.zeros((m, 6))
    nl = np.zeros(m, np.int32)
    if m:
        lib.orc_links(ctypes.byref(P.c), ctypes.byref(D), float(mu), float(qbar), m, _ip(pi), _ip(pj), _dp(F),
                      _dp(T), _ip(nl))
    return dict(F=F, T=T, links=nl)


def surface_geometry(parts, k, y, nrm):
    """(x1[3], S1, S2, Gamma0, Gamma2, p) of particle k at surface point y."""
    lib = _load()
    P = _as_particles(parts)
    out = np.zeros(8)
    y = np.ascontiguousarray(y, np.float64)
    nrm = np.ascontiguousarray(nrm, np.float64)
    lib.orc_surface_geometry(ctypes.byref(P.c), int(k), _dp(y), _dp(nrm), _dp(out))
    return out[:3], out[3], out[4], out[5], out[6], out[7]


def g_value(parts, dom, i, j, n):
    lib = _load()
    P = _as_particles(parts)
    D = _domain(dom)
    n = np.ascontiguousarray(n, np.float64)
    return lib.orc_g(ctypes.byref(P.c), ctypes.byref(D), int(i), int(j), _dp(n))


def step(parts, dom, prm=None):
    """The whole path on the CPU: candidates, closest points, pair forces, sums."""
    p = dict(DEFAULT_PARAMS)
    if prm:
        p.update(prm)
    P = _as_particles(parts)
    pi, pj = candidates(P, dom, p["list_cutoff"])
    cp = closest(P, dom, pi, pj)
    pf = pair_force(P, dom, p, pi, pj, cp)
    f, t = apply(P.n, pi, pj, pf["FT"], pf["lever"])
    return dict(pi=pi, pj=pj, force=f, torque=t, **cp, FT=pf["FT"], lever=pf["lever"],
                pair_status=pf["status"])


# ---------------------------------------------------------------------------
# learned warm start: labels, features and the FP64 network
# ---------------------------------------------------------------------------
MLP_SHAPES = dict(W1=(128, 12), b1=(128,), W2=(128, 128), b2=(128,), W3=(4, 128), b3=(4,))


def surface_pq(parts, k, y):
    """(p, q) of Eq. lub:spheroid of surface point y of particle k."""
    lib = _load()
    P = _as_particles(parts)
    out = np.zeros(2)
    lib.orc_surface_pq(ctypes.byref(P.c), int(k), _dp(np.ascontiguousarray(y, np.float64)), _dp(out))
    return out


def pq_labels(parts, dom, pi, pj, cp=None):
    """Targets (p_i, q_i, p_j, q_j) of the closest points [m, 4]."""
    P = _as_particles(parts)
    pi = np.ascontiguousarray(pi, np.int32)
    pj = np.ascontiguousarray(pj, np.int32)
    if cp is None:
        cp = closest(P, dom, pi, pj)
    out = np.zeros((len(pi), 4))
    if len(pi):
        _load().orc_pq_labels(ctypes.byref(P.c), len(pi), _ip(pi), _ip(pj),
                              _dp(np.ascontiguousarray(cp["yi"], np.float64)),
                              _dp(np.ascontiguousarray(cp["yj"], np.float64)), _dp(out))
    return out


def mlp_features(parts, dom, pi, pj):
    """The 12 input features of each pair [m, 12] (before standardisation)."""
    lib = _load()
    P = _as_particles(parts)
    D = _domain(dom)
    pi = np.ascontiguousarray(pi, np.int32)
    pj = np.ascontiguousarray(pj, np.int32)
    f = np.zeros((len(pi), 12))
    if len(pi):
        lib.orc_mlp_features(ctypes.byref(P.c), ctypes.byref(D), len(pi), _ip(pi), _ip(pj), _dp(f))
    return f


def mlp_baseline(parts, dom, pi, pj):
    """(p, q) of the line-of-centres start on both particles [m, 4]."""
    lib = _load()
    P = _as_particles(parts)
    D = _domain(dom)
    pi = np.ascontiguousarray(pi, np.int32)
    pj = np.ascontiguousarray(pj, np.int32)
    out = np.zeros((len(pi), 4))
    if len(pi):
        lib.orc_mlp_baseline(ctypes.byref(P.c), ctypes.byref(D), len(pi), _ip(pi), _ip(pj), _dp(out))
    return out


def wrap_pi(a):
    return a - 2 * np.pi * np.floor(a / (2 * np.pi) + 0.5)


def mlp_targets(labels, baseline):
    """Corrections the network learns (azimuths wrapped) and the loss weights
    (1, cos^2 p_i, 1, cos^2 p_j): the arc length on the parameter sphere,
    ds^2 = dp^2 + cos^2 p dq^2, so the azimuth counts little near the poles
    where it is undefined."""
    t = labels - baseline
    t[:, 1] = wrap_pi(t[:, 1])
    t[:, 3] = wrap_pi(t[:, 3])
    w = np.ones_like(t)
    w[:, 1] = np.cos(labels[:, 0]) ** 2
    w[:, 3] = np.cos(labels[:, 2]) ** 2
    return t, w


def mlp_loss_grad(x, tgt, w, want_grad=True, wgt=None):
    """Loss, gradients (dict like w) and outputs of the network on standardised x."""
    lib = _load()
    x = np.ascontiguousarray(x, np.float64)
    tgt = np.ascontiguousarray(tgt, np.float64)
    ww = {k: np.ascontiguousarray(w[k], np.float64) for k in MLP_SHAPES}
    g = {k: np.zeros(sh) for k, sh in MLP_SHAPES.items()}
    out = np.zeros((len(x), 4))
    args = [_dp(ww[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]
    gargs = [_dp(g[k]) if want_grad else None for k in ("W1", "b1", "W2", "b2", "W3", "b3")]
    wg = None if wgt is None else np.ascontiguousarray(wgt, np.float64)
    loss = lib.orc_mlp_loss_grad(len(x), _dp(x), _dp(tgt), _dp(wg) if wg is not None else None, *args, *gargs,
                                 _dp(out))
    return loss, (g if want_grad else None), out


# ---------------------------------------------------------------------------
# particle sub-step (Sec. II), plain numpy in float64
# ---------------------------------------------------------------------------
def rigid_step(parts, force, torque, density, dt, f_ext=None, t_ext=None):
    """One explicit sub-step of every particle: semi-implicit Euler on the
    rigid-body equations (translation, then angular momentum, orientation,
    angular velocity).  force, torque [n, 3] (lubrication, about the centres),
    f_ext, t_ext [n, 3] or None.  Returns new arrays in a copy of parts
    (float64)."""
    out = {k: np.array(v, np.float64) for k, v in parts.items()}
    n = len(out["x"])
    a = out["r_perp"]
    c = out["r_par"]
    m = density * 4.0 / 3.0 * np.pi * c * a * a
    ipar = 0.4 * m * a * a
    iperp = 0.2 * m * (c * c + a * a)
    F = np.asarray(force, np.float64) + (0 if f_ext is None else np.asarray(f_ext, np.float64))
    T = np.asarray(torque, np.float64) + (0 if t_ext is None else np.asarray(t_ext, np.float64))
    v = np.stack([out["vx"], out["vy"], out["vz"]], 1) + dt * F / m[:, None]
    for d, k in enumerate(("x", "y", "z")):
        out[k] = out[k] + dt * v[:, d]
    for d, k in enumerate(("vx", "vy", "vz")):
        out[k] = v[:, d]
    q = np.stack([out["qw"], out["qx"], out["qy"], out["qz"]], 1)
    q /= np.linalg.norm(q, axis=1, keepdims=True)

    def axis(q):
        w, x, y, z = q.T
        s = 2.0 / (w * w + x * x + y * y + z * z)
        return np.stack([s * (x * z + w * y), s * (y * z - w * x), 1 - s * (x * x + y * y)], 1)

    def inertia(o, vec, inverse):
        on = np.sum(o * vec, 1, keepdims=True)
        cp = (1.0 / ipar if inverse else ipar)[:, None]
        cq = (1.0 / iperp if inverse else iperp)[:, None]
        return cq * (vec - on * o) + cp * on * o

    o = axis(q)
    w = np.stack([out["wx"], out["wy"], out["wz"]], 1)
    L = inertia(o, w, False) + dt * T
    wm = inertia(o, L, True)
    ang = dt * np.linalg.norm(wm, axis=1)
    s = np.where(ang > 0, np.sin(0.5 * ang) * dt / np.where(ang > 0, ang, 1.0), 0.0)
    r = np.stack([np.cos(0.5 * ang), s * wm[:, 0], s * wm[:, 1], s * wm[:, 2]], 1)
    r0, r1, r2, r3 = r.T
    q0, q1, q2, q3 = q.T
    nq = np.stack([r0 * q0 - r1 * q1 - r2 * q2 - r3 * q3, r0 * q1 + r1 * q0 + r2 * q3 - r3 * q2,
                   r0 * q2 - r1 * q3 + r2 * q0 + r3 * q1, r0 * q3 + r1 * q2 - r2 * q1 + r3 * q0], 1)
    nq /= np.linalg.norm(nq, axis=1, keepdims=True)
    for d, k in enumerate(("qw", "qx", "qy", "qz")):
        out[k] = nq[:, d]
    wn = inertia(axis(nq), L, True)
    for d, k in enumerate(("wx", "wy", "wz")):
        out[k] = wn[:, d]
    return out
