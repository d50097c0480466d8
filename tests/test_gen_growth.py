"""The growth packing of gen (the paper's initialisation of dense
suspensions, Sec. IV), checked independently of its own overlap test: the
oracle's closest points (a separate solver with its own certificate) give a
positive gap for every pair and every wall contact, at the volume fraction
asked for, above what random sequential placement reaches."""
import os
import subprocess
import sys

import numpy as np

import gen
import oracle


def packing(N, phi, seed, walls=False):
    rng = np.random.default_rng(seed)
    sh = gen.aspect_shapes(N, rng)
    vol = float(np.sum(4.0 / 3.0 * np.pi * sh[:, 0].astype(np.float64) * sh[:, 1] ** 2))
    if walls:
        Lxy = (vol / phi / 2.0) ** (1.0 / 3.0)
        L, per, w = (Lxy, Lxy, 2.0 * Lxy), (True, True, False), [(0.0, 1), (2.0 * Lxy, -1)]
    else:
        Lc = (vol / phi) ** (1.0 / 3.0)
        L, per, w = (Lc, Lc, Lc), (True, True, True), []
    parts, dom, sweeps = gen.grow(sh, L, periodic=per, walls=w, seed=seed)
    return parts, dom, vol / float(np.prod(L)), sweeps


def check_gaps(parts, dom):
    pi, pj = oracle.candidates(parts, dom, 1.0)
    cp = oracle.closest(parts, dom, pi, pj)
    assert np.all((cp["status"] & (oracle.ST_NOCONV | oracle.ST_DEGENERATE)) == 0)
    a = np.minimum(parts["r_par"][pi], parts["r_perp"][pi]).astype(np.float64)
    # sizes reset from 1.02: gaps of order 2 % of the sizes (orientations rounded to float)
    assert np.all(cp["h"] > 5e-3 * a), cp["h"].min()
    return pi, pj, cp["h"]


def test_periodic_packing_at_half_volume_fraction():
    parts, dom, phi, sweeps = packing(400, 0.5, seed=3)
    assert abs(phi - 0.5) < 1e-12 and sweeps > 0
    pi, pj, h = check_gaps(parts, dom)
    assert len(pi) > 2 * 400            # a dense suspension: several partners each
    assert np.median(h) < 0.5


def test_packing_between_walls():
    parts, dom, phi, _ = packing(300, 0.45, seed=4, walls=True)
    pi, pj, h = check_gaps(parts, dom)
    assert np.any(pj < 0)               # particles near both walls
    assert set((-1 - pj[pj < 0]).tolist()) == {0, 1}


def test_same_packing_for_any_thread_count():
    code = ("import sys, hashlib; sys.path.insert(0, %r); sys.path.insert(0, %r); import numpy as np;"
            "from test_gen_growth import packing; p = packing(200, 0.45, seed=7)[0];"
            "print(hashlib.sha1(np.concatenate([p[k].astype(np.float64) for k in ('x','y','z','qw','qx')]).tobytes()).hexdigest())"
            % (os.path.dirname(os.path.dirname(os.path.abspath(__file__))), os.path.dirname(os.path.abspath(__file__))))
    out = []
    for threads in ("1", "4"):
        env = dict(os.environ, OMP_NUM_THREADS=threads)
        out.append(subprocess.check_output([sys.executable, "-c", code], env=env).decode().strip())
    assert out[0] == out[1]
