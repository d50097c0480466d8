"""The link-based lubrication kernel (lub_links, Eq. methods:dlub) against
the oracle's brute force: the same contributing links per pair (an integer,
exact), forces and torques equal up to the order of the sums."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

MU, QBAR = 1.0 / 6.0, 0.6


@pytest.fixture(scope="module")
def lub():
    import torch

    import paper_1308_6482_gb300 as lub
    from paper_1308_6482_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    return lub


def run(lub, parts, dom, pi=None, pj=None):
    import torch
    pl = lub.Pipeline(parts, dom, lub.default_params(precision="mixed"))
    if pi is None:
        pl.build_pairs()
    else:
        pl.set_pairs(pi, pj)
    F, T, nl = pl.links(QBAR)
    torch.cuda.synchronize()
    m = min(pl.count(), pl.cap)
    C = pl.cap
    return (pl.pair_i[:m].cpu().numpy(), pl.pair_j[:m].cpu().numpy(),
            F.cpu().numpy().reshape(3, C)[:, :m].T, T.cpu().numpy().reshape(6, C)[:, :m].T, nl[:m].cpu().numpy())


def check(parts, dom, pi, pj, F, T, nl):
    ref = oracle.links(parts, dom, pi, pj, MU, QBAR)
    np.testing.assert_array_equal(nl, ref["links"])
    sf = max(np.abs(ref["F"]).max(), 1e-300)
    st = max(np.abs(ref["T"]).max(), 1e-300)
    np.testing.assert_allclose(F, ref["F"], rtol=1e-9, atol=1e-12 * sf)
    np.testing.assert_allclose(T, ref["T"], rtol=1e-9, atol=1e-12 * st)
    return ref


def test_single_links_worked_by_hand(lub):
    for xj, r, want in ((1.3, 0.6, 1), (2.05, 0.9, 1)):
        p = {k: np.zeros(2) for k in ("x", "y", "z", "qx", "qy", "qz", "vx", "vy", "vz", "wx", "wy", "wz")}
        p["qw"] = np.ones(2)
        p["x"][1] = xj
        p["r_par"] = p["r_perp"] = np.full(2, r)
        p["vx"][1] = -0.01
        dom = dict(L=(60.0, 60.0, 60.0), periodic=(False, False, False), walls=[])
        pi, pj = np.array([0], np.int32), np.array([1], np.int32)
        _, _, F, T, nl = run(lub, p, dom, pi, pj)
        assert nl[0] == want
        # the library keeps radii and velocities in float32
        r32, v32 = float(np.float32(r)), float(np.float32(-0.01))
        h = (xj - r32) - r32
        lam = 1.0 / r32
        fx = 3 * QBAR * MU / (2 * lam) * (1 / h ** 2 - 1) * v32   # e = -x^, e.(v_i - v_j) = v_j
        np.testing.assert_allclose(F[0], [fx, 0, 0], rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("kind", ["aspect", "spheres"])
def test_pair_stream_parity(lub, kind):
    # 600 pairs over the links' range: h from 0.02 to 3 lattice units
    parts, dom, pi, pj = gen.pair_stream(600, seed=81, kind=kind, gap_range=(0.02, 3.0))
    rng = np.random.default_rng(82)
    for k in ("wx", "wy", "wz"):
        parts[k] = rng.normal(0, 1e-3, len(parts["x"])).astype(np.float32)
    qi, qj, F, T, nl = run(lub, parts, dom, pi, pj)
    ref = check(parts, dom, pi, pj, F, T, nl)
    assert (ref["links"] > 0).mean() > 0.5 and ref["links"].max() > 20


def test_suspension_parity_with_the_library_pair_list(lub):
    parts, dom = gen.config_mixed_suspension(N=1500, phi=0.3, seed=83)
    pi, pj, F, T, nl = run(lub, parts, dom)
    qi, qj = oracle.candidates(parts, dom, 1.0)
    np.testing.assert_array_equal(pi, qi)
    check(parts, dom, pi, pj, F, T, nl)


def test_wall_pairs_give_nothing(lub):
    parts, dom = gen.config_prolate_wall(seed=2)
    pi, pj, F, T, nl = run(lub, parts, dom)
    w = pj < 0
    assert w.any()
    assert np.all(nl[w] == 0) and not np.any(F[w]) and not np.any(T[w])
    check(parts, dom, pi[~w], pj[~w], F[~w], T[~w], nl[~w])
