"""The large dense run at its full size, in the benchmark's launch configuration.

1,048,576 spheroids (aspect ratios log-uniform in [1/3, 3]) at Phi = 0.5 in a
1024^3 box periodic in x and y between plane walls at z = 0 and z = 1024,
run the way the benchmark times it: mixed precision, the gated learned warm
start, launch shapes from the autotuner, one lub_pairs_build + lub_correct
step captured in a CUDA graph and replayed.  The oracle's pre-filter over
all pairs is O(N^2), out of reach at this size, so the checks are sampled and
the oracle computes each sampled output on its own:

* pair list: every pair that touches a particle of an inner window (a
  48 x 48 column of the box through both walls), bit for bit, against the
  oracle's pre-filter over the particles within reach of the window;
* per pair: gap, normal, status, forces, torques and lever arms of every pair
  touching the window and of 20,000 pairs drawn from the whole list, within
  the parity bounds of the mixed mode;
* per particle: the force and torque sums of the window's particles (their
  pair sets are the verified ones) within the sums of their pairs' bounds.

Properties that hold at any size are checked on the whole list: canonical
order, no pair twice, every index in range, the count within capacity.
"""
import os

import numpy as np
import pytest

import gen
import oracle
from parity import compare, oracle_ref

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1308_6482_gb300",
                       "mlp_weights.npz")
X0, Y0, W = 500.0, 500.0, 48.0  # the inner window: x in [X0, X0 + W), y in [Y0, Y0 + W), every z


@pytest.fixture(scope="module")
def run():
    import torch

    import paper_1308_6482_gb300 as lub
    from paper_1308_6482_gb300 import build
    from paper_1308_6482_gb300.mlp import WarmStartMLP
    build.build()
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    parts, dom = gen.large_config()
    assert len(parts["x"]) == 1 << 20 and len(dom["walls"]) == 2
    rmax = float(max(parts["r_par"].max(), parts["r_perp"].max())) + 0.05
    P = lub.DeviceParticles(parts, dev, max_semi_axis=rmax)
    pl = lub.Pipeline(P, dom, lub.default_params(precision="mixed", warm_start=lub.LUB_WARM_MLP), capacity=1024,
                      device=dev)
    WarmStartMLP.load(WEIGHTS, device=dev).install(pl.ctx)
    npairs = pl.build_pairs()
    pl._alloc(int(npairs * 1.3) + 4096, dev)
    pl.build_pairs()
    pl.autotune(reps=3)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        pl.step(form="fused", pair_forces=True, stream=stream)
        pl.step(form="fused", pair_forces=True, stream=stream)
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        pl.step(form="fused", pair_forces=True, stream=stream)
    stream.synchronize()
    # every output the checks read is overwritten before the replay, so the
    # results below are the replayed graph's
    for t, v in ((pl.pair_i, -7), (pl.pair_j, -7), (pl.nrm, float("nan")), (pl.gap, float("nan")),
                 (pl.status, 255), (pl.FT, float("nan")), (pl.lever, float("nan")), (pl.force, float("nan")),
                 (pl.torque, float("nan"))):
        t.fill_(v)
    with torch.cuda.stream(stream):
        g.replay()
    stream.synchronize()
    res = pl.results()
    assert pl.count() <= pl.cap
    del g
    return parts, dom, res, rmax


def window(parts, margin=0.0):
    x, y = parts["x"], parts["y"]
    return (x >= X0 - margin) & (x < X0 + W + margin) & (y >= Y0 - margin) & (y < Y0 + W + margin)


def test_large_run_whole_list_properties(run):
    parts, dom, res, rmax = run
    pi, pj = res["pi"].astype(np.int64), res["pj"].astype(np.int64)
    n = len(parts["x"])
    assert len(pi) > 4 * n
    assert np.all((pi >= 0) & (pi < n))
    wall = pj < 0
    assert np.all(pj[~wall] > pi[~wall]) and np.all(pj[wall] >= -2)
    # particle pairs by (i, j), then wall pairs by (i, w), none twice
    nw = int(wall.sum())
    assert nw > 0 and np.all(wall[len(pi) - nw:])
    kp = pi[:len(pi) - nw] * n + pj[:len(pi) - nw]
    kw = pi[len(pi) - nw:] * 2 + (-1 - pj[len(pi) - nw:])
    assert np.all(np.diff(kp) > 0) and np.all(np.diff(kw) > 0)
    # the sums are finite everywhere
    assert np.all(np.isfinite(res["force"])) and np.all(np.isfinite(res["torque"]))


def test_large_run_window_pairs_and_sampled_results(run):
    parts, dom, res, rmax = run
    pi, pj = res["pi"], res["pj"]
    inner = window(parts)
    reach = 2.0 * rmax + 1.0 + 0.5  # 2 Rmax + Delta_L, and more
    sel = np.flatnonzero(window(parts, margin=reach))
    assert 2000 < inner.sum() and len(sel) < 20000
    sub = {k: v[sel] for k, v in parts.items()}
    si, sj = oracle.candidates(sub, dom, 1.0)
    oi = sel[si]
    oj = np.where(sj >= 0, sel[np.maximum(sj, 0)], sj)
    touch_o = inner[oi] | ((oj >= 0) & inner[np.maximum(oj, 0)])
    touch_g = inner[pi] | ((pj >= 0) & inner[np.maximum(pj, 0)])
    np.testing.assert_array_equal(pi[touch_g], oi[touch_o])
    np.testing.assert_array_equal(pj[touch_g], oj[touch_o])
    assert set(pj[touch_g][pj[touch_g] < 0]) == {-1, -2}  # the window reaches both walls
    # per pair: the window's pairs and 20,000 drawn from the whole list; per
    # particle: the window's particles
    rng = np.random.default_rng(20)
    K = np.union1d(np.flatnonzero(touch_g), rng.choice(len(pi), 20000, replace=False))
    g = {k: res[k][K] for k in ("n", "h", "status", "FT", "lever")}
    g["force"], g["torque"] = res["force"], res["torque"]
    ref = oracle_ref(parts, dom, pi[K], pj[K])
    compare(parts, dom, g, ref, "mixed", pi[K], pj[K], check_particles=np.flatnonzero(inner))
