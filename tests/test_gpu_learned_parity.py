"""The learned warm start against the oracle in every form the benchmark times.

The network only chooses where Newton starts; the closest points, gaps and
forces it leads to are defined by the paper alone (Sec. III A: the common
normal and the gap h; Sec. III B and the Appendix: the resistance), so each
learned form must meet the same element-by-element bounds as the cold start:

* mixed precision with the network starting every pair (LUB_WARM_MLP_ALL:
  FP32 Newton from the network's start, the float-float step, FP32
  resistance) on fresh min-axis-scaled pairs, with both tensor-core engines
  (mma.sync inside the solve's kernel, tcgen05 as a launch of its own);
* mixed precision with the network starting only the FP64 solves of the
  pairs the FP32 stage fails (LUB_WARM_MLP), every spheroid pair made to fail
  by an FP32 tolerance it cannot reach: those FP64 solves take fewer
  iterations than from the line of centres and give the same results;
* the ensemble (many suspensions in one launch per stage), every member
  against the oracle run on it alone, in both precisions;
* a window of the large dense run: its growth-packed base slab (16,384
  spheroids at Phi = 0.5 between two walls), the pair list from the cell-list
  builder, mixed precision.
"""
import os

import numpy as np
import pytest

import gen
import oracle
from parity import compare, gpu_params, oracle_ref

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1308_6482_gb300",
                       "mlp_weights.npz")


@pytest.fixture(scope="module")
def env():
    import torch

    import paper_1308_6482_gb300 as lub
    from paper_1308_6482_gb300 import build
    from paper_1308_6482_gb300.mlp import WarmStartMLP
    build.build()
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    return lub, torch, WarmStartMLP.load(WEIGHTS)


def learned(env, parts, dom, prec, pi=None, pj=None, engine="mma_sync", offsets=None, warm="mlp_all", **kw):
    lub, torch, net = env
    P = lub.DeviceParticles(parts, batch_offsets=offsets)
    pl = lub.Pipeline(P, dom, gpu_params(prec, warm_start={"mlp": lub.LUB_WARM_MLP, "mlp_all": lub.LUB_WARM_MLP_ALL,
                                                          "none": lub.LUB_WARM_NONE}[warm], **kw))
    net.install(pl.ctx)
    lub.lub_mlp_engine(pl.ctx.h, engine)
    if pi is None:
        pl.build_pairs()
    else:
        pl.set_pairs(pi, pj)
    pl.closest()
    pl.resistance()
    pl.apply()
    torch.cuda.synchronize()
    return pl.results()


@pytest.mark.parametrize("engine", ["mma_sync", "tcgen05"])
def test_learned_mixed_fresh_pairs(env, engine):
    # 20,000 fresh pairs (a seed the training set never used), gaps log-uniform
    # in [1e-4, 1] times the smaller semi-axis
    parts, dom, pi, pj = gen.pair_stream(20000, seed=9002, kind="aspect", gap_range=(1e-4, 1.0),
                                         gap_scale="min_axis")
    g = learned(env, parts, dom, "mixed", pi, pj, engine=engine)
    compare(parts, dom, g, oracle_ref(parts, dom, pi, pj), "mixed", pi, pj)


def test_learned_start_of_the_fp64_fallback(env):
    lub = env[0]
    parts, dom, pi, pj = gen.pair_stream(4000, seed=9003, kind="aspect", gap_range=(1e-4, 1.0),
                                         gap_scale="min_axis")
    cold = learned(env, parts, dom, "mixed", pi, pj, warm="none", newton_tol=1e-12)
    warm = learned(env, parts, dom, "mixed", pi, pj, warm="mlp", newton_tol=1e-12)
    fell = (warm["status"] & lub.LUB_ST_FP64) != 0
    assert fell.mean() > 0.9 and np.array_equal(fell, (cold["status"] & lub.LUB_ST_FP64) != 0)
    # the FP64 iterations from the network's start against those from the line of centres
    assert warm["iters"][fell].mean() < 0.85 * cold["iters"][fell].mean()
    compare(parts, dom, warm, oracle_ref(parts, dom, pi, pj), "mixed", pi, pj)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_learned_ensemble_every_member(env, prec):
    lub = env[0]
    rng_members = [gen.config_prolate_wall(seed=2),
                   gen.config_mixed_suspension(N=1200, phi=0.3, seed=15)]
    for seed, (n, phi) in enumerate(((700, 0.2), (900, 0.35), (600, 0.45))):
        rng = np.random.default_rng(60 + seed)
        sh = gen.aspect_shapes(n, rng)
        vol = float(np.sum(4 / 3 * np.pi * sh[:, 0].astype(np.float64) * sh[:, 1].astype(np.float64) ** 2))
        Lb = (vol / phi) ** (1 / 3)
        walls = [(0.0, 1), (Lb, -1)] if seed % 2 == 0 else []
        per = (True, True, not walls)
        p, d, _ = gen.grow(sh, (Lb, Lb, Lb), periodic=per, walls=walls, seed=70 + seed)
        rng_members.append((p, d))
    parts, doms, off = lub.make_ensemble(rng_members)
    res = learned(env, parts, doms, prec, offsets=off, warm="mlp_all" if prec == "mixed" else "mlp")
    for b, (p, d) in enumerate(rng_members):
        o0, o1 = int(off[b]), int(off[b + 1])
        sel = (res["pi"] >= o0) & (res["pi"] < o1)
        g = {k: v[sel] for k, v in res.items() if k not in ("force", "torque")}
        g["pi"] = res["pi"][sel] - o0
        g["pj"] = np.where(res["pj"][sel] >= 0, res["pj"][sel] - o0, res["pj"][sel])
        g["force"], g["torque"] = res["force"][o0:o1], res["torque"][o0:o1]
        pi, pj = oracle.candidates(p, d, 1.0)
        np.testing.assert_array_equal(g["pi"], pi)
        np.testing.assert_array_equal(g["pj"], pj)
        compare(p, d, g, oracle_ref(p, d, pi, pj), prec, pi, pj)


def test_learned_mixed_large_run_window(env):
    # the growth-packed slab the 1,048,576-particle run tiles 8 x 8: 16,384
    # spheroids, Phi = 0.5, walls at z = 0 and z = 1024
    parts, dom = gen.large_config(base_only=True)
    assert len(parts["x"]) == 16384 and len(dom["walls"]) == 2
    g = learned(env, parts, dom, "mixed")
    pi, pj = oracle.candidates(parts, dom, 1.0)
    np.testing.assert_array_equal(g["pi"], pi)
    np.testing.assert_array_equal(g["pj"], pj)
    assert np.any(pj < 0) and len(pi) > 3 * len(parts["x"])
    compare(parts, dom, g, oracle_ref(parts, dom, pi, pj), "mixed", pi, pj)
