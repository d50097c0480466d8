"""Ensemble mode: many independent suspensions, one launch per stage.

The suspensions are independent problems, so the definition of the ensemble
result is each suspension's own result: every member is checked against the
oracle run on that suspension alone (its own box and walls), and the whole
ensemble against separate single-suspension runs of the library (bit for bit
in FP64 with the deterministic reduction).  Also: a CUDA-graph replay of the
ensemble step, the autotuner, and argument errors.
"""
import numpy as np
import pytest

import gen
import oracle
from parity import compare, gpu_params, oracle_ref, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lub():
    import torch

    import paper_1308_6482_gb300 as lub
    from paper_1308_6482_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    return lub


def one_sphere_near_wall():
    parts = dict(x=np.array([20.0]), y=np.array([21.0]), z=np.array([3.4]),
                 qw=np.ones(1, np.float32), qx=np.zeros(1, np.float32), qy=np.zeros(1, np.float32),
                 qz=np.zeros(1, np.float32), r_par=np.full(1, 3.0, np.float32), r_perp=np.full(1, 3.0, np.float32))
    gen.velocities(parts, np.random.default_rng(3))
    return parts, dict(L=(40.0, 40.0, 40.0), periodic=(True, True, False), walls=[(0.0, 1)])


def empty_suspension():
    z = np.zeros(0)
    zf = np.zeros(0, np.float32)
    parts = dict(x=z, y=z, z=z, qw=zf, qx=zf, qy=zf, qz=zf, r_par=zf, r_perp=zf, vx=zf, vy=zf, vz=zf, wx=zf, wy=zf,
                 wz=zf)
    return parts, dict(L=(50.0, 50.0, 50.0), periodic=(True, True, True), walls=[])


def aspect_suspension(N, phi, seed, walls):
    rng = np.random.default_rng(seed)
    lam = np.exp(rng.uniform(np.log(1 / 3), np.log(3.0), N))
    sh = np.stack([4.5 * lam ** (2 / 3), 4.5 * lam ** (-1 / 3)], 1).astype(np.float32)
    vol = float(np.sum(4 / 3 * np.pi * sh[:, 0].astype(np.float64) * sh[:, 1] ** 2))
    L = (vol / phi) ** (1 / 3)
    if walls:
        return gen.suspension(sh, (L, L, L), periodic=(True, True, False), walls=[(0.0, 1), (L, -1)],
                              attach_prob=0.8, wall_min=1e-3, seed=seed)
    return gen.suspension(sh, (L, L, L), attach_prob=0.8, seed=seed)


def members():
    return [gen.config_prolate_wall(seed=1),
            gen.config_mixed_suspension(N=1500, phi=0.3, seed=5),
            empty_suspension(),
            one_sphere_near_wall(),
            aspect_suspension(800, 0.2, 11, walls=True),
            aspect_suspension(1200, 0.35, 12, walls=False)]


def run_ensemble(lub, sus, prec, deterministic=0, tune=False):
    import torch
    parts, doms, off = lub.make_ensemble(sus)
    P = lub.DeviceParticles(parts, batch_offsets=off)
    pl = lub.Pipeline(P, doms, gpu_params(prec))
    pl.build_pairs()
    if tune:
        pl.autotune(reps=1)
    pl.closest()
    pl.resistance()
    pl.apply(deterministic=deterministic)
    torch.cuda.synchronize()
    return pl, pl.results(), off


def split(res, off, b):
    """The part of an ensemble result that belongs to suspension b, local indices."""
    o0, o1 = int(off[b]), int(off[b + 1])
    sel = (res["pi"] >= o0) & (res["pi"] < o1)
    out = {k: v[sel] for k, v in res.items() if k not in ("force", "torque")}
    out["pi"] = res["pi"][sel] - o0
    out["pj"] = np.where(res["pj"][sel] >= 0, res["pj"][sel] - o0, res["pj"][sel])
    out["force"] = res["force"][o0:o1]
    out["torque"] = res["torque"][o0:o1]
    return out


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_every_member_matches_the_oracle(lub, prec):
    sus = members()
    _, res, off = run_ensemble(lub, sus, prec)
    # pairs never cross suspensions
    b_i = np.searchsorted(off, res["pi"], side="right") - 1
    wall = res["pj"] < 0
    b_j = np.searchsorted(off, np.where(wall, res["pi"], res["pj"]), side="right") - 1
    np.testing.assert_array_equal(b_i, b_j)
    for b, (parts, dom) in enumerate(sus):
        g = split(res, off, b)
        pi, pj = oracle.candidates(parts, dom, 1.0)
        np.testing.assert_array_equal(g["pi"], pi)
        np.testing.assert_array_equal(g["pj"], pj)
        if len(pi) == 0:
            assert np.all(g["force"] == 0) and np.all(g["torque"] == 0)
            continue
        compare(parts, dom, g, oracle_ref(parts, dom, pi, pj), prec, pi, pj)
    assert len(res["pi"]) > 1000 and np.any(res["pj"] < 0)


def test_ensemble_equals_separate_runs_bitwise(lub):
    sus = members()
    _, res, off = run_ensemble(lub, sus, "fp64", deterministic=1)
    for b, (parts, dom) in enumerate(sus):
        if len(parts["x"]) == 0:
            continue
        g = split(res, off, b)
        one = run_gpu(parts, dom, "fp64", deterministic=1)
        for k in ("pi", "pj", "h", "n", "status", "FT", "lever", "force", "torque"):
            np.testing.assert_array_equal(g[k], one[k], err_msg="%s of suspension %d" % (k, b))


def test_graph_replay_of_the_ensemble_step(lub):
    import torch
    sus = members()
    parts, doms, off = lub.make_ensemble(sus)
    P = lub.DeviceParticles(parts, batch_offsets=off)
    pl = lub.Pipeline(P, doms, gpu_params("mixed"))
    pl.build_pairs()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        pl.step(stream=s)                      # eager: uploads the tables, sizes the scratch
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        pl.step(stream=s)
    # move every particle a little, replay, and compare with an eager step on the same poses
    rng = np.random.default_rng(17)
    for k in ("x", "y", "z"):
        P.t[k] += torch.as_tensor(rng.normal(0, 0.01, P.n), device=P.t[k].device)
    g.replay()
    torch.cuda.synchronize()
    rep = pl.results()
    pl2 = lub.Pipeline(P, doms, gpu_params("mixed"))
    pl2.step(sync_count=True)
    torch.cuda.synchronize()
    eag = pl2.results()
    np.testing.assert_array_equal(rep["pi"], eag["pi"])
    np.testing.assert_array_equal(rep["pj"], eag["pj"])
    np.testing.assert_array_equal(rep["h"], eag["h"])
    np.testing.assert_array_equal(rep["FT"], eag["FT"])


def test_autotuner_shapes_and_unchanged_results(lub):
    sus = members()
    pl, tuned, _ = run_ensemble(lub, sus, "fp64", deterministic=1, tune=True)
    shapes = {lub.TUNE_NAMES[k]: lub.lub_get_launch_shape(pl.ctx.h, k) for k in range(lub.LUB_TUNE_COUNT)}
    for name in ("closest_fp64", "resistance", "apply", "sweep"):
        b, p = shapes[name]
        assert b >= 32 and b % 32 == 0 and 1 <= p <= 256, (name, b, p)
    _, plain, _ = run_ensemble(lub, sus, "fp64", deterministic=1)
    for k in ("pi", "pj", "h", "n", "FT", "force", "torque"):
        np.testing.assert_array_equal(tuned[k], plain[k], err_msg=k)
    # shapes can be set and reset by hand; a shape outside the kernel's limit is refused
    lub.lub_set_launch_shape(pl.ctx.h, lub.LUB_TUNE_RESISTANCE, 64, 4)
    assert lub.lub_get_launch_shape(pl.ctx.h, lub.LUB_TUNE_RESISTANCE) == (64, 4)
    lub.lub_set_launch_shape(pl.ctx.h, lub.LUB_TUNE_RESISTANCE, 0, 0)
    assert lub.lub_get_launch_shape(pl.ctx.h, lub.LUB_TUNE_RESISTANCE) == (0, 0)
    with pytest.raises(lub.LubError):
        lub.lub_set_launch_shape(pl.ctx.h, lub.LUB_TUNE_RESISTANCE, 512, 4)


def test_ensemble_argument_errors(lub):
    sus = members()[:2]
    parts, doms, off = lub.make_ensemble(sus)
    bad = off.copy()
    bad[-1] -= 1                              # does not end at n
    P = lub.DeviceParticles(parts, batch_offsets=bad)
    pl = lub.Pipeline(P, doms, gpu_params("fp64"))
    with pytest.raises(lub.LubError) as e:
        pl.build_pairs()
    assert e.value.code == lub.LUB_ERR_ARG
    bad = off.copy()
    bad[1] = bad[2] + 1                        # decreasing
    P = lub.DeviceParticles(parts, batch_offsets=bad)
    pl = lub.Pipeline(P, doms, gpu_params("fp64"))
    with pytest.raises(lub.LubError):
        pl.build_pairs()
    # a pair that crosses two suspensions is flagged, not computed
    P = lub.DeviceParticles(parts, batch_offsets=off)
    pl = lub.Pipeline(P, doms, gpu_params("fp64"))
    pl.set_pairs(np.array([0, 1], np.int32), np.array([int(off[1]), 2], np.int32))
    pl.closest()
    r = pl.results()
    assert r["status"][0] & lub.LUB_ST_DEGENERATE
    assert not (r["status"][1] & lub.LUB_ST_DEGENERATE)
