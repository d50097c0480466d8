"""lub_correct (closest points, resistance and the atomic scatter in one
call: one pass over the pairs in FP64; in mixed precision the kernels of
lub_closest_points and lub_resistance_apply on one set of particle records)
against the oracle (full parity), and against the three separate calls: the same pair lists and statuses, normals
and gaps equal up to rounding (the compiler may contract the same arithmetic
into multiply-adds differently inside the fused kernel), particle sums equal
up to the order of the atomic additions where the pair terms are the same.
"""
import numpy as np
import pytest

import gen
import oracle
from parity import compare, gpu_params, oracle_ref

# unit roundoff of each mode's arithmetic, for sums of the same terms in another order
EPS = {"fp64": 2.0 ** -53, "mixed": 2.0 ** -24}

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


def run(lub, parts, dom, prec, fused, pi=None, pj=None, per_pair=True, warm="none", offsets=None, net=None):
    import torch
    P = lub.DeviceParticles(parts, batch_offsets=offsets)
    pl = lub.Pipeline(P, dom, gpu_params(prec, warm_start={"none": 0, "previous": 1, "mlp": 2}[warm]))
    if net is not None:
        net.install(pl.ctx)
    if pi is None:
        pl.build_pairs()
    else:
        pl.set_pairs(pi, pj)
    if fused:
        pl.correct(per_pair=per_pair)
    else:
        pl.closest()
        pl.resistance()
        pl.apply()
    torch.cuda.synchronize()
    return pl.results()


def sums_close(a, b, res, prec):
    """Particle sums of the same pair terms in another order of additions."""
    n = len(a["force"])
    pi, pj = res["pi"], res["pj"]
    FT = res["FT"].astype(np.float64)
    lev = np.linalg.norm(res["lever"][:, :3].astype(np.float64), axis=1)
    levj = np.linalg.norm(res["lever"][:, 3:].astype(np.float64), axis=1)
    f = np.linalg.norm(FT[:, :3], axis=1)
    t = np.linalg.norm(FT[:, 3:], axis=1)
    sf, st = np.zeros(n), np.zeros(n)
    np.add.at(sf, pi, f)
    np.add.at(st, pi, t + lev * f)
    w = pj >= 0
    np.add.at(sf, pj[w], f[w])
    np.add.at(st, pj[w], (t + levj * f)[w])
    tol = 64 * EPS[prec]
    assert np.all(np.linalg.norm(a["force"] - b["force"], axis=1) <= tol * sf + 1e-30)
    assert np.all(np.linalg.norm(a["torque"] - b["torque"], axis=1) <= tol * st + 1e-30)


def same_pairs(a, b, prec):
    """Pair lists and statuses equal, normals and gaps equal up to rounding."""
    np.testing.assert_array_equal(a["pi"], b["pi"])
    np.testing.assert_array_equal(a["pj"], b["pj"])
    np.testing.assert_array_equal(a["status"] & 7, b["status"] & 7)
    ok = (b["status"] & 6) == 0
    tol_n = 1e-12 if prec == "fp64" else 1e-11
    assert np.abs(a["n"] - b["n"])[ok].max(initial=0) <= tol_n
    sc = np.abs(b["h"]) + 10.0
    assert np.all(np.abs(a["h"] - b["h"])[ok] <= 1e-10 * sc[ok])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["suspension", "wall", "stream"])
def test_fused_matches_separate_calls_and_oracle(lub, prec, case):
    pi = pj = None
    if case == "suspension":
        parts, dom = gen.config_mixed_suspension(N=3000, phi=0.3, seed=31)
    elif case == "wall":
        parts, dom = gen.config_prolate_wall(seed=3)
    else:  # gaps spanning the FP64 switch: the refinement kernel runs
        parts, dom, pi, pj = gen.pair_stream(3000, seed=33, kind="aspect", gap_range=(1e-4, 1.0),
                                             gap_scale="min_axis")
    sep = run(lub, parts, dom, prec, False, pi, pj)
    fus = run(lub, parts, dom, prec, True, pi, pj)
    same_pairs(fus, sep, prec)
    if pi is None:
        pi, pj = oracle.candidates(parts, dom, 1.0)
    compare(parts, dom, fus, oracle_ref(parts, dom, pi, pj), prec, pi, pj)


@pytest.mark.parametrize("fused", [False, True])
def test_mixed_fp64_fallback(lub, fused):
    """Mixed mode with an FP32 Newton tolerance it cannot reach: every
    spheroid pair goes to the work list and is solved again in FP64 from the
    line of centres (LUB_ST_FP64), with oracle parity."""
    import torch
    parts, dom, pi, pj = gen.pair_stream(2000, seed=37, kind="aspect", gap_range=(1e-4, 1.0),
                                         gap_scale="min_axis")
    P = lub.DeviceParticles(parts)
    pl = lub.Pipeline(P, dom, gpu_params("mixed", newton_tol=1e-12))
    pl.set_pairs(pi, pj)
    if fused:
        pl.correct()
    else:
        pl.closest()
        pl.resistance()
        pl.apply()
    torch.cuda.synchronize()
    g = pl.results()
    sph = (parts["r_par"][pi] == parts["r_perp"][pi]) & (parts["r_par"][pj] == parts["r_perp"][pj])
    assert np.all((g["status"][~sph] & lub.LUB_ST_FP64) != 0)
    compare(parts, dom, g, oracle_ref(parts, dom, pi, pj), "mixed", pi, pj)


def test_optional_outputs_and_accumulate(lub):
    import torch
    parts, dom = gen.config_mixed_suspension(N=2000, phi=0.3, seed=35)
    full = run(lub, parts, dom, "mixed", True)
    lean = run(lub, parts, dom, "mixed", True, per_pair=False)
    np.testing.assert_array_equal(lean["n"], full["n"])
    sums_close(lean, full, full, "mixed")
    # accumulate: a second pass adds the same forces again
    pl = lub.Pipeline(parts, dom, gpu_params("mixed"))
    pl.build_pairs()
    pl.correct()
    lub.lub_correct(pl.ctx.h, pl.P.c, pl.D, pl.prm, pl.pair_i, pl.pair_j, pl.d_count, pl.cap, pl.nrm, None, None,
                    None, None, None, pl.force, pl.torque, 1)
    torch.cuda.synchronize()
    twice = pl.results()
    # the same pair terms summed twice, in another order of atomic additions
    half = dict(twice, force=twice["force"] / 2, torque=twice["torque"] / 2)
    sums_close(half, full, full, "mixed")


def test_fused_ensemble_and_warm_starts(lub):
    from paper_1308_6482_gb300.mlp import WarmStartMLP
    sus = [gen.config_prolate_wall(seed=1), gen.config_mixed_suspension(N=1500, phi=0.3, seed=5)]
    parts, doms, off = lub.make_ensemble(sus)
    sep = run(lub, parts, doms, "mixed", False, offsets=off)
    fus = run(lub, parts, doms, "mixed", True, offsets=off)
    same_pairs(fus, sep, "mixed")
    for b, (p, d) in enumerate(sus):
        o0, o1 = int(off[b]), int(off[b + 1])
        sel = (fus["pi"] >= o0) & (fus["pi"] < o1)
        g = {k: v[sel] for k, v in fus.items() if k not in ("force", "torque")}
        g["pi"] = g["pi"] - o0
        g["pj"] = np.where(g["pj"] >= 0, g["pj"] - o0, g["pj"])
        g["force"], g["torque"] = fus["force"][o0:o1], fus["torque"][o0:o1]
        compare(p, d, g, oracle_ref(p, d, g["pi"], g["pj"]), "mixed", g["pi"], g["pj"])
    net = WarmStartMLP.load()
    p2, d2, qi, qj = gen.pair_stream(2000, seed=37, kind="aspect", gap_range=(1e-4, 1.0), gap_scale="min_axis")
    sep = run(lub, p2, d2, "fp64", False, qi, qj, warm="mlp", net=net)
    fus = run(lub, p2, d2, "fp64", True, qi, qj, warm="mlp", net=net)
    same_pairs(fus, sep, "fp64")
    assert np.mean(fus["iters"]) < np.mean(run(lub, p2, d2, "fp64", True, qi, qj)["iters"])
    compare(p2, d2, fus, oracle_ref(p2, d2, qi, qj), "fp64", qi, qj)


def test_fused_degenerate_pairs(lub):
    parts, dom, pi, pj = gen.pair_stream(8, seed=47, kind="aspect", gap_range=(1e-3, 0.1))
    n = len(parts["x"])
    bad_i = np.r_[pi, [0, -5, n + 3, 2, 4]].astype(np.int32)
    bad_j = np.r_[pj, [0, 1, 1, n + 7, -9]].astype(np.int32)
    for prec in ("fp64", "mixed"):
        g = run(lub, parts, dom, prec, True, bad_i, bad_j)
        assert np.all(g["status"][len(pi):] & lub.LUB_ST_DEGENERATE)
        assert np.all(g["FT"][len(pi):] == 0)
        ok = run(lub, parts, dom, prec, True, pi, pj)
        np.testing.assert_array_equal(g["force"], ok["force"]) if prec == "fp64" else sums_close(g, ok, ok, prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_resistance_apply_in_one_pass(lub, prec):
    """lub_resistance_apply: resistance and the scatter in one pass."""
    import torch
    parts, dom = gen.config_prolate_wall(seed=3)
    sep = run(lub, parts, dom, prec, False)
    pl = lub.Pipeline(parts, dom, gpu_params(prec))
    pl.step(form="merged", sync_count=True)
    torch.cuda.synchronize()
    mer = pl.results()
    same_pairs(mer, sep, prec)
    pi, pj = oracle.candidates(parts, dom, 1.0)
    compare(parts, dom, mer, oracle_ref(parts, dom, pi, pj), prec, pi, pj)
    # FT and lever are optional
    pl2 = lub.Pipeline(parts, dom, gpu_params(prec))
    pl2.build_pairs()
    pl2.closest()
    pl2.resistance_apply(per_pair=False)
    torch.cuda.synchronize()
    sums_close(pl2.results(), mer, mer, prec)
