"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Inputs are seeded synthetic pairs and suspensions from ``gen``; expected
values always come from ``oracle``.  Tolerances are documented in
``tests/parity.py``.
"""
import numpy as np
import pytest

import gen
import oracle
from parity import compare, oracle_ref, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_1308_6482_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("kind", ["aspect", "mixed", "spheres"])
def test_pair_stream_parity(prec, kind):
    # 2,500 pairs: many tiles of 128 threads plus a ragged tail
    parts, dom, pi, pj = gen.pair_stream(2500, seed=41, kind=kind, gap_range=(1e-4, 1.0))
    g = run_gpu(parts, dom, prec, pi, pj)
    ref = oracle_ref(parts, dom, pi, pj)
    compare(parts, dom, g, ref, prec, pi, pj)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_min_axis_scaled_gaps(prec):
    # gaps log-uniform in [1e-4, 1] times the smaller semi-axis (h/a from near contact to the list cut-off)
    parts, dom, pi, pj = gen.pair_stream(3000, seed=43, kind="aspect", gap_range=(1e-4, 1.0), gap_scale="min_axis")
    g = run_gpu(parts, dom, prec, pi, pj)
    ref = oracle_ref(parts, dom, pi, pj)
    compare(parts, dom, g, ref, prec, pi, pj)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_suspension_with_wall_full_step(prec):
    parts, dom = gen.config_prolate_wall(seed=1)
    g = run_gpu(parts, dom, prec)
    pi, pj = oracle.candidates(parts, dom, 1.0)
    np.testing.assert_array_equal(g["pi"], pi)
    np.testing.assert_array_equal(g["pj"], pj)
    assert np.any(pj < 0)
    ref = oracle_ref(parts, dom, pi, pj)
    compare(parts, dom, g, ref, prec, pi, pj)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_mixed_suspension_full_step(prec):
    parts, dom = gen.config_mixed_suspension(N=3000, phi=0.3, seed=7)
    g = run_gpu(parts, dom, prec)
    pi, pj = oracle.candidates(parts, dom, 1.0)
    np.testing.assert_array_equal(g["pi"], pi)
    np.testing.assert_array_equal(g["pj"], pj)
    ref = oracle_ref(parts, dom, pi, pj)
    compare(parts, dom, g, ref, prec, pi, pj)


def test_full_size_suspension_parity():
    """The 32,768-particle, Phi = 0.3 mixed suspension the benchmark times, in
    the benchmark's launch configuration: the whole pair list and every pair
    and particle result against the oracle."""
    parts, dom = gen.config_mixed_suspension()
    g = run_gpu(parts, dom, "mixed")
    pi, pj = oracle.candidates(parts, dom, 1.0)
    np.testing.assert_array_equal(g["pi"], pi)
    np.testing.assert_array_equal(g["pj"], pj)
    ref = oracle_ref(parts, dom, pi, pj)
    compare(parts, dom, g, ref, "mixed", pi, pj)


def test_contact_branch_parity():
    # h_c = 0.01, eps_c = 100 (Sec. IV C): gaps on both sides of h_c and small overlaps
    parts, dom, pi, pj = gen.pair_stream(1500, seed=45, kind="aspect", gap_range=(1e-4, 0.05))
    rng = np.random.default_rng(3)
    cp0 = oracle.closest(parts, dom, pi, pj)
    push = rng.uniform(0, 0.03, len(pi))  # some become overlapping
    for kk, ax in zip(("x", "y", "z"), range(3)):
        parts[kk] = parts[kk].copy()
        parts[kk][pj] -= push * cp0["n"][:, ax]
    for prec in ("fp64", "mixed"):
        g = run_gpu(parts, dom, prec, pi, pj, h_c=0.01, eps_c=100.0)
        ref = oracle_ref(parts, dom, pi, pj, h_c=0.01, eps_c=100.0)
        assert np.any(ref["cp"]["h"] < 0)
        compare(parts, dom, g, ref, prec, pi, pj)


def test_overlap_without_contact_model():
    parts, dom, pi, pj = gen.pair_stream(500, seed=46, kind="mixed", gap_range=(1e-3, 0.05))
    cp0 = oracle.closest(parts, dom, pi, pj)
    for kk, ax in zip(("x", "y", "z"), range(3)):
        parts[kk] = parts[kk].copy()
        parts[kk][pj] -= 2 * cp0["h"] * cp0["n"][:, ax]
    g = run_gpu(parts, dom, "mixed", pi, pj)
    ref = oracle_ref(parts, dom, pi, pj)
    assert np.all(g["status"] & 1)
    assert np.all(g["FT"] == 0)
    compare(parts, dom, g, ref, "mixed", pi, pj)


def test_deterministic_apply_is_reproducible():
    parts, dom = gen.config_mixed_suspension(N=3000, phi=0.3, seed=8)
    a = run_gpu(parts, dom, "mixed", deterministic=1)
    b = run_gpu(parts, dom, "mixed", deterministic=1)
    c = run_gpu(parts, dom, "mixed", deterministic=0)
    np.testing.assert_array_equal(a["force"], b["force"])
    np.testing.assert_array_equal(a["torque"], b["torque"])
    np.testing.assert_allclose(a["force"], c["force"], rtol=0, atol=1e-5 * np.abs(a["force"]).max())
    pi, pj = a["pi"], a["pj"]
    ref = oracle_ref(parts, dom, pi, pj)
    compare(parts, dom, a, ref, "mixed", pi, pj)


def test_empty_inputs():
    import torch

    import paper_1308_6482_gb300 as lub
    parts, dom = gen.config_mixed_suspension(N=50, phi=0.01, seed=9)
    pl = lub.Pipeline(parts, dom, lub.default_params(list_cutoff=0.0), capacity=64)
    cnt = pl.build_pairs()
    pl.closest()
    pl.resistance()
    pl.apply()
    torch.cuda.synchronize()
    r = pl.results()
    assert cnt == len(r["pi"])
    assert np.all(np.isfinite(r["force"]))
    # zero pairs given explicitly
    pl.set_pairs(np.zeros(0, np.int32), np.zeros(0, np.int32))
    pl.closest()
    pl.resistance()
    pl.apply()
    torch.cuda.synchronize()
    assert np.all(pl.results()["force"] == 0)


def test_capacity_overflow_reports_required_count():
    import torch

    import paper_1308_6482_gb300 as lub
    parts, dom = gen.config_mixed_suspension(N=2000, phi=0.3, seed=10)
    pi, pj = oracle.candidates(parts, dom, 1.0)
    pl = lub.Pipeline(parts, dom, lub.default_params(), capacity=16)
    rc, cnt = lub.lub_pairs_build(pl.ctx.h, pl.P.c, pl.D, pl.prm, pl.pair_i, pl.pair_j, pl.cap, pl.d_count,
                                  h_count=True)
    assert rc == lub.LUB_ERR_CAPACITY and cnt == len(pi)
    assert pl.count() == len(pi)
    # the downstream calls clamp to capacity and stay in bounds
    pl.closest()
    pl.resistance()
    pl.apply()
    torch.cuda.synchronize()
    # growing and rebuilding gives the full list
    cnt2 = pl.build_pairs()
    assert cnt2 == len(pi)
    np.testing.assert_array_equal(pl.results()["pi"], pi)


def crowded_particle(n_around=30, gap=0.5):
    """Particle 0 (the lowest index, so every pair counts for it) with
    n_around small spheres at the given gap around it: more partners than
    the builder's per-particle slots, so the overflow path runs."""
    rng = np.random.default_rng(5)
    k = np.arange(n_around) + 0.5
    th = np.arccos(1 - 2 * k / n_around)
    ph = np.pi * (1 + 5 ** 0.5) * k
    u = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
    c = np.array([50.0, 50.0, 50.0])
    pos = np.vstack([c, c + (3.0 + gap + 1.0) * u])
    n = len(pos)
    r = np.r_[3.0, np.full(n_around, 1.0)].astype(np.float32)
    q = gen.random_quaternions(n, rng)
    parts = dict(x=pos[:, 0].copy(), y=pos[:, 1].copy(), z=pos[:, 2].copy(), qw=q[:, 0].copy(), qx=q[:, 1].copy(),
                 qy=q[:, 2].copy(), qz=q[:, 3].copy(), r_par=r, r_perp=r.copy())
    gen.velocities(parts, rng)
    return parts, dict(L=(100.0, 100.0, 100.0), periodic=(True, True, True), walls=[])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_more_partners_than_slots(prec):
    import paper_1308_6482_gb300 as lub
    parts, dom = crowded_particle()
    pi, pj = oracle.candidates(parts, dom, 1.0)
    assert np.sum(pi == 0) > 16
    g = run_gpu(parts, dom, prec)
    np.testing.assert_array_equal(g["pi"], pi)
    np.testing.assert_array_equal(g["pj"], pj)
    compare(parts, dom, g, oracle_ref(parts, dom, pi, pj), prec, pi, pj)
    # the overflow entries need room in the arrays while the build runs: the
    # required capacity reported is the pairs plus those entries
    pl = lub.Pipeline(parts, dom, lub.default_params(), capacity=len(pi))
    rc, need = lub.lub_pairs_build(pl.ctx.h, pl.P.c, pl.D, pl.prm, pl.pair_i, pl.pair_j, pl.cap, pl.d_count,
                                   h_count=True)
    assert rc == lub.LUB_ERR_CAPACITY and need == len(pi) + (np.sum(pi == 0) - 16)
    pl2 = lub.Pipeline(parts, dom, lub.default_params(), capacity=need)
    assert pl2.build_pairs() == len(pi)
    np.testing.assert_array_equal(pl2.results()["pj"], pj)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_more_partners_than_slots_on_the_filters_edge(prec):
    """The crowded particle with its 30 partners at a gap of Delta_L - 2e-5:
    every candidate lies inside the sweep's FP32 margin, so all are decided
    after the sweep, and those accepted beyond the particle's 16 slots stay
    in the buffer of decided candidates, where the compaction collects
    them."""
    parts, dom = crowded_particle(gap=1.0 - 2e-5)
    pi, pj = oracle.candidates(parts, dom, 1.0)
    assert np.sum(pi == 0) == 30
    g = run_gpu(parts, dom, prec)
    np.testing.assert_array_equal(g["pi"], pi)
    np.testing.assert_array_equal(g["pj"], pj)
    compare(parts, dom, g, oracle_ref(parts, dom, pi, pj), prec, pi, pj)


def test_degenerate_pairs_are_flagged_not_faulted():
    import torch
    parts, dom, pi, pj = gen.pair_stream(8, seed=47, kind="aspect", gap_range=(1e-3, 0.1))
    n = len(parts["x"])
    parts["r_perp"] = parts["r_perp"].copy()
    parts["r_perp"][1] = 0.0                       # zero semi-axis
    parts["x"] = parts["x"].copy()
    parts["x"][5] = parts["x"][4]
    parts["y"] = parts["y"].copy()
    parts["y"][5] = parts["y"][4]
    parts["z"] = parts["z"].copy()
    parts["z"][5] = parts["z"][4]                  # coincident centres
    bad_i = np.array([0, 4, n + 5, 2, -3, 6], np.int32)
    bad_j = np.array([1, 5, 3, -7, 2, 6], np.int32)  # bad index, bad wall index, i == j
    g = run_gpu(parts, dom, "mixed", bad_i, bad_j)
    torch.cuda.synchronize()
    assert np.all(g["status"] & 4)
    assert np.all(g["FT"] == 0)
    assert np.all(np.isfinite(g["force"]))


def test_packed_particles_give_the_same_results():
    """One device buffer for all particle arrays (one copy per update) is a
    layout change only."""
    import torch

    import paper_1308_6482_gb300 as lub
    parts, dom = gen.config_mixed_suspension(N=2000, phi=0.3, seed=12)
    a = run_gpu(parts, dom, "fp64", deterministic=1)
    P = lub.DeviceParticles(parts, packed=True)
    hb = P.host_blob(parts)
    assert hb.numel() == P.blob.numel()
    np.testing.assert_array_equal(P.t["y"].cpu().numpy(), parts["y"])
    np.testing.assert_array_equal(P.t["qz"].cpu().numpy(), parts["qz"])
    pl = lub.Pipeline(P, dom, lub.default_params(precision="fp64"))
    pl.step(deterministic=1, sync_count=True)
    torch.cuda.synchronize()
    b = pl.results()
    for k in ("pi", "pj", "n", "h", "FT", "force", "torque"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    # force and torque read back in one piece
    ft = pl.ft_particles.cpu().numpy()
    np.testing.assert_array_equal(ft[:3 * P.n].reshape(3, -1).T, b["force"])


@pytest.mark.parametrize("L", [9.5, 11.5, 14.5])
def test_small_periodic_boxes_list_every_pair_once(L):
    """Two or three cells per periodic axis: a neighbour cell can coincide with
    another under a different image offset; every pair must still be listed
    exactly once (against the oracle's all-pairs minimum-image search)."""
    import paper_1308_6482_gb300 as lub
    rng = np.random.default_rng(int(L * 10))
    sh = np.tile([[1.8, 1.2]], (14, 1)).astype(np.float32)   # Rmax 1.8: range 2 * 1.8 + 1 = 4.6
    parts, dom = gen.suspension(sh, (L, L, L), attach_prob=0.7, seed=int(L * 10))
    pi, pj = oracle.candidates(parts, dom, 1.0)
    g = run_gpu(parts, dom, "fp64")
    np.testing.assert_array_equal(g["pi"], pi)
    np.testing.assert_array_equal(g["pj"], pj)
    assert len(pi) > 10
    compare(parts, dom, g, oracle_ref(parts, dom, pi, pj), "fp64", pi, pj)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_normal_only_model_parity(prec):
    """The "normal only" model (K~33 alone, Sec. IV C) against the oracle's."""
    parts, dom = gen.config_mixed_suspension(N=3000, phi=0.3, seed=14)
    g = run_gpu(parts, dom, prec, model=1)
    pi, pj = oracle.candidates(parts, dom, 1.0)
    compare(parts, dom, g, oracle_ref(parts, dom, pi, pj, model=1.0), prec, pi, pj)
    assert np.all(g["FT"][:, 3:] == 0)
    F = g["FT"][:, :3].astype(np.float64)
    assert np.abs(np.cross(F, g["n"])).max() <= 1e-5 * np.abs(F).max()


@pytest.mark.parametrize("P", [500, 3000])
def test_candidates_at_the_list_cutoff(P):
    """Sphere pairs at gaps within 1e-4 of Delta_L = 1.  For spheres the
    pre-filter values are h - Delta_L, so the FP32 tests leave every one of
    these inside their margin and the sweep leaves each to the FP64 test
    after it: 500 and 3,000 pairs (1,000 and 6,000 particles) give the
    oracle's set exactly."""
    parts, dom, _, _ = gen.pair_stream(P, seed=71, kind="spheres", gap_range=(1 - 1e-4, 1 + 1e-4))
    pi, pj = oracle.candidates(parts, dom, 1.0)
    assert P // 4 < len(pi) < 3 * P // 4             # both sides of the cut-off
    g = run_gpu(parts, dom, "fp64")
    np.testing.assert_array_equal(g["pi"], pi)
    np.testing.assert_array_equal(g["pj"], pj)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_candidates_on_the_filters_edge_beyond_the_buffer(prec):
    """A periodic simple cubic lattice of 1,000 spheres (radius 2) whose
    neighbours sit at gaps of Delta_L - 2e-5 along x and z and Delta_L + 2e-5
    along y: each of the 3,000 neighbour pairs lies inside the FP32 margin,
    more than the buffer of candidates left to the FP64 test holds (about one
    per particle), so the rest wait, tagged, at the tail of the pair arrays
    (the build asks for that room, then succeeds).  The list is the
    oracle's: the x and z neighbours, 2,000 pairs."""
    n, R = 10, 2.0
    a = np.array([2 * R + 1.0 - 2e-5, 2 * R + 1.0 + 2e-5, 2 * R + 1.0 - 2e-5])
    ii, jj, kk = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    pos = (np.stack([ii.ravel(), jj.ravel(), kk.ravel()], 1) + 0.5) * a
    N = len(pos)
    rng = np.random.default_rng(9)
    q = gen.random_quaternions(N, rng)
    r = np.full(N, R, np.float32)
    parts = dict(x=pos[:, 0].copy(), y=pos[:, 1].copy(), z=pos[:, 2].copy(), qw=q[:, 0].copy(), qx=q[:, 1].copy(),
                 qy=q[:, 2].copy(), qz=q[:, 3].copy(), r_par=r, r_perp=r.copy())
    gen.velocities(parts, rng)
    dom = dict(L=tuple(float(x) for x in n * a), periodic=(True, True, True), walls=[])
    pi, pj = oracle.candidates(parts, dom, 1.0)
    assert len(pi) == 2 * N
    g = run_gpu(parts, dom, prec)
    np.testing.assert_array_equal(g["pi"], pi)
    np.testing.assert_array_equal(g["pj"], pj)
    compare(parts, dom, g, oracle_ref(parts, dom, pi, pj), prec, pi, pj)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_candidates_exactly_on_the_list_cutoff(prec):
    """Sphere pairs (radius 2) whose centres lie exactly 2R + Delta_L = 5
    apart, and 2^-30 nearer or farther (positions exactly representable):
    the FP32 and float-float tests leave all of them inside their margins,
    so the FP64 test decides each, as the oracle does: the pair at 5 and the
    nearer ones are listed, the farther ones not."""
    offs = [0.0, 2.0 ** -30, -(2.0 ** -30), 0.0, 2.0 ** -30, -(2.0 ** -30)]
    xs, ys, zs = [], [], []
    for k, o in enumerate(offs):
        base = np.array([10.0 + 20.0 * (k % 3), 10.0 + 20.0 * (k // 3), 30.0])
        ax = k // 3  # along x for the first three, along y for the rest
        other = base.copy()
        other[ax] += 5.0 + o
        for pnt in (base, other):
            xs.append(pnt[0])
            ys.append(pnt[1])
            zs.append(pnt[2])
    n = len(xs)
    rng = np.random.default_rng(12)
    q = gen.random_quaternions(n, rng)
    r = np.full(n, 2.0, np.float32)
    parts = dict(x=np.array(xs), y=np.array(ys), z=np.array(zs), qw=q[:, 0].copy(), qx=q[:, 1].copy(),
                 qy=q[:, 2].copy(), qz=q[:, 3].copy(), r_par=r, r_perp=r.copy())
    gen.velocities(parts, rng)
    dom = dict(L=(100.0, 100.0, 100.0), periodic=(True, True, True), walls=[])
    pi, pj = oracle.candidates(parts, dom, 1.0)
    np.testing.assert_array_equal(pi, [0, 4, 6, 10])
    g = run_gpu(parts, dom, prec)
    np.testing.assert_array_equal(g["pi"], pi)
    np.testing.assert_array_equal(g["pj"], pj)


@pytest.mark.parametrize("case", ["periodic", "walls", "five_cells"])
def test_dense_packings(case):
    """Growth packings at Phi = 0.5 of spheroids with aspect ratios in
    [1/3, 3]: the longest set the cell range 2 Rmax + Delta_L (about 19.7), so
    a cell holds about 10 particles and every (particle, row) item of the
    sweep has some 30 candidates in its x window (the warp shares them out
    over its lanes).  The pair list must be the oracle's, with full parity;
    'five_cells' is a small periodic box (two cells per axis)."""
    rng = np.random.default_rng({"periodic": 21, "walls": 22, "five_cells": 23}[case])
    if case == "five_cells":
        sh = gen.aspect_shapes(400, rng)
        rmax = float(sh.max())
        side = 5.2 * (2 * rmax + 1.0) / 2          # floor(side / (range / 2)) = 5
        vol = float(np.sum(4.0 / 3.0 * np.pi * sh[:, 0].astype(np.float64) * sh[:, 1] ** 2))
        n = int(min(400, 0.5 * side ** 3 / (vol / 400)))
        sh = sh[:n]
        L, per, walls = (side, side, side), (True, True, True), []
    else:
        sh = gen.aspect_shapes(3000, rng)
        vol = float(np.sum(4.0 / 3.0 * np.pi * sh[:, 0].astype(np.float64) * sh[:, 1] ** 2))
        if case == "walls":
            a = (vol / 0.5 / 2.0) ** (1.0 / 3.0)
            L, per, walls = (a, a, 2 * a), (True, True, False), [(0.0, 1), (2 * a, -1)]
        else:
            a = (vol / 0.5) ** (1.0 / 3.0)
            L, per, walls = (a, a, a), (True, True, True), []
    parts, dom, _ = gen.grow(sh, L, periodic=per, walls=walls, seed=5)
    pi, pj = oracle.candidates(parts, dom, 1.0)
    assert len(pi) > 2 * len(sh)
    g = run_gpu(parts, dom, "mixed")
    np.testing.assert_array_equal(g["pi"], pi)
    np.testing.assert_array_equal(g["pj"], pj)
    compare(parts, dom, g, oracle_ref(parts, dom, pi, pj), "mixed", pi, pj)


@pytest.mark.parametrize("shift", [(0.0, 0.0, 0.0), (-0.3, 0.25, -0.1)])
def test_open_box_with_particles_outside_it(shift):
    """A box open on every axis (no periodic image, no wall): the sweep's x
    windows are clamped to the grid instead of wrapped.  Shifted by a
    fraction of the box, a quarter of the particles lie outside [0, L) on
    some axis and sit in the edge cells; every pair must still be listed
    exactly once (against the oracle's all-pairs search)."""
    rng = np.random.default_rng(31)
    sh = gen.aspect_shapes(1500, rng)
    L = 120.0
    parts, dom = gen.suspension(sh, (L, L, L), periodic=(False, False, False), attach_prob=0.8, seed=32)
    for k, f in zip(("x", "y", "z"), shift):
        parts[k] = parts[k] + f * L
    pi, pj = oracle.candidates(parts, dom, 1.0)
    assert len(pi) > len(sh)
    g = run_gpu(parts, dom, "mixed")
    np.testing.assert_array_equal(g["pi"], pi)
    np.testing.assert_array_equal(g["pj"], pj)
    compare(parts, dom, g, oracle_ref(parts, dom, pi, pj), "mixed", pi, pj)


def test_wall_pairs_at_the_list_cutoff():
    """Particles whose wall gap lies within 1e-4 of Delta_L = 1: the FP32 wall
    pre-filter leaves them inside its margin and the exact FP64 test decides;
    the wall pairs must be the oracle's."""
    rng = np.random.default_rng(91)
    n = 200
    L = 400.0
    r_par = rng.uniform(2.0, 8.0, n).astype(np.float32)
    r_perp = rng.uniform(2.0, 8.0, n).astype(np.float32)
    q = gen.random_quaternions(n, rng)
    # half-width along z of each spheroid, then z so that the gap to the wall
    # at z = 0 is 1 + u, |u| < 1e-4
    o_z = 1.0 - 2.0 * (q[:, 1].astype(np.float64) ** 2 + q[:, 2].astype(np.float64) ** 2)
    o_z /= (q.astype(np.float64) ** 2).sum(1)
    sz = np.sqrt(r_perp.astype(np.float64) ** 2 + (r_par.astype(np.float64) ** 2 - r_perp.astype(np.float64) ** 2) * o_z ** 2)
    u = rng.uniform(-1e-4, 1e-4, n)
    side = int(np.ceil(np.sqrt(n)))
    idx = np.arange(n)
    parts = dict(x=(idx % side + 0.5) * (L / side), y=(idx // side + 0.5) * (L / side), z=sz + 1.0 + u,
                 qw=q[:, 0].copy(), qx=q[:, 1].copy(), qy=q[:, 2].copy(), qz=q[:, 3].copy(), r_par=r_par,
                 r_perp=r_perp)
    gen.velocities(parts, rng)
    dom = dict(L=(L, L, L), periodic=(True, True, False), walls=[(0.0, 1)])
    pi, pj = oracle.candidates(parts, dom, 1.0)
    assert 0.25 * n < np.sum(pj < 0) < 0.75 * n          # both sides of the cut-off
    g = run_gpu(parts, dom, "fp64")
    np.testing.assert_array_equal(g["pi"], pi)
    np.testing.assert_array_equal(g["pj"], pj)


@pytest.mark.parametrize("offset", [0.0, 2000.0])
def test_mixed_precision_far_from_the_origin(offset):
    """The FP32 stage takes its separations from float-float positions (about
    48 bits, 2e-12 absolute at |r| = 2000): pairs placed near |r| = 2000 keep
    gap and force parity in mixed precision, including the gaps just above
    the FP64 switch that the float-float gap decides alone."""
    parts, dom, pi, pj = gen.pair_stream(2000, seed=93, kind="aspect", gap_range=(1e-3, 1.0), gap_scale="min_axis")
    parts = dict(parts)
    for k in ("x", "y", "z"):
        parts[k] = np.asarray(parts[k], np.float64) + offset
    dom = dict(dom, L=tuple(v + 2 * offset for v in dom["L"]))
    g = run_gpu(parts, dom, "mixed", pi, pj)
    compare(parts, dom, g, oracle_ref(parts, dom, pi, pj), "mixed", pi, pj)
