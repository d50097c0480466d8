"""Runtime support entry points (no counterpart in the paper): the kernel
trace, the pipe probes and the seeded random rigid motions.

* lub_random_motion against a numpy restatement of Philox4x32-10 (Salmon et
  al., SC 2011) and the Box-Muller transform: the same draws, the same
  displacements and rotations; repeatable per (seed, step); sample moments;
* lub_trace_enable / lub_trace_read: one interval per traced kernel of an
  eager step, none while the stream is captured, none once disabled;
* lub_probe_peak: FP32 and FP64 FMA throughput within broad physical bounds.
"""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu

M32 = np.uint64(0xFFFFFFFF)


@pytest.fixture(scope="module")
def env():
    import torch

    import paper_1308_6482_gb300 as lub
    from paper_1308_6482_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    return lub, torch


def philox4x32_10(c, key):
    """c: 4 uint64 arrays holding 32-bit words; key: (k0, k1)."""
    c0, c1, c2, c3 = (np.asarray(v, np.uint64) & M32 for v in c)
    k0, k1 = np.uint64(key[0]), np.uint64(key[1])
    for r in range(10):
        if r:
            k0 = (k0 + np.uint64(0x9E3779B9)) & M32
            k1 = (k1 + np.uint64(0xBB67AE85)) & M32
        p0 = np.uint64(0xD2511F53) * c0
        p1 = np.uint64(0xCD9E8D57) * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & M32
        hi1, lo1 = p1 >> np.uint64(32), p1 & M32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def box_muller(a, b):
    u1 = ((a >> np.uint64(8)) + np.uint64(1)).astype(np.float64) * 2.0 ** -24
    u2 = (b >> np.uint64(8)).astype(np.float64) * 2.0 ** -24
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)


def expected_motion(parts, seed, step, sr, st):
    n = len(parts["x"])
    k = np.arange(n, dtype=np.uint64)
    s = np.uint64(step)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    r0 = philox4x32_10((k, s & M32, s >> np.uint64(32), np.zeros(n, np.uint64)), key)
    r1 = philox4x32_10((k, s & M32, s >> np.uint64(32), np.ones(n, np.uint64)), key)
    g0 = box_muller(r0[0], r0[1])
    g1 = box_muller(r0[2], r0[3])
    g2 = box_muller(r1[0], r1[1])
    out = {c: np.asarray(parts[c], np.float64).copy() for c in ("x", "y", "z")}
    out["x"] += sr * g0[0]
    out["y"] += sr * g0[1]
    out["z"] += sr * g1[0]
    th = st * np.stack([g1[1], g2[0], g2[1]], 1)
    a = np.linalg.norm(th, axis=1)
    sc = np.where(a > 0, np.sin(0.5 * a) / np.where(a > 0, a, 1), 0.5)
    dq = np.concatenate([np.cos(0.5 * a)[:, None], sc[:, None] * th], 1)
    q = np.stack([parts[c] for c in ("qw", "qx", "qy", "qz")], 1).astype(np.float64)
    dw, dx, dy, dz = dq.T
    w, x, y, z = q.T
    nq = np.stack([dw * w - dx * x - dy * y - dz * z, dw * x + dx * w + dy * z - dz * y,
                   dw * y - dx * z + dy * w + dz * x, dw * z + dx * y - dy * x + dz * w], 1)
    nq /= np.linalg.norm(nq, axis=1, keepdims=True)
    for i, c in enumerate(("qw", "qx", "qy", "qz")):
        out[c] = nq[:, i]
    return out


def moved(lub, torch, parts, seed, step, sr, st):
    P = lub.DeviceParticles(parts)
    ctx = lub.Context()
    lub.lub_random_motion(ctx.h, P.c, seed, step, sr, st)
    torch.cuda.synchronize()
    return {c: P.t[c].cpu().numpy().astype(np.float64) for c in ("x", "y", "z", "qw", "qx", "qy", "qz")}


def test_random_motion_matches_its_definition(env):
    lub, torch = env
    parts, _ = gen.config_mixed_suspension(N=20000, phi=0.3, seed=3)
    seed, step, sr, st = 0x1234567890ABCDEF, 7, 0.01, 0.005
    got = moved(lub, torch, parts, seed, step, sr, st)
    ref = expected_motion(parts, seed, step, sr, st)
    for c in ("x", "y", "z"):
        # float draws added to the double positions: |error| ~ 1e-6 of sigma_r
        np.testing.assert_allclose(got[c], ref[c], rtol=0, atol=2e-6 * sr * 6)
    for c in ("qw", "qx", "qy", "qz"):
        np.testing.assert_allclose(got[c], ref[c], rtol=0, atol=2e-6)
    again = moved(lub, torch, parts, seed, step, sr, st)
    for c in got:
        np.testing.assert_array_equal(got[c], again[c])
    other = moved(lub, torch, parts, seed, step + 1, sr, st)
    assert np.mean(other["x"] != got["x"]) > 0.99


def test_random_motion_moments(env):
    lub, torch = env
    n = 1 << 20
    zf = np.zeros(n, np.float32)
    parts = dict(x=np.zeros(n), y=np.zeros(n), z=np.zeros(n), qw=np.ones(n, np.float32), qx=zf, qy=zf, qz=zf,
                 r_par=np.full(n, 4.0, np.float32), r_perp=np.full(n, 2.0, np.float32))
    got = moved(lub, torch, parts, 99, 3, 0.01, 0.005)
    d = np.stack([got["x"], got["y"], got["z"]], 1)
    assert np.all(np.abs(d.mean(0)) < 5 * 0.01 / np.sqrt(n))
    assert np.all(np.abs(d.std(0) / 0.01 - 1) < 0.01)
    # rotation angle from the identity: theta = 2 acos(qw), E[theta^2] = 3 sigma_t^2
    th = 2 * np.arccos(np.clip(got["qw"], -1, 1))
    assert abs(np.mean(th ** 2) / (3 * 0.005 ** 2) - 1) < 0.02
    q = np.stack([got[c] for c in ("qw", "qx", "qy", "qz")], 1)
    assert np.abs(np.linalg.norm(q, axis=1) - 1).max() < 1e-6


def test_trace_records_each_traced_kernel(env):
    lub, torch = env
    parts, dom = gen.config_mixed_suspension(N=4000, phi=0.3, seed=9)
    pl = lub.Pipeline(parts, dom, lub.default_params())
    pl.build_pairs()
    lub.lub_trace_enable(pl.ctx.h, 1)
    pl.build_pairs(sync_count=False, grow=False)
    pl.closest()
    pl.resistance_apply()
    torch.cuda.synchronize()
    for k in (lub.LUB_TRACE_SWEEP, lub.LUB_TRACE_CLOSEST, lub.LUB_TRACE_RESISTANCE):
        ms, n = lub.lub_trace_read(pl.ctx.h, k)
        assert n == 1 and 0.0 < ms < 100.0, (k, ms, n)
        assert lub.lub_trace_read(pl.ctx.h, k) == (0.0, 0)   # a read forgets the intervals
    assert lub.lub_trace_read(pl.ctx.h, lub.LUB_TRACE_APPLY) == (0.0, 0)
    # nothing is recorded while the stream is captured
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        pl.closest(stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert lub.lub_trace_read(pl.ctx.h, lub.LUB_TRACE_CLOSEST) == (0.0, 0)
    lub.lub_trace_enable(pl.ctx.h, 0)
    pl.closest()
    torch.cuda.synchronize()
    assert lub.lub_trace_read(pl.ctx.h, lub.LUB_TRACE_CLOSEST) == (0.0, 0)


def test_pipe_probes(env):
    lub, torch = env
    ctx = lub.Context()
    f32 = lub.lub_probe_peak(ctx.h, lub.LUB_PROBE_FP32)
    f64 = lub.lub_probe_peak(ctx.h, lub.LUB_PROBE_FP64)
    # 152 SMs x 128 FP32 lanes x 2 FLOP at 1-2.1 GHz; FP64 far below
    assert 20.0 < f32 < 100.0 and 0.2 < f64 < 10.0 and f32 > 20 * f64, (f32, f64)


def test_random_motion_device_counters(env):
    """Two calls alternating two device counters move like host steps s, s + 1
    and leave s + 2 behind: what a graph of several motions replays."""
    lub, torch = env
    parts, _ = gen.config_mixed_suspension(N=5000, phi=0.3, seed=4)
    P = lub.DeviceParticles(parts)
    ctx = lub.Context()
    c = torch.tensor([40, -1], dtype=torch.int64, device="cuda")
    lub.lub_random_motion(ctx.h, P.c, 5, 0, 0.01, 0.005, step_dev=c[0:], next_dev=c[1:])
    lub.lub_random_motion(ctx.h, P.c, 5, 0, 0.01, 0.005, step_dev=c[1:], next_dev=c[0:])
    torch.cuda.synchronize()
    assert c.tolist() == [42, 41]
    Q = lub.DeviceParticles(parts)
    lub.lub_random_motion(ctx.h, Q.c, 5, 40, 0.01, 0.005)
    lub.lub_random_motion(ctx.h, Q.c, 5, 41, 0.01, 0.005)
    torch.cuda.synchronize()
    for k in ("x", "y", "z", "qw", "qx", "qy", "qz"):
        assert torch.equal(P.t[k], Q.t[k]), k
