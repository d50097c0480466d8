"""The learned warm start on the GPU, checked against the oracle's FP64 network.

* features: the library's kernel against the oracle's definition;
* training: FP32 forward/backward gradients against the oracle's FP64
  backward (itself pinned by finite differences), one Adam step against the
  update of Kingma & Ba written out;
* inference: tensor-core outputs (BF16 weights and activations) against the
  FP64 forward with the same BF16-rounded weights and activations;
* a network with zero outputs gives back the line-of-centres start exactly;
* the trained network (weights shipped with the package): Newton from its
  prediction needs fewer FP64 iterations than from the line of centres, the
  slowest lane of each warp too, and gives the same results (parity with the
  oracle).
"""
import os

import numpy as np
import pytest

import gen
import oracle
from parity import compare, oracle_ref, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import paper_1308_6482_gb300 as lub
    from paper_1308_6482_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    return lub, torch


def device_pairs(lub, torch, parts, dom, pi, pj):
    P = lub.DeviceParticles(parts)
    D = lub.make_domain(dom)
    return P, D, torch.as_tensor(pi).cuda(), torch.as_tensor(pj).cuda()


def test_features_match_oracle(env):
    lub, torch = env
    parts, dom, pi, pj = gen.pair_stream(3000, seed=71, kind="aspect", gap_range=(1e-4, 1.0), gap_scale="min_axis")
    ctx = lub.Context()
    P, D, tpi, tpj = device_pairs(lub, torch, parts, dom, pi, pj)
    out = torch.empty((len(pi), 12), dtype=torch.float32, device="cuda")
    lub.lub_mlp_features(ctx.h, P.c, D, tpi, tpj, len(pi), None, None, out)
    torch.cuda.synchronize()
    ref = oracle.mlp_features(parts, dom, pi, pj)
    got = out.cpu().numpy()
    reg = [c for c in range(12) if c != 9]
    np.testing.assert_allclose(got[:, reg], ref[:, reg], rtol=0, atol=2e-5 * np.abs(ref[:, reg]).max())
    # asinh(g/a): g is a difference of lengths ~10 in FP32
    np.testing.assert_allclose(got[:, 9], ref[:, 9], rtol=0, atol=2e-4)


def test_forward_backward_match_oracle(env):
    lub, torch = env
    from paper_1308_6482_gb300.mlp import init_params, unpack
    rng = np.random.default_rng(5)
    nb = 777  # several tiles plus a ragged tail
    x = rng.standard_normal((nb, 12)).astype(np.float32)
    t = rng.uniform(-3, 3, (nb, 4)).astype(np.float32)
    wt = rng.uniform(0, 1, (nb, 4)).astype(np.float32)
    params = init_params(seed=3)
    params[128 * 12:128 * 12 + 128] = rng.standard_normal(128) * 0.1  # non-zero biases
    ctx = lub.Context()
    dp = torch.as_tensor(params).cuda()
    grads = torch.zeros_like(dp)
    work = torch.empty(nb * lub._lib.LUB_MLP_WORK_PER_SAMPLE, device="cuda")
    lrows = torch.empty(nb, device="cuda")
    lub.lub_mlp_forward_backward(ctx.h, dp, torch.as_tensor(x).cuda(), torch.as_tensor(t).cuda(),
                                 torch.as_tensor(wt).cuda(), nb, grads, work, lrows)
    torch.cuda.synchronize()
    w = {k: v.astype(np.float64) for k, v in unpack(params).items()}
    loss, g, _ = oracle.mlp_loss_grad(x.astype(np.float64), t.astype(np.float64), w, wgt=wt.astype(np.float64))
    assert float(lrows.mean().item()) == pytest.approx(loss, rel=1e-5)
    gg = unpack(grads.cpu().numpy())
    for k in g:
        sc = np.abs(g[k]).max()
        assert np.abs(gg[k] - g[k]).max() <= 1e-4 * sc, k


def test_adam_step(env):
    lub, torch = env
    rng = np.random.default_rng(6)
    n = 1000
    p = rng.standard_normal(n).astype(np.float32)
    g = rng.standard_normal(n).astype(np.float32)
    m = rng.standard_normal(n).astype(np.float32) * 0.1
    v = rng.uniform(0, 1, n).astype(np.float32)
    ctx = lub.Context()
    dp, dg, dm, dv = [torch.as_tensor(a.copy()).cuda() for a in (p, g, m, v)]
    lr, b1, b2, eps, step = 1e-3, 0.9, 0.999, 1e-8, 7
    lub.lub_mlp_adam(ctx.h, dp, dg, dm, dv, n, step, lr, b1, b2, eps)
    torch.cuda.synchronize()
    m1 = b1 * m + (1 - b1) * g
    v1 = b2 * v + (1 - b2) * g * g
    p1 = p - lr * (m1 / (1 - b1 ** step)) / (np.sqrt(v1 / (1 - b2 ** step)) + eps)
    np.testing.assert_allclose(dp.cpu().numpy(), p1, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(dm.cpu().numpy(), m1, rtol=1e-6, atol=1e-7)


def bf16(a):
    """Round float32 values to bfloat16 (nearest even), returned as float64."""
    a = np.ascontiguousarray(a, np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("engine", ["mma_sync", "tcgen05"])
def test_tensor_core_inference_matches_bf16_reference(env, engine):
    lub, torch = env
    from paper_1308_6482_gb300.mlp import WarmStartMLP, init_params, unpack
    from scipy.special import erf
    parts, dom, pi, pj = gen.pair_stream(1000, seed=72, kind="aspect", gap_range=(1e-4, 1.0), gap_scale="min_axis")
    rng = np.random.default_rng(8)
    params = init_params(seed=9)
    params[-4:] = rng.standard_normal(4)
    raw = oracle.mlp_features(parts, dom, pi, pj)
    mean = raw.mean(0).astype(np.float32)
    istd = (1.0 / raw.std(0)).astype(np.float32)
    net = WarmStartMLP(params, mean, istd)
    ctx = lub.Context()
    net.install(ctx)
    lub.lub_mlp_engine(ctx.h, engine)
    P, D, tpi, tpj = device_pairs(lub, torch, parts, dom, pi, pj)
    m = len(pi)
    dc = torch.tensor([m], dtype=torch.int32, device="cuda")
    pq = torch.zeros(4 * m, dtype=torch.float32, device="cuda")
    lub.lub_mlp_predict(ctx.h, P.c, D, tpi, tpj, dc, m, pq)
    torch.cuda.synchronize()
    got = pq.cpu().numpy().reshape(4, m).T
    gelu = lambda z: 0.5 * z * (1 + erf(z / np.sqrt(2)))
    w = unpack(params)
    xs = bf16(((raw - mean) * istd).astype(np.float32))
    h1 = bf16(gelu(xs @ bf16(w["W1"]).T + w["b1"]).astype(np.float32))
    h2 = bf16(gelu(h1 @ bf16(w["W2"]).T + w["b2"]).astype(np.float32))
    y = h2 @ bf16(w["W3"]).T + w["b3"]
    err = np.abs(got - y)
    # BF16 activations: a few ulps (2^-8) of the layer scales; a layout error is O(1)
    assert err.max() <= 3e-2 * np.abs(y).max(), err.max()
    assert np.median(err) <= 3e-3 * np.abs(y).max()


def test_zero_network_gives_back_the_cold_start(env):
    """A network that outputs zero corrections must start Newton exactly on
    the line of centres: same iterations and results as the cold start."""
    lub, torch = env
    from paper_1308_6482_gb300.mlp import WarmStartMLP
    parts, dom, pi, pj = gen.pair_stream(2000, seed=73, kind="aspect", gap_range=(1e-4, 1.0), gap_scale="min_axis")
    net = WarmStartMLP(np.zeros(lub.LUB_MLP_PARAMS, np.float32))
    cold = run_gpu(parts, dom, "fp64", pi, pj)
    pl = lub.Pipeline(parts, dom, lub.default_params(precision="fp64", warm_start="mlp"))
    net.install(pl.ctx)
    pl.set_pairs(pi, pj)
    pl.closest()
    torch.cuda.synchronize()
    warm = pl.results()
    assert np.mean(warm["iters"] != cold["iters"]) < 0.01
    np.testing.assert_allclose(warm["h"], cold["h"], rtol=0, atol=1e-10)


def test_tcgen05_engine_gives_the_same_start(env):
    """The two tensor-core paths: the same outputs up to the order of the FP32
    accumulation (BF16 activations can round differently), the same Newton
    results."""
    lub, torch = env
    from paper_1308_6482_gb300.mlp import WarmStartMLP
    parts, dom, pi, pj = gen.pair_stream(3000, seed=74, kind="aspect", gap_range=(1e-4, 1.0), gap_scale="min_axis")
    net = WarmStartMLP.load(WEIGHTS)
    out = {}
    for engine in ("mma_sync", "tcgen05"):
        pl = lub.Pipeline(parts, dom, lub.default_params(precision="fp64", warm_start="mlp"))
        net.install(pl.ctx)
        lub.lub_mlp_engine(pl.ctx.h, engine)
        pl.set_pairs(pi, pj)
        pq = torch.zeros(4 * pl.cap, dtype=torch.float32, device="cuda")
        lub.lub_mlp_predict(pl.ctx.h, pl.P.c, pl.D, pl.pair_i, pl.pair_j, pl.d_count, pl.cap, pq)
        pl.closest()
        torch.cuda.synchronize()
        out[engine] = (pq.cpu().numpy().reshape(4, -1)[:, :len(pi)].T, pl.results())
    (ya, ra), (yb, rb) = out["mma_sync"], out["tcgen05"]
    err = np.abs(ya - yb)
    assert np.median(err) <= 2e-3 * np.abs(ya).max() and err.max() <= 3e-2 * np.abs(ya).max()
    np.testing.assert_array_equal(ra["status"] & 7, rb["status"] & 7)
    np.testing.assert_allclose(ra["h"], rb["h"], rtol=0, atol=1e-10)
    assert abs(ra["iters"].mean() - rb["iters"].mean()) < 0.05


WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1308_6482_gb300",
                       "mlp_weights.npz")


def test_trained_network_saves_fp64_newton_iterations(env):
    """Fresh pairs (a seed the training set never used): the FP64 solve from
    the network's start takes fewer iterations and keeps FP64 parity."""
    lub, torch = env
    assert os.path.exists(WEIGHTS), "the trained network is part of the package"
    from paper_1308_6482_gb300.mlp import WarmStartMLP
    parts, dom, pi, pj = gen.pair_stream(20000, seed=9001, kind="aspect", gap_range=(1e-4, 1.0),
                                         gap_scale="min_axis")
    cold = run_gpu(parts, dom, "fp64", pi, pj)
    net = WarmStartMLP.load(WEIGHTS)
    pl = lub.Pipeline(parts, dom, lub.default_params(precision="fp64", warm_start="mlp"))
    net.install(pl.ctx)
    pl.set_pairs(pi, pj)
    pl.closest()
    pl.resistance()
    pl.apply()
    torch.cuda.synchronize()
    warm = pl.results()
    it_c, it_w = cold["iters"].mean(), warm["iters"].mean()
    # measured on GB300: 4.81 -> 3.71 per pair, 6.4 -> 4.4 for the slowest lane of a warp
    assert it_w < 0.85 * it_c, (it_c, it_w)
    wmax = lambda it: it[:len(it) // 32 * 32].reshape(-1, 32).max(1).mean()
    assert wmax(warm["iters"]) < 0.8 * wmax(cold["iters"])
    ref = oracle_ref(parts, dom, pi, pj)
    compare(parts, dom, warm, ref, "fp64", pi, pj)
