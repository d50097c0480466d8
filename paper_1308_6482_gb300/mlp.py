"""The learned warm start: training and installation of the network.

The network (12 -> 128 -> 128 -> 4, GELU) maps a pair's relative pose to the
surface parameters (p_i, q_i, p_j, q_j) of its closest points, as corrections
to those of the line-of-centres start; the library's closest-point call turns
them into Newton's start (LUB_WARM_MLP).  Features,
forward, backward and Adam run in the library's own kernels
(lub_mlp_features, lub_mlp_forward_backward, lub_mlp_adam); torch only holds
device buffers and draws the batch permutation.

Weights file (npz): params [LUB_MLP_PARAMS] float32 packed
[W1 | b1 | W2 | b2 | W3 | b3] (W row-major [out][in]), mean [12], istd [12].
"""
import os

import numpy as np

from . import _lib as L

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "mlp_weights.npz")
SHAPES = (("W1", (128, 12)), ("b1", (128,)), ("W2", (128, 128)), ("b2", (128,)), ("W3", (4, 128)), ("b3", (4,)))


def unpack(params):
    """Dict of the layer arrays from the packed parameter vector (numpy)."""
    out, o = {}, 0
    for k, sh in SHAPES:
        n = int(np.prod(sh))
        out[k] = np.asarray(params[o:o + n]).reshape(sh)
        o += n
    return out


def init_params(seed=0):
    """He-scaled normal weights, zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for k, sh in SHAPES:
        if k.startswith("W"):
            parts.append(rng.standard_normal(sh) * np.sqrt(2.0 / sh[1]))
        else:
            parts.append(np.zeros(sh))
    return np.concatenate([p.reshape(-1) for p in parts]).astype(np.float32)


class WarmStartMLP:
    def __init__(self, params=None, mean=None, istd=None, device="cuda", seed=0):
        import torch
        self.torch = torch
        self.device = device
        p = init_params(seed) if params is None else np.asarray(params, np.float32)
        assert p.size == L.LUB_MLP_PARAMS
        self.params = torch.as_tensor(p).to(device)
        self.mean = torch.as_tensor(np.zeros(12, np.float32) if mean is None else np.asarray(mean, np.float32)).to(device)
        self.istd = torch.as_tensor(np.ones(12, np.float32) if istd is None else np.asarray(istd, np.float32)).to(device)

    # ------------------------------------------------------------------
    @classmethod
    def load(cls, path=DEFAULT_WEIGHTS, device="cuda"):
        if not os.path.exists(path):
            raise FileNotFoundError("no trained network at %s (train one with train_mlp.py)" % path)
        d = np.load(path)
        return cls(d["params"], d["mean"], d["istd"], device=device)

    def save(self, path, **meta):
        np.savez(path, params=self.params.cpu().numpy(), mean=self.mean.cpu().numpy(), istd=self.istd.cpu().numpy(),
                 **meta)

    def install(self, ctx):
        """Give the context a BF16 copy for LUB_WARM_MLP."""
        L.lub_mlp_set(ctx.h if hasattr(ctx, "h") else ctx, self.params, self.mean, self.istd)

    # ------------------------------------------------------------------
    def features(self, ctx, particles, domain, pi, pj, standardise=True):
        """Features [n, 12] (torch, on the device) from the library's kernel."""
        torch = self.torch
        n = int(pi.numel())
        out = torch.empty((n, 12), dtype=torch.float32, device=self.device)
        L.lub_mlp_features(ctx.h, particles.c, domain, pi, pj, n, self.mean if standardise else None,
                           self.istd if standardise else None, out)
        return out

    def fit_standardisation(self, raw):
        m = raw.mean(0)
        s = raw.std(0)
        # constant features (e.g. a fixed shape) keep unit scale
        s = self.torch.where(s > 1e-6, s, self.torch.ones_like(s))
        self.mean = m.contiguous().float()
        self.istd = (1.0 / s).contiguous().float()

    def train(self, ctx, x, target, weight=None, epochs=30, batch=4096, lr=2e-3, seed=0, log=None):
        """Adam on standardised features x [n,12], targets and loss weights [n,4] (torch, device).

        Cosine learning-rate decay; returns the per-epoch mean losses."""
        torch = self.torch
        n = int(x.shape[0])
        nb = min(batch, n)
        steps_per_epoch = max(1, n // nb)
        grads = torch.zeros(L.LUB_MLP_PARAMS, dtype=torch.float32, device=self.device)
        m = torch.zeros_like(grads)
        v = torch.zeros_like(grads)
        work = torch.empty(nb * L.LUB_MLP_WORK_PER_SAMPLE, dtype=torch.float32, device=self.device)
        lrows = torch.empty(nb, dtype=torch.float32, device=self.device)
        g = torch.Generator(device=self.device)
        g.manual_seed(seed)
        total = epochs * steps_per_epoch
        t = 0
        hist = []
        for ep in range(epochs):
            perm = torch.randperm(n, generator=g, device=self.device)
            acc = torch.zeros((), dtype=torch.float64, device=self.device)
            for b in range(steps_per_epoch):
                idx = perm[b * nb:(b + 1) * nb]
                xb = x.index_select(0, idx).contiguous()
                tb = target.index_select(0, idx).contiguous()
                wb = None if weight is None else weight.index_select(0, idx).contiguous()
                L.lub_mlp_forward_backward(ctx.h, self.params, xb, tb, wb, nb, grads, work, lrows)
                t += 1
                lr_t = lr * 0.5 * (1.0 + np.cos(np.pi * (t - 1) / total))
                L.lub_mlp_adam(ctx.h, self.params, grads, m, v, L.LUB_MLP_PARAMS, t, lr_t)
                acc += lrows.double().mean()
            hist.append(float(acc.item()) / steps_per_epoch)
            if log:
                log("epoch %d loss %.5f" % (ep, hist[-1]))
        return hist
