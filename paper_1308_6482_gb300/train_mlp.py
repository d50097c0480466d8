"""Train the learned warm start on a data set written by the oracle's data
writer (raw pair geometry + closest-point surface parameters), with the
library's own feature, forward/backward and Adam kernels on the GPU.

    python -m paper_1308_6482_gb300.train_mlp --data train.npz --out mlp_weights.npz
"""
import argparse
import json
import time

import numpy as np


def load_pairs(path, device):
    import torch

    from . import DeviceParticles, make_domain
    d = np.load(path)
    parts = {k: d[k] for k in ("x", "y", "z", "qw", "qx", "qy", "qz", "r_par", "r_perp")}
    n = len(parts["x"])
    for k in ("vx", "vy", "vz", "wx", "wy", "wz"):
        parts[k] = np.zeros(n, np.float32)
    P = DeviceParticles(parts, device)
    dom = make_domain(dict(L=tuple(d["L"]), periodic=(False, False, False), walls=[]))
    pi = torch.as_tensor(d["pi"]).to(device)
    pj = torch.as_tensor(d["pj"]).to(device)
    tgt = torch.as_tensor(d["targets"].astype(np.float32)).to(device)
    wgt = torch.as_tensor(d["weights"].astype(np.float32)).to(device)
    return P, dom, pi, pj, tgt, wgt


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--data", required=True)
    ap.add_argument("--out", required=True)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--lr", type=float, default=5e-3)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args()
    import torch

    from . import Context
    from .mlp import WarmStartMLP
    dev = "cuda"
    ctx = Context()
    P, dom, pi, pj, tgt, wgt = load_pairs(a.data, dev)
    net = WarmStartMLP(seed=a.seed, device=dev)
    raw = net.features(ctx, P, dom, pi, pj, standardise=False)
    net.fit_standardisation(raw)
    x = net.features(ctx, P, dom, pi, pj, standardise=True)
    t0 = time.time()
    hist = net.train(ctx, x, tgt, wgt, epochs=a.epochs, batch=a.batch, lr=a.lr, seed=a.seed, log=print)
    torch.cuda.synchronize()
    meta = dict(data=a.data, pairs=int(pi.numel()), epochs=a.epochs, batch=a.batch, lr=a.lr, seed=a.seed,
                train_seconds=time.time() - t0, loss=hist)
    net.save(a.out, meta=json.dumps(meta))
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
