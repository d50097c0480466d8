"""Write a training or test set of the learned warm start.

TEST INFRASTRUCTURE (part of the oracle).  Seeded pair stream of spheroid
pairs (aspect ratio log-uniform in [1/3, 3], equivalent radius 4.5, gap
log-uniform in [1e-4, 1] times the smaller semi-axis), solved by the FP64
oracle; the labels are the surface parameters (p_i, q_i, p_j, q_j) of
Eq. lub:spheroid at the closest points, the targets their corrections to
those of the line-of-centres start (azimuths wrapped), the weights
(1, cos^2 p_i, 1, cos^2 p_j) of the loss.  The file holds the raw pair
geometry (so the features are computed by the same code that uses them) and
the labels; nothing from the CUDA library.

    python oracle/make_mlp_data.py --pairs 2000000 --seed 301 --out train.npz
"""
import argparse
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import gen  # noqa: E402
import oracle  # noqa: E402


def make(pairs, seed):
    parts, dom, pi, pj = gen.pair_stream(pairs, seed=seed, kind="aspect", gap_range=(1e-4, 1.0),
                                         gap_scale="min_axis")
    P = oracle.Particles(parts)
    cp = oracle.closest(P, dom, pi, pj)
    ok = cp["status"] == 0
    lab = oracle.pq_labels(P, dom, pi, pj, cp)
    base = oracle.mlp_baseline(P, dom, pi, pj)
    tgt, wgt = oracle.mlp_targets(lab, base)
    return parts, dom, pi[ok], pj[ok], lab[ok], tgt[ok], wgt[ok], cp["h"][ok]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=2000000)
    ap.add_argument("--seed", type=int, default=301)
    ap.add_argument("--out", required=True)
    a = ap.parse_args()
    t0 = time.time()
    parts, dom, pi, pj, lab, tgt, wgt, h = make(a.pairs, a.seed)
    keep = ("x", "y", "z", "qw", "qx", "qy", "qz", "r_par", "r_perp")
    np.savez(a.out, **{k: parts[k] for k in keep}, L=np.asarray(dom["L"]), pi=pi, pj=pj, labels=lab, targets=tgt,
             weights=wgt, h=h)
    print("wrote %s: %d pairs in %.1f s" % (a.out, len(pi), time.time() - t0))


if __name__ == "__main__":
    main()
