"""The ensemble and large workloads' generators: periodic tiling keeps the
suspension's pair structure (each pair of the tiled box is a periodic-image
pair of the base, so the pair count grows exactly by k^3), members (growth
packings) hit their targets, and the large run is a tiled slab."""
import numpy as np

import gen
import oracle


def test_tiling_multiplies_the_pairs_by_k_cubed():
    rng = np.random.default_rng(2)
    sh = gen.aspect_shapes(150, rng)
    vol = float(np.sum(4.0 / 3.0 * np.pi * sh[:, 0].astype(np.float64) * sh[:, 1] ** 2))
    L = (vol / 0.2) ** (1.0 / 3.0)
    base, dom = gen.suspension(sh, (L, L, L), attach_prob=0.9, seed=3)
    pi, pj = oracle.candidates(base, dom, 1.0)
    for k in (2, 3):
        big, bdom = gen.tile_periodic(base, dom, k, rng)
        assert len(big["x"]) == k ** 3 * len(base["x"])
        assert bdom["L"] == tuple(k * v for v in dom["L"])
        qi, qj = oracle.candidates(big, bdom, 1.0)
        assert len(qi) == k ** 3 * len(pi)
        # every tiled pair maps to a base pair (indices modulo the base size)
        n = len(base["x"])
        a, b = np.minimum(qi % n, qj % n), np.maximum(qi % n, qj % n)
        base_set = set(zip(pi.tolist(), pj.tolist()))
        assert set(zip(a.tolist(), b.tolist())) <= base_set


def test_members_are_near_their_target_pair_counts():
    sus, meta = gen.ensemble(n_susp=6, seed=9, pairs_range=(1e3, 1e4), processes=1)
    for (parts, dom), phi, target in zip(sus, meta["phi"], meta["target_pairs"]):
        pi, _ = oracle.candidates(parts, dom, 1.0)
        assert 0.3 * target < len(pi) < 3.0 * target
        vol = float(np.sum(4.0 / 3.0 * np.pi * parts["r_par"].astype(np.float64) * parts["r_perp"] ** 2))
        assert abs(vol / np.prod(dom["L"]) - phi) < 1e-6


def test_large_config_tiles_the_slab_in_x_and_y_only():
    parts, dom = gen.large_config(N=2048, phi=0.3, seed=3, k=2, L=137.5)   # equivalent radius 4.5
    assert len(parts["x"]) == 2048
    assert dom["periodic"] == (True, True, False) and len(dom["walls"]) == 2
    L = dom["L"]
    assert L[0] == L[1] == L[2] and dom["walls"][1][0] == L[2]
    z = np.asarray(parts["z"])
    assert z.min() > 0 and z.max() < L[2]
    # a copy of the base slab: the pairs of the tiled box are 4 x those of the base
    rng = np.random.default_rng(3)
    base = {k: np.asarray(v)[:512] for k, v in parts.items()}
    bdom = dict(dom, L=(L[0] / 2, L[1] / 2, L[2]))
    pi, pj = oracle.candidates(base, bdom, 1.0)
    qi, qj = oracle.candidates(parts, dom, 1.0)
    assert len(qi) == 4 * len(pi) and np.sum(qj < 0) == 4 * np.sum(pj < 0) > 0
