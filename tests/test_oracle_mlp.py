"""Pins of the oracle's network (the learned warm start's reference).

The backward pass is checked against central finite differences of the
forward pass in FP64; the features against rigid-motion invariance and
their definitions' special cases; the (p, q) labels against the surface
parametrisation of Eq. lub:spheroid.
"""
import numpy as np
import pytest

import gen
import oracle
from helpers import axis_angle_quat, quat_to_mat, rigid_transform, spheroid_point


def random_weights(rng, scale=0.3):
    return {k: scale * rng.standard_normal(sh) for k, sh in oracle.MLP_SHAPES.items()}


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    w = random_weights(rng)
    x = rng.standard_normal((7, 12))
    t = rng.uniform(-3, 3, (7, 4))
    loss, g, _ = oracle.mlp_loss_grad(x, t, w)
    eps = 1e-6
    for k in oracle.MLP_SHAPES:
        flat = w[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(12, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp, _, _ = oracle.mlp_loss_grad(x, t, w, want_grad=False)
            flat[idx] = old - eps
            lm, _, _ = oracle.mlp_loss_grad(x, t, w, want_grad=False)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            an = g[k].reshape(-1)[idx]
            assert an == pytest.approx(fd, rel=1e-6, abs=1e-9), (k, idx)


def test_weighted_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    w = random_weights(rng)
    x = rng.standard_normal((5, 12))
    t = rng.uniform(-3, 3, (5, 4))
    wt = rng.uniform(0, 1, (5, 4))
    loss, g, _ = oracle.mlp_loss_grad(x, t, w, wgt=wt)
    eps = 1e-6
    for k in ("W3", "b1"):
        flat = w[k].reshape(-1)
        for idx in rng.choice(flat.size, size=6, replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp, _, _ = oracle.mlp_loss_grad(x, t, w, want_grad=False, wgt=wt)
            flat[idx] = old - eps
            lm, _, _ = oracle.mlp_loss_grad(x, t, w, want_grad=False, wgt=wt)
            flat[idx] = old
            assert g[k].reshape(-1)[idx] == pytest.approx((lp - lm) / (2 * eps), rel=1e-6, abs=1e-9)


def test_baseline_normals_are_the_line_of_centres():
    """At the line-of-centres start the outward normals are +d^ on i and -d^ on j."""
    parts, dom, pi, pj = gen.pair_stream(20, seed=63, kind="aspect", gap_range=(1e-3, 0.5))
    base = oracle.mlp_baseline(parts, dom, pi, pj)
    for k in range(len(pi)):
        i, j = pi[k], pj[k]
        d = np.array([float(parts[c][j]) - float(parts[c][i]) for c in ("x", "y", "z")])
        d /= np.linalg.norm(d)
        for idx, (p, q), e in ((i, base[k, :2], d), (j, base[k, 2:], -d)):
            qq = [float(parts[f][idx]) for f in ("qw", "qx", "qy", "qz")]
            from helpers import spheroid_normal
            n = spheroid_normal(qq, float(parts["r_par"][idx]), float(parts["r_perp"][idx]), p, q)
            np.testing.assert_allclose(n, e, atol=1e-10)


def test_loss_wraps_the_azimuth():
    rng = np.random.default_rng(1)
    w = random_weights(rng)
    x = rng.standard_normal((5, 12))
    _, _, y = oracle.mlp_loss_grad(x, np.zeros((5, 4)), w, want_grad=False)
    t = y.copy()
    t[:, 1] += 2 * np.pi
    t[:, 3] -= 4 * np.pi
    loss, _, _ = oracle.mlp_loss_grad(x, t, w, want_grad=False)
    assert loss == pytest.approx(0.0, abs=1e-20)


def test_features_are_invariant_under_rigid_motion():
    parts, dom, pi, pj = gen.pair_stream(40, seed=61, kind="aspect", gap_range=(1e-4, 0.5))
    parts = {k: np.asarray(v, np.float64) for k, v in parts.items()}
    dom = dict(L=(1e5,) * 3, periodic=(False,) * 3, walls=[])
    f0 = oracle.mlp_features(parts, dom, pi, pj)
    qR = axis_angle_quat([0.2, 0.9, -0.4], 2.3)
    moved = rigid_transform(parts, quat_to_mat(qR), np.array([5.0, -7.0, 11.0]), qR)
    f1 = oracle.mlp_features(moved, dom, pi, pj)
    np.testing.assert_allclose(f1, f0, rtol=0, atol=1e-9)


def test_features_are_invariant_under_rotations_about_each_axis():
    """Turning i about its own symmetry axis or j about its own changes neither
    the pair's geometry nor the targets: the features must not change."""
    parts, dom, pi, pj = gen.pair_stream(40, seed=64, kind="aspect", gap_range=(1e-4, 0.5))
    parts = {k: np.asarray(v, np.float64) for k, v in parts.items()}
    f0 = oracle.mlp_features(parts, dom, pi, pj)
    from helpers import quat_mul
    for side in (pi, pj):
        moved = {k: v.copy() for k, v in parts.items()}
        for t, k in enumerate(side):
            q = [moved[c][k] for c in ("qw", "qx", "qy", "qz")]
            spin = axis_angle_quat([0, 0, 1], 0.3 + 0.7 * t)    # about the body z (symmetry) axis
            nq = quat_mul(q, spin)
            for c, v in zip(("qw", "qx", "qy", "qz"), nq):
                moved[c][k] = v
        f1 = oracle.mlp_features(moved, dom, pi, pj)
        np.testing.assert_allclose(f1, f0, rtol=0, atol=1e-9)


def test_feature_definitions_special_cases():
    # identity orientations: body frame = lab frame; d = (6, 8, 1) lies at
    # azimuth atan2(8, 6) about i's axis, so the turned frame maps j's axis
    # (0, 0, 1) to itself and the distance from the axis is 10
    from helpers import make_parts
    parts = make_parts([[0, 0, 0], [6.0, 8.0, 1.0]], [[1, 0, 0, 0]] * 2, [6.0, 3.0], [3.0, 6.0])
    dom = dict(L=(1e3,) * 3, periodic=(False,) * 3, walls=[])
    f = oracle.mlp_features(parts, dom, np.array([0], np.int32), np.array([1], np.int32))[0]
    np.testing.assert_allclose(f[:2], [10.0 / 3.0, 1.0 / 3.0])
    np.testing.assert_allclose(f[2:5], [0, 0, 1], atol=1e-15)
    np.testing.assert_allclose(f[5:9], np.log([6.0, 3.0, 3.0, 6.0]))
    d = np.array([6.0, 8.0, 1.0])
    e = d / np.linalg.norm(d)
    si = np.sqrt(3.0 ** 2 * (e[0] ** 2 + e[1] ** 2) + 6.0 ** 2 * e[2] ** 2)
    sj = np.sqrt(6.0 ** 2 * (e[0] ** 2 + e[1] ** 2) + 3.0 ** 2 * e[2] ** 2)
    assert f[9] == pytest.approx(np.arcsinh((np.linalg.norm(d) - si - sj) / 3.0), rel=1e-12)
    np.testing.assert_allclose(f[10:], np.log([si / 3.0, sj / 6.0]), rtol=1e-13)
    # j's axis tilted in the plane of d and i's axis: its turned components are
    # (cos, 0, sin) of the tilt measured from the d direction
    t = 0.4
    q_tilt = axis_angle_quat([-0.8, 0.6, 0], t)                  # towards d, about the horizontal normal of d
    parts = make_parts([[0, 0, 0], [6.0, 8.0, 1.0]], [[1, 0, 0, 0], q_tilt], [6.0, 3.0], [3.0, 6.0])
    f = oracle.mlp_features(parts, dom, np.array([0], np.int32), np.array([1], np.int32))[0]
    np.testing.assert_allclose(f[2:5], [np.sin(t), 0.0, np.cos(t)], atol=1e-12)


def test_pq_labels_reproduce_the_closest_points():
    parts, dom, pi, pj = gen.pair_stream(30, seed=62, kind="aspect", gap_range=(1e-4, 0.8))
    cp = oracle.closest(parts, dom, pi, pj)
    lab = oracle.pq_labels(parts, dom, pi, pj, cp)
    for k in range(len(pi)):
        for idx, (p, q), y in ((pi[k], lab[k, :2], cp["yi"][k]), (pj[k], lab[k, 2:], cp["yj"][k])):
            qq = [float(parts[f][idx]) for f in ("qw", "qx", "qy", "qz")]
            r = [parts["x"][idx], parts["y"][idx], parts["z"][idx]]
            yy = spheroid_point(qq, parts["r_par"][idx], parts["r_perp"][idx], r, p, q)
            np.testing.assert_allclose(yy, y, atol=1e-9)
