"""Pins of the oracle's link-based lubrication (Ding and Aidun, Eq.
methods:dlub of Sec. II), the comparison model of the scope's last row:

* two configurations with exactly one qualifying link, worked by hand from
  the printed formula: a direct link between a site of j and one of i, and a
  pair of links through a fluid site;
* the exchange (i, j) -> (j, i) flips the force and swaps the torques (each
  link enters both orders with the same h*, lambda* and velocities);
* moving both particles by a lattice vector changes nothing (the links move
  with them), nor does a common velocity (only differences enter);
* the partial forces act along their links, so the pair's total torque
  about the origin vanishes;
* pairs beyond the links' reach give nothing.
"""
import numpy as np

import gen
import oracle

MU, QBAR = 1.0 / 6.0, 0.6
FREE = dict(L=(60.0, 60.0, 60.0), periodic=(False, False, False), walls=[])


def two_spheres(xj, r, vi=(0, 0, 0), vj=(0, 0, 0)):
    p = {k: np.zeros(2) for k in ("x", "y", "z", "qx", "qy", "qz", "vx", "vy", "vz", "wx", "wy", "wz")}
    p["qw"] = np.ones(2)
    p["x"][1] = xj
    p["r_par"] = np.full(2, r)
    p["r_perp"] = np.full(2, r)
    for d, k in enumerate(("vx", "vy", "vz")):
        p[k][0], p[k][1] = vi[d], vj[d]
    return p


def dlub(cr, lam, h, e, dv):
    """Eq. methods:dlub for one link: -3 qbar mu / (2 c_r^2 lambda*) c^ (c^.dv) (1/h*^2 - 1/c_r^2)."""
    e = np.asarray(e, float)
    return -3 * QBAR * MU / (2 * cr * cr * lam) * e * (e @ np.asarray(dv, float)) * (1 / h ** 2 - 1 / cr ** 2)


def test_one_direct_link():
    # spheres of radius 0.6 at x = 0 and 1.3: i holds the site (0,0,0), j the
    # site (1,0,0); the one link from (1,0,0) to (0,0,0) leaves j at x = 0.7 and
    # enters i at x = 0.6, h* = 0.1 < 1; lambda* = 1 / 0.6
    p = two_spheres(1.3, 0.6, vj=(-0.01, 0.002, 0.0))
    r = oracle.links(p, FREE, [0], [1], MU, QBAR)
    assert r["links"][0] == 1
    want = dlub(1.0, 1 / 0.6, 0.1, (-1, 0, 0), np.array([0, 0, 0]) - np.array([-0.01, 0.002, 0]))
    np.testing.assert_allclose(r["F"][0], want, rtol=1e-12, atol=1e-15)
    assert r["F"][0, 0] < 0            # j approaches: i is pushed away from j
    np.testing.assert_allclose(r["T"][0], 0.0, atol=1e-15)   # along the line of centres


def test_one_link_pair_through_a_fluid_site():
    # radius 0.9 at x = 0 and 2.05: sites (0,0,0) of i and (2,0,0) of j, the
    # site (1,0,0) between them is fluid; h* = (2.05 - 0.9) - 0.9 = 0.25 < c_r = 1
    p = two_spheres(2.05, 0.9, vi=(0.003, 0.0, -0.001))
    r = oracle.links(p, FREE, [0], [1], MU, QBAR)
    assert r["links"][0] == 1
    want = dlub(1.0, 1 / 0.9, 0.25, (-1, 0, 0), (0.003, 0.0, -0.001))
    np.testing.assert_allclose(r["F"][0], want, rtol=1e-12, atol=1e-15)


def near_pairs(seed, P=40):
    parts, dom, pi, pj = gen.pair_stream(P, seed=seed, kind="aspect", gap_range=(0.05, 1.5))
    rng = np.random.default_rng(seed)
    for k in ("wx", "wy", "wz"):
        parts[k] = rng.normal(0, 1e-3, len(parts["x"]))
    return parts, dom, pi, pj


def test_exchange_flips_the_force_and_swaps_the_torques():
    parts, dom, pi, pj = near_pairs(5)
    a = oracle.links(parts, dom, pi, pj, MU, QBAR)
    b = oracle.links(parts, dom, pj, pi, MU, QBAR)
    assert a["links"].sum() > 10 * len(pi)
    np.testing.assert_array_equal(a["links"], b["links"])
    sc = np.abs(a["F"]).max()
    np.testing.assert_allclose(a["F"], -b["F"], rtol=0, atol=1e-12 * sc)
    st = np.abs(a["T"]).max()
    np.testing.assert_allclose(a["T"][:, :3], b["T"][:, 3:], rtol=0, atol=1e-12 * st)


def test_lattice_shift_and_common_velocity_change_nothing():
    parts, dom, pi, pj = near_pairs(6)
    a = oracle.links(parts, dom, pi, pj, MU, QBAR)
    parts = {k: np.asarray(v, np.float64) for k, v in parts.items()}   # the shifts exact
    a = oracle.links(parts, dom, pi, pj, MU, QBAR)
    moved = dict(parts)
    for k, s in (("x", 3.0), ("y", -2.0), ("z", 5.0)):
        moved[k] = parts[k] + s
    for k, s in (("vx", 0.01), ("vy", -0.02), ("vz", 0.005)):
        moved[k] = parts[k] + s
    b = oracle.links(moved, dom, pi, pj, MU, QBAR)
    np.testing.assert_array_equal(a["links"], b["links"])
    np.testing.assert_allclose(b["F"], a["F"], rtol=0, atol=1e-11 * np.abs(a["F"]).max())


def test_total_torque_about_the_origin_vanishes():
    parts, dom, pi, pj = near_pairs(7)
    r = oracle.links(parts, dom, pi, pj, MU, QBAR)
    pos = np.stack([parts["x"], parts["y"], parts["z"]], 1)
    total = np.cross(pos[pi], r["F"]) + r["T"][:, :3] + np.cross(pos[pj], -r["F"]) + r["T"][:, 3:]
    scale = np.abs(np.cross(pos[pi], r["F"])).max()
    assert np.abs(total).max() <= 1e-10 * scale


def test_far_pairs_have_no_links():
    p = two_spheres(12.0, 4.0)
    r = oracle.links(p, FREE, [0], [1], MU, QBAR)
    assert r["links"][0] == 0 and not np.any(r["F"])
