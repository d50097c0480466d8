"""Pins of the oracle's particle sub-step (Sec. II: explicit particle updates
at a fraction of the LB time step), against closed forms of rigid-body
motion:

* a free particle under a constant force follows the semi-implicit Euler
  recurrences exactly: v_n = v_0 + n dt F/m, x_n = x_0 + dt sum_k v_k;
* a sphere spun up by a constant torque along its angular velocity turns by
  dt sum_k |w_k| about that axis;
* a torque-free symmetric top keeps its angular momentum L exactly, and its
  symmetry axis precesses about L at the rate |L| / I_perp (w = L / I_perp +
  c o, so do/dt = (L / I_perp) x o), converging at first order in dt.
"""
import numpy as np
import pytest

import oracle


def body(n, rpar, rperp, q=None, v=None, w=None):
    p = dict(x=np.zeros(n), y=np.zeros(n), z=np.zeros(n), r_par=np.full(n, rpar), r_perp=np.full(n, rperp))
    q = np.tile([1.0, 0, 0, 0], (n, 1)) if q is None else np.asarray(q, np.float64)
    for d, k in enumerate(("qw", "qx", "qy", "qz")):
        p[k] = q[:, d].copy()
    v = np.zeros((n, 3)) if v is None else np.asarray(v, np.float64)
    w = np.zeros((n, 3)) if w is None else np.asarray(w, np.float64)
    for d, k in enumerate(("vx", "vy", "vz")):
        p[k] = v[:, d].copy()
    for d, k in enumerate(("wx", "wy", "wz")):
        p[k] = w[:, d].copy()
    return p


def axis(p):
    w, x, y, z = (np.asarray(p[k]) for k in ("qw", "qx", "qy", "qz"))
    s = 2.0 / (w * w + x * x + y * y + z * z)
    return np.stack([s * (x * z + w * y), s * (y * z - w * x), 1 - s * (x * x + y * y)], 1)


def test_constant_force_recurrence():
    rng = np.random.default_rng(1)
    p = body(3, 6.0, 3.0, v=rng.normal(0, 1e-2, (3, 3)))
    x0 = np.stack([p["x"], p["y"], p["z"]], 1)
    v0 = np.stack([p["vx"], p["vy"], p["vz"]], 1)
    F = rng.normal(0, 1.0, (3, 3))
    rho, dt, n = 1.3, 0.1, 50
    m = rho * 4 / 3 * np.pi * 6.0 * 3.0 ** 2
    zero = np.zeros((3, 3))
    for _ in range(n):
        p = oracle.rigid_step(p, zero, zero, rho, dt, f_ext=F)
    k = np.arange(1, n + 1)
    v_n = v0 + n * dt * F / m
    x_n = x0 + dt * (n * v0 + (dt * F / m) * k.sum())
    np.testing.assert_allclose(np.stack([p["vx"], p["vy"], p["vz"]], 1), v_n, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(np.stack([p["x"], p["y"], p["z"]], 1), x_n, rtol=1e-12, atol=1e-12)


def test_sphere_spun_up_about_a_fixed_axis():
    e = np.array([1.0, 2.0, -2.0]) / 3.0
    w0 = 0.01 * e
    T = 3.0 * e
    rho, dt, n, R = 1.0, 0.05, 200, 4.0
    p = body(1, R, R, w=[w0])
    I = 0.4 * rho * 4 / 3 * np.pi * R ** 3 * R * R
    for _ in range(n):
        p = oracle.rigid_step(p, np.zeros((1, 3)), np.zeros((1, 3)), rho, dt, t_ext=[T])
    wn = np.array([p["wx"][0], p["wy"][0], p["wz"][0]])
    np.testing.assert_allclose(wn, w0 + n * dt * T / I, rtol=1e-12)
    theta = dt * sum(np.linalg.norm(w0 + k * dt * T / I) for k in range(1, n + 1))
    q = np.array([p["qw"][0], p["qx"][0], p["qy"][0], p["qz"][0]])
    np.testing.assert_allclose(q, np.r_[np.cos(theta / 2), np.sin(theta / 2) * e], atol=1e-12)


def precession_error(dt, t_end=2.0):
    rpar, rperp, rho = 6.0, 3.0, 1.0
    tilt = 0.7
    q0 = [[np.cos(tilt / 2), np.sin(tilt / 2), 0.0, 0.0]]          # axis tilted about x
    w0 = np.array([[0.2, -0.1, 0.5]])
    p = body(1, rpar, rperp, q=q0, w=w0)
    m = rho * 4 / 3 * np.pi * rpar * rperp ** 2
    ipar, iperp = 0.4 * m * rperp ** 2, 0.2 * m * (rpar ** 2 + rperp ** 2)
    o0 = axis(p)[0]
    L0 = iperp * (w0[0] - o0 * (o0 @ w0[0])) + ipar * o0 * (o0 @ w0[0])
    n = int(round(t_end / dt))
    for _ in range(n):
        p = oracle.rigid_step(p, np.zeros((1, 3)), np.zeros((1, 3)), rho, dt)
    o = axis(p)[0]
    w = np.array([p["wx"][0], p["wy"][0], p["wz"][0]])
    L = iperp * (w - o * (o @ w)) + ipar * o * (o @ w)
    # exact: o rotated about L^ by |L| t / I_perp (Rodrigues)
    k = L0 / np.linalg.norm(L0)
    ang = np.linalg.norm(L0) * t_end / iperp
    o_ex = o0 * np.cos(ang) + np.cross(k, o0) * np.sin(ang) + k * (k @ o0) * (1 - np.cos(ang))
    return np.linalg.norm(L - L0) / np.linalg.norm(L0), np.linalg.norm(o - o_ex), ang


def test_torque_free_symmetric_top_precesses_about_L():
    errL, err1, ang = precession_error(0.01)
    assert ang > 0.5                        # a sizeable precession angle
    assert errL < 1e-13                     # angular momentum kept exactly
    assert err1 < 1e-3
    _, err2, _ = precession_error(0.005)
    assert err2 < 0.6 * err1                # first-order convergence to the exact motion
