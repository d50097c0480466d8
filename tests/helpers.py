"""Shared test helpers: small particle configurations and rigid transforms.

Nothing here computes lubrication quantities; expected values come from the
oracle or from closed forms written in the tests themselves.
"""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

FIELDS = ("x", "y", "z", "qw", "qx", "qy", "qz", "r_par", "r_perp", "vx", "vy", "vz", "wx", "wy", "wz")


def read_constants():
    out = {}
    with open(os.path.join(GOLDEN, "paper_constants.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, val = line.split()[:2]
            out[name] = float(val)
    return out


def make_parts(pos, quat, rpar, rperp, v=None, w=None):
    pos = np.asarray(pos, np.float64).reshape(-1, 3)
    n = len(pos)
    quat = np.asarray(quat, np.float64).reshape(n, 4)
    v = np.zeros((n, 3)) if v is None else np.asarray(v, np.float64).reshape(n, 3)
    w = np.zeros((n, 3)) if w is None else np.asarray(w, np.float64).reshape(n, 3)
    return dict(x=pos[:, 0].copy(), y=pos[:, 1].copy(), z=pos[:, 2].copy(),
                qw=quat[:, 0].copy(), qx=quat[:, 1].copy(), qy=quat[:, 2].copy(), qz=quat[:, 3].copy(),
                r_par=np.asarray(rpar, np.float64).reshape(n).copy(),
                r_perp=np.asarray(rperp, np.float64).reshape(n).copy(),
                vx=v[:, 0].copy(), vy=v[:, 1].copy(), vz=v[:, 2].copy(),
                wx=w[:, 0].copy(), wy=w[:, 1].copy(), wz=w[:, 2].copy())


def open_domain(L=1e4):
    return dict(L=(L, L, L), periodic=(False, False, False), walls=[])


def quat_mul(a, b):
    """Hamilton product, scalar first, broadcasting over leading dims."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    w1, x1, y1, z1 = np.moveaxis(a, -1, 0)
    w2, x2, y2, z2 = np.moveaxis(b, -1, 0)
    return np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], axis=-1)


def quat_to_mat(q):
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def axis_angle_quat(axis, ang):
    axis = np.asarray(axis, np.float64)
    axis = axis / np.linalg.norm(axis)
    return np.concatenate([[np.cos(ang / 2)], np.sin(ang / 2) * axis])


def quat_from_z_to(o):
    """A quaternion rotating body z onto the unit vector o."""
    o = np.asarray(o, np.float64)
    o = o / np.linalg.norm(o)
    z = np.array([0.0, 0.0, 1.0])
    c = float(np.dot(z, o))
    if c > 1 - 1e-15:
        return np.array([1.0, 0, 0, 0])
    if c < -1 + 1e-15:
        return np.array([0.0, 1.0, 0, 0])
    ax = np.cross(z, o)
    return axis_angle_quat(ax, np.arccos(c))


def rigid_transform(parts, R, t, qR):
    """Rotate (R, quaternion qR) and translate (t) a configuration with its velocities."""
    out = {k: np.array(v, np.float64, copy=True) for k, v in parts.items()}
    pos = np.stack([out["x"], out["y"], out["z"]], 1) @ R.T + t
    out["x"], out["y"], out["z"] = pos[:, 0].copy(), pos[:, 1].copy(), pos[:, 2].copy()
    q = np.stack([out["qw"], out["qx"], out["qy"], out["qz"]], 1)
    q2 = quat_mul(np.broadcast_to(qR, q.shape), q)
    out["qw"], out["qx"], out["qy"], out["qz"] = [q2[:, k].copy() for k in range(4)]
    for a, b, c in (("vx", "vy", "vz"), ("wx", "wy", "wz")):
        v = np.stack([out[a], out[b], out[c]], 1) @ R.T
        out[a], out[b], out[c] = v[:, 0].copy(), v[:, 1].copy(), v[:, 2].copy()
    return out


def spheroid_point(q, rpar, rperp, r, p, qq):
    """Lab position of the surface point (p, q) of Eq. lub:spheroid."""
    yb = np.array([rperp * np.cos(p) * np.cos(qq), rperp * np.cos(p) * np.sin(qq), rpar * np.sin(p)])
    return np.asarray(r) + quat_to_mat(q) @ yb


def spheroid_normal(q, rpar, rperp, p, qq):
    """Outward unit normal at (p, q), from the implicit form x^2/a^2 + y^2/a^2 + z^2/c^2 = 1."""
    yb = np.array([rperp * np.cos(p) * np.cos(qq), rperp * np.cos(p) * np.sin(qq), rpar * np.sin(p)])
    g = np.array([yb[0] / rperp ** 2, yb[1] / rperp ** 2, yb[2] / rpar ** 2])
    n = quat_to_mat(q) @ g
    return n / np.linalg.norm(n)
