"""Reynolds thin-film lubrication between two exact spheroid surfaces near
their points of closest approach: an independent check of the ln h
coefficients of the Appendix that the exchange symmetry cannot pin.

The gap H(x) = z_j(x) - z_i(x) over the tangent plane at y*_i (axes e1, e2,
normal e3 from i towards j) is taken from the spheroids themselves, not from
their quadratic and cubic expansions.  For a pure squeeze (j translating
along e3 at unit speed relative to i, no rotation, mu = 1) the film pressure
solves the Reynolds equation

    div(H^3 grad p) = 12 mu dH/dt = 12,   p = 0 on the rim r = R0,

here by finite volumes on a log-polar grid (cells r in [r_in, R0], theta in
[0, 2 pi), zero flux through the tiny inner rim).  The fluid acts on i with
the pressure on its tilted surface and the wall shear of the Poiseuille
profile, -(H/2) grad p; integrated by parts (p = 0 on the rim) the
tangential force is

    F_t = int p grad z_m dA,   z_m = (z_i + z_j) / 2,

and the torque about y*_i, to leading order, that of the pressure:
T = (-int p x2 dA, int p x1 dA); the normal force is -int p dA.  These are
the forces of the lubrication theory the Appendix expands (Sec. III B);
differencing two small gaps leaves the coefficient of ln h.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def spheroid_matrix(q, r_par, r_perp):
    """A with (y - r)^T A (y - r) = 1 on the surface; q scalar first, body z = axis."""
    qd = np.asarray(q, np.float64)
    w, x, y, z = qd / np.linalg.norm(qd)
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    a, c = float(r_perp), float(r_par)  # in double: float32 semi-axes would shift the surface by ~1e-7 R
    D = np.diag([1 / a ** 2, 1 / a ** 2, 1 / c ** 2])
    return R @ D @ R.T


def surface_height(A, c, y0, e1, e2, e3, x1, x2):
    """Height z along e3 of the spheroid (A, centre c) over y0 + x1 e1 + x2 e2,
    the root nearest y0 (a surface point), and its gradient (dz/dx1, dz/dx2)."""
    d0 = (y0 - c)[None, None, :] + x1[..., None] * e1 + x2[..., None] * e2
    Ae3 = A @ e3
    a = e3 @ Ae3
    b = d0 @ Ae3
    cc = np.einsum("...i,ij,...j->...", d0, A, d0) - 1.0
    disc = np.sqrt(np.maximum(b * b - a * cc, 0.0))
    z = -cc / (b + np.where(b >= 0, disc, -disc))
    w = d0 + z[..., None] * e3
    Aw = w @ A
    den = Aw @ e3
    return z, -(Aw @ e1) / den, -(Aw @ e2) / den


def squeeze(Ai, ci, Aj, cj, yi, e1, e2, e3, h, R0, nr=480, nth=96, r_in=None):
    """Normal force, tangential force (e1, e2) and tangential torque (e1, e2)
    on i for unit squeeze (mu = 1), with j's contact point at yi + h e3; Aj
    None: j is a plane wall through that point, normal to e3."""
    if r_in is None:
        r_in = 1e-3 * np.sqrt(h)
    re = np.geomspace(r_in, R0, nr + 1)          # radial cell edges
    rc = np.sqrt(re[:-1] * re[1:])               # cell centres
    dth = 2 * np.pi / nth
    th = (np.arange(nth) + 0.5) * dth
    tf = np.arange(nth) * dth                     # angular faces (between th[l-1] and th[l])
    yj = yi + h * e3

    def gap(r, t):
        x1, x2 = r * np.cos(t), r * np.sin(t)
        zi, gi1, gi2 = surface_height(Ai, ci, yi, e1, e2, e3, x1, x2)
        if Aj is None:
            zj, gj1, gj2 = np.zeros_like(zi), np.zeros_like(zi), np.zeros_like(zi)
        else:
            zj, gj1, gj2 = surface_height(Aj, cj, yj, e1, e2, e3, x1, x2)
        return h + zj - zi, 0.5 * (gi1 + gj1), 0.5 * (gi2 + gj2), x1, x2

    Rc, Tc = np.meshgrid(rc, th, indexing="ij")
    Hc, gm1, gm2, X1, X2 = gap(Rc, Tc)
    # H^3 on the radial faces (edges re[1..nr]) and angular faces
    Rr, Tr = np.meshgrid(re[1:], th, indexing="ij")
    Hr3 = gap(Rr, Tr)[0] ** 3
    Ra, Ta = np.meshgrid(rc, tf, indexing="ij")
    Ha3 = gap(Ra, Ta)[0] ** 3
    area = 0.5 * (re[1:] ** 2 - re[:-1] ** 2)[:, None] * dth * np.ones((1, nth))
    idx = np.arange(nr * nth).reshape(nr, nth)
    rows, cols, vals = [], [], []
    diag = np.zeros((nr, nth))

    def couple(a, b, g):
        rows.extend([a.ravel(), b.ravel(), a.ravel(), b.ravel()])
        cols.extend([b.ravel(), a.ravel(), a.ravel(), b.ravel()])
        vals.extend([g.ravel(), g.ravel(), -g.ravel(), -g.ravel()])

    # radial faces between cells k and k+1
    gr = (re[1:-1, None] * Hr3[:-1] * dth) / (rc[1:] - rc[:-1])[:, None]
    couple(idx[:-1], idx[1:], gr)
    # outer rim: p = 0 at re[nr]
    diag[-1] -= re[-1] * Hr3[-1] * dth / (re[-1] - rc[-1])
    # angular faces between l-1 and l (periodic)
    ga = Ha3 * (re[1:] - re[:-1])[:, None] / (rc[:, None] * dth)
    couple(idx, np.roll(idx, 1, axis=1), ga)
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    M = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nr * nth,) * 2)
    # symmetric diagonal scaling: H^3 spans many decades between the contact
    # point and the rim, which a direct solve of the raw system does not survive
    s = 1.0 / np.sqrt(np.abs(M.diagonal()))
    S = sp.diags(s)
    y = spla.spsolve((S @ M @ S).tocsc(), s * (12.0 * area).ravel())
    p = (s * y).reshape(nr, nth)
    pa = p * area
    return dict(F3=-pa.sum(), F=np.array([(pa * gm1).sum(), (pa * gm2).sum()]),
                T=np.array([-(pa * X2).sum(), (pa * X1).sum()]), pmax=np.abs(p).max())
