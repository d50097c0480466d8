"""Parity helpers: run the CUDA path through the C ABI and the oracle on the
same seeded inputs, and compare them element by element.

Tolerances (written here, used by every GPU parity test):
  * indices and pair lists: bit-exact;
  * gap: |h_gpu - h_ref| <= 1e-10 (|d| + Rmax_i + Rmax_j) in both precisions
    (the gap is always evaluated in double);
  * unit normals: |n_gpu - n_ref| <= 1e-10 in both precisions (the mixed
    mode refines every FP32 normal in float-float);
  * forces and torques, per pair: the error of the lab force vector is at
    most
        tol * B_F,  B_F = sum_{g in force rows, d} |mu K~_gd u_d|  (+ |F_r| when the repulsion acts)
    and that of the torque about y*_i at most tol * (B_T + |y*_i - r_i| B_F),
    B_T the same sum over the torque rows, with tol = 1e-9 (FP64 mode) or
    1e-5 (mixed mode): the component-wise relative error against the terms
    that make up the rows, and for the torque against the terms of the
    torque on the particle about its centre, T_i + (y*_i - r_i) x F_i.  (The
    torque rows alone can vanish identically: for equal spheres c - lambda =
    0 makes K14, K15, K24, K25 zero, so with Delta_r < h < Delta_t every
    torque element is a cancellation that any rounding order leaves at
    rounding level, against an oracle bound of zero.)  Per particle the
    bound is the sum of the bounds of its pairs, with lever arms for the
    torque;
  * lever arms: 1e-12 (FP64) or 2e-6 (mixed) times the semi-axis.
"""
import numpy as np

import oracle

TOL = {"fp64": 1e-9, "mixed": 1e-5}


def prm_dict(prec="mixed", **kw):
    d = dict(oracle.DEFAULT_PARAMS)
    d.update(kw)
    return d


def gpu_params(prec, **kw):
    import paper_1308_6482_gb300 as lub
    return lub.default_params(precision=prec, **kw)


def run_gpu(parts, dom, prec, pi=None, pj=None, deterministic=0, capacity=None, **kw):
    import torch

    import paper_1308_6482_gb300 as lub
    pl = lub.Pipeline(parts, dom, gpu_params(prec, **kw), capacity=capacity)
    if pi is None:
        pl.build_pairs()
    else:
        pl.set_pairs(pi, pj)
    pl.closest()
    pl.resistance()
    pl.apply(deterministic=deterministic)
    torch.cuda.synchronize()
    return pl.results()


def oracle_ref(parts, dom, pi, pj, **kw):
    prm = prm_dict(**kw)
    cp = oracle.closest(parts, dom, pi, pj)
    pf = oracle.pair_force(parts, dom, prm, pi, pj, cp, want_k=True, want_geom=True)
    f, t = oracle.apply(len(parts["x"]), pi, pj, pf["FT"], pf["lever"])
    absK = np.abs(pf["Kt"]) * prm["mu"]
    terms = absK * np.abs(pf["geom"][:, None, 27:33])
    bf = terms[:, :3, :].sum(axis=(1, 2))
    bt = terms[:, 3:, :].sum(axis=(1, 2))
    if prm["h_c"] > 0:
        h = cp["h"]
        fr = np.where(h <= prm["h_c"], np.where(h > 0, prm["eps_c"] * (prm["h_c"] - h), prm["eps_c"] * prm["h_c"]), 0)
        bf = bf + np.abs(fr)
    return dict(cp=cp, pf=pf, force=f, torque=t, bound_f=bf, bound_t=bt)


def scale_of(parts, dom, pi, pj):
    pos = np.stack([parts["x"], parts["y"], parts["z"]], 1).astype(np.float64)
    rm = np.maximum(parts["r_par"], parts["r_perp"]).astype(np.float64)
    out = np.empty(len(pi))
    wall = pj < 0
    d = pos[np.where(wall, pi, pj)] - pos[pi]
    L = np.asarray(dom["L"])
    per = np.asarray(dom["periodic"], bool)
    d[:, per] -= L[per] * np.floor(d[:, per] / L[per] + 0.5)
    out[:] = np.linalg.norm(d, axis=1) + rm[pi] + np.where(wall, 0, rm[np.maximum(pj, 0)])
    return out


def compare(parts, dom, g, ref, prec, pi, pj, check_particles=True):
    """Assert parity of a GPU result dict against an oracle reference.
    check_particles: True (every particle), False (none) or an index array
    (those particles only: the ones whose pairs are all among pi, pj)."""
    tol = TOL[prec]
    cp, pf = ref["cp"], ref["pf"]
    st_ref = pf["status"] & 7
    st_gpu = g["status"].astype(np.int64) & 7
    np.testing.assert_array_equal(st_gpu, st_ref)
    ok = (st_ref & (oracle.ST_NOCONV | oracle.ST_DEGENERATE)) == 0
    sc = scale_of(parts, dom, pi, pj)
    dh = np.abs(g["h"] - cp["h"])
    assert np.all(dh[ok] <= 1e-10 * sc[ok]), ("gap", dh[ok].max(), np.argmax(np.where(ok, dh / sc, 0)))
    dn = np.linalg.norm(g["n"] - cp["n"], axis=1)
    assert np.all(dn[ok] <= 1e-10), ("normal", float(dn[ok].max(initial=0)), int(np.argmax(np.where(ok, dn, 0))))
    errF = np.linalg.norm(g["FT"][:, :3] - pf["FT"][:, :3], axis=1)
    errT = np.linalg.norm(g["FT"][:, 3:] - pf["FT"][:, 3:], axis=1)
    lev = np.linalg.norm(pf["lever"][:, :3], axis=1)
    levj = np.linalg.norm(pf["lever"][:, 3:], axis=1)
    allow_f = tol * ref["bound_f"]
    allow_t = tol * ref["bound_t"]  # torque rows only
    allow_ti = allow_t + lev * allow_f
    rf = errF / (allow_f + 1e-300)
    rt = errT / (allow_ti + 1e-300)
    assert np.all(rf <= 1.0), ("pair force", float(rf.max()), int(np.argmax(rf)))
    assert np.all(rt <= 1.0), ("pair torque", float(rt.max()), int(np.argmax(rt)))
    rmax = np.maximum(parts["r_par"], parts["r_perp"]).astype(np.float64)
    ltol = (1e-12 if prec == "fp64" else 2e-6) * rmax[pi][:, None]
    act = (pf["FT"] != 0).any(1)
    assert np.all(np.abs(g["lever"] - pf["lever"])[act] <= ltol[act]), "lever"
    if check_particles is not False:
        sel = slice(None) if check_particles is True else np.asarray(check_particles)
        n = len(parts["x"])
        BF = np.zeros(n)
        BT = np.zeros(n)
        np.add.at(BF, pi, allow_f)
        np.add.at(BT, pi, allow_t + lev * allow_f)
        wj = pj >= 0
        np.add.at(BF, pj[wj], allow_f[wj])
        np.add.at(BT, pj[wj], (allow_t + levj * allow_f)[wj])
        ef = np.linalg.norm(g["force"][sel] - ref["force"][sel], axis=1)
        et = np.linalg.norm(g["torque"][sel] - ref["torque"][sel], axis=1)
        BF, BT = BF[sel], BT[sel]
        assert np.all(ef <= BF + 1e-30), ("particle force", float((ef / (BF + 1e-300)).max()))
        assert np.all(et <= BT + 1e-30), ("particle torque", float((et / (BT + 1e-300)).max()))
    return dict(max_rf=float(rf.max(initial=0)), max_rt=float(rt.max(initial=0)))
