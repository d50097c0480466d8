"""Parity helpers: run the CUDA path through the C ABI and the oracle on the
same seeded inputs, and compare them element by element.

Tolerances (written here, used by every GPU parity test):
  * indices and pair lists: bit-exact;
  * gap: |h_gpu - h_ref| <= 1e-10 (|d| + Rmax_i + Rmax_j) in both precisions
    (the gap is always evaluated in double);
  * forces and torques, per pair: the error of the lab force (torque)
    vector is at most
        tol * sum_{g in rows, d} |mu K~_gd u_d|  (+ |F_r| when the repulsion acts)
      + KAPPA * eps * sum_{g, d} |mu K~_gd| S_d    (rows of both kinds, torque
                                                    rows divided by a for forces,
                                                    force rows times a for torques)
    with tol = 1e-9 (FP64 mode) or 1e-5 (mixed mode).  The first term is the
    component-wise relative error against the terms that make up the row.
    The second is the rounding floor of forming the relative surface velocity
    u from the inputs in the mode's arithmetic: S_d = |v_i| + |v_j| +
    |w_i||y*_i - r_i| + |w_j||y*_j - r_j| for the translational columns and
    |w_i| + |w_j| for the rotational ones, eps = 2^-24 (mixed) or 2^-53
    (FP64), KAPPA = 64, a = the smaller semi-axis of the pair.  Without it a
    normal velocity that is a near-cancellation of FP32 inputs (u_3 << S)
    could never meet a relative bound in FP32 arithmetic.  Per particle the
    bound is the sum of the bounds of its pairs, with lever arms for the
    torque;
  * lever arms: 1e-12 (FP64) or 2e-6 (mixed) times the semi-axis.
"""
import numpy as np

import oracle

TOL = {"fp64": 1e-9, "mixed": 1e-5}
EPS = {"fp64": 2.0 ** -53, "mixed": 2.0 ** -24}
KAPPA = 64.0


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
    # velocity scales of the rounding floor
    v = np.stack([parts[k] for k in ("vx", "vy", "vz")], 1).astype(np.float64)
    w = np.stack([parts[k] for k in ("wx", "wy", "wz")], 1).astype(np.float64)
    wall = pj < 0
    jj = np.where(wall, 0, pj)
    vn_j = np.where(wall, 0.0, np.linalg.norm(v[jj], axis=1))
    wn_j = np.where(wall, 0.0, np.linalg.norm(w[jj], axis=1))
    vn_i, wn_i = np.linalg.norm(v[pi], axis=1), np.linalg.norm(w[pi], axis=1)
    li, lj = np.linalg.norm(pf["lever"][:, :3], axis=1), np.linalg.norm(pf["lever"][:, 3:], axis=1)
    S = np.zeros((len(pi), 6))
    S[:, :3] = (vn_i + vn_j + wn_i * li + wn_j * lj)[:, None]
    S[:, 3:] = (wn_i + wn_j)[:, None]
    mag = absK * S[:, None, :]
    mf = mag[:, :3, :].sum(axis=(1, 2))
    mt = mag[:, 3:, :].sum(axis=(1, 2))
    rp, rq = parts["r_par"].astype(np.float64), parts["r_perp"].astype(np.float64)
    a = np.minimum(rp[pi], rq[pi])
    a = np.where(wall, a, np.minimum(a, np.minimum(rp[jj], rq[jj])))
    floor_f = mf + mt / a
    floor_t = mt + mf * a
    return dict(cp=cp, pf=pf, force=f, torque=t, bound_f=bf, bound_t=bt, floor_f=floor_f, floor_t=floor_t)


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
    """Assert parity of a GPU result dict against an oracle reference."""
    tol = TOL[prec]
    fl = KAPPA * EPS[prec]
    cp, pf = ref["cp"], ref["pf"]
    st_ref = pf["status"] & 7
    st_gpu = g["status"].astype(np.int64) & 7
    np.testing.assert_array_equal(st_gpu, st_ref)
    ok = (st_ref & (oracle.ST_NOCONV | oracle.ST_DEGENERATE)) == 0
    sc = scale_of(parts, dom, pi, pj)
    dh = np.abs(g["h"] - cp["h"])
    assert np.all(dh[ok] <= 1e-10 * sc[ok]), ("gap", dh[ok].max(), np.argmax(np.where(ok, dh / sc, 0)))
    errF = np.linalg.norm(g["FT"][:, :3] - pf["FT"][:, :3], axis=1)
    errT = np.linalg.norm(g["FT"][:, 3:] - pf["FT"][:, 3:], axis=1)
    allow_f = tol * ref["bound_f"] + fl * ref["floor_f"]
    allow_t = tol * ref["bound_t"] + fl * ref["floor_t"]
    rf = errF / (allow_f + 1e-300)
    rt = errT / (allow_t + 1e-300)
    assert np.all(rf <= 1.0), ("pair force", float(rf.max()), int(np.argmax(rf)))
    assert np.all(rt <= 1.0), ("pair torque", float(rt.max()), int(np.argmax(rt)))
    rmax = np.maximum(parts["r_par"], parts["r_perp"]).astype(np.float64)
    ltol = (1e-12 if prec == "fp64" else 2e-6) * rmax[pi][:, None]
    act = (pf["FT"] != 0).any(1)
    assert np.all(np.abs(g["lever"] - pf["lever"])[act] <= ltol[act]), "lever"
    if check_particles:
        n = len(parts["x"])
        lev = np.linalg.norm(pf["lever"][:, :3], axis=1)
        levj = np.linalg.norm(pf["lever"][:, 3:], axis=1)
        BF = np.zeros(n)
        BT = np.zeros(n)
        np.add.at(BF, pi, allow_f)
        np.add.at(BT, pi, allow_t + lev * allow_f)
        wj = pj >= 0
        np.add.at(BF, pj[wj], allow_f[wj])
        np.add.at(BT, pj[wj], (allow_t + levj * allow_f)[wj])
        ef = np.linalg.norm(g["force"] - ref["force"], axis=1)
        et = np.linalg.norm(g["torque"] - ref["torque"], axis=1)
        # summation of the pair terms in the mode's arithmetic adds its own rounding
        sf = np.zeros(n)
        st_ = np.zeros(n)
        np.add.at(sf, pi, np.linalg.norm(pf["FT"][:, :3], axis=1))
        np.add.at(sf, pj[wj], np.linalg.norm(pf["FT"][wj, :3], axis=1))
        tt = np.linalg.norm(pf["FT"][:, 3:], axis=1) + lev * np.linalg.norm(pf["FT"][:, :3], axis=1)
        np.add.at(st_, pi, tt)
        np.add.at(st_, pj[wj], (np.linalg.norm(pf["FT"][:, 3:], axis=1) + levj * np.linalg.norm(pf["FT"][:, :3], axis=1))[wj])
        BF += fl * sf
        BT += fl * st_
        assert np.all(ef <= BF + 1e-30), ("particle force", float((ef / (BF + 1e-300)).max()))
        assert np.all(et <= BT + 1e-30), ("particle torque", float((et / (BT + 1e-300)).max()))
    return dict(max_rf=float(rf.max(initial=0)), max_rt=float(rt.max(initial=0)))
