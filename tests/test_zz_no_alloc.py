"""lub_pairs_build_static: the pair build for callers that cannot allocate
device memory (a host code that owns a fixed device-memory budget and
forbids allocation after start-up, since cudaMalloc synchronises the device
and can fail mid-run).  It runs on a fixed static device array of the
library instead of a context's scratch.

Checked through the C ABI against lub_pairs_build on two calls in a row with
different inputs (the array keeps the previous call's contents, so the second
call shows that what must start at zero is cleared), on a sparse box whose
natural cell grid exceeds the array's cell limit (the coarsened grid), plus
the size limit.
"""
import ctypes

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lub():
    import torch

    import paper_1308_6482_gb300 as lubmod
    from paper_1308_6482_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    return lubmod


def _static_vs_context(lub, parts, dom):
    import torch
    pl = lub.Pipeline(parts, dom, lub.default_params())
    cnt = pl.build_pairs()                     # the existing entry point (context scratch)
    ref = pl.results()
    cap = pl.cap
    pi = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
    pj = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
    dc = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = lub.lub_pairs_build_static(pl.P.c, pl.D, pl.prm, pi, pj, cap, dc)
    assert rc == lub.LUB_OK
    torch.cuda.synchronize()
    m = int(dc.item())
    assert m == cnt
    np.testing.assert_array_equal(pi[:m].cpu().numpy(), ref["pi"])
    np.testing.assert_array_equal(pj[:m].cpu().numpy(), ref["pj"])
    return m


def test_static_scratch_matches_context_build_twice(lub):
    # call 1: the 32,768-particle, Phi = 0.3 mixed suspension of the benchmark
    parts, dom = gen.config_mixed_suspension()
    m1 = _static_vs_context(lub, parts, dom)
    # call 2: a different, smaller suspension with a wall (other grid, fewer cells)
    parts2, dom2 = gen.config_prolate_wall(seed=3)
    m2 = _static_vs_context(lub, parts2, dom2)
    assert m1 > 10000 and m2 > 0


def test_static_coarsens_a_grid_beyond_its_cell_limit(lub):
    # 20,000 unit spheres placed uniformly in a periodic 400^3 box: cells of
    # the full range (2 r + Delta_L = 3) would be 133^3 = 2.4M, above
    # LUB_STATIC_MAX_CELLS; the static build coarsens its grid and must still
    # list the same pairs as the context build
    rng = np.random.default_rng(17)
    n, L = 20000, 400.0
    c = rng.uniform(0.0, L, size=(n, 3))
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    parts = dict(x=c[:, 0], y=c[:, 1], z=c[:, 2], qw=q[:, 0].astype(np.float32), qx=q[:, 1].astype(np.float32),
                 qy=q[:, 2].astype(np.float32), qz=q[:, 3].astype(np.float32),
                 r_par=np.ones(n, np.float32), r_perp=np.ones(n, np.float32))
    gen.velocities(parts, rng)
    dom = dict(L=(L, L, L), periodic=(True, True, True), walls=[])
    assert n <= lub._lib.LUB_STATIC_MAX_PARTICLES and (L / 3.0) ** 3 > lub._lib.LUB_STATIC_MAX_CELLS
    assert _static_vs_context(lub, parts, dom) > 100


def test_static_rejects_sizes_beyond_its_limit(lub):
    import torch
    dc = torch.zeros(1, dtype=torch.int32, device="cuda")
    p = lub._lib.lub_particles()
    p.n = lub._lib.LUB_STATIC_MAX_PARTICLES + 1
    p.max_semi_axis = 1.0
    d = lub.make_domain(dict(L=(100.0, 100.0, 100.0), periodic=(True, True, True)))
    prm = lub.default_params()
    rc = lub.load_library().lub_pairs_build_static(ctypes.byref(p), ctypes.byref(d), ctypes.byref(prm), None, None,
                                                   0, dc.data_ptr(), None)
    assert rc == lub.LUB_ERR_LIMIT
