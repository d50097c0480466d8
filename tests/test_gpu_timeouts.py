"""Bounded device waits: a wait that runs out returns, and the host learns of
it (lub_sync_status reports LUB_ERR_TIMEOUT), with the context usable after.

The waits are made to run out without faulting or hanging the GPU, in the
test build of the library (liblub_testing.so: the same sources with short
wait bounds and two test hooks, LUB_TESTING), run in a child process:

* the decoupled look-back of the device-wide scan: one tile never publishes
  its total (as if its block never ran), so the next tile's look-back polls
  to its bound, sets the timeout bit and carries on;
* the tcgen05 network: the elected thread issues no MMA and no commit, so
  every mbarrier wait for an MMA polls to its bound; with nothing in flight
  the kernel frees its TMEM and returns.

The product build's status word stays clear in normal operation.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import ctypes, json, sys, time
sys.path.insert(0, ROOT)
import numpy as np
import torch
import gen
import paper_1308_6482_gb300 as lub
from paper_1308_6482_gb300.mlp import WarmStartMLP
L = lub.load_library()
vp = ctypes.c_void_p
L.lub_test_scan.restype = ctypes.c_int
L.lub_test_scan.argtypes = [vp, vp, ctypes.c_int64, vp, ctypes.c_int32, vp]
L.lub_test_skip_tc_mma.restype = ctypes.c_int
L.lub_test_skip_tc_mma.argtypes = [ctypes.c_int32]
torch.cuda.set_device(0)
out = {"library": lub.library_path()}

def status(ctx):
    try:
        lub.lub_sync_status(ctx.h)
        return 0
    except lub.LubError as e:
        return e.code

ctx = lub.Context()
n = 300000
data = torch.ones(n, dtype=torch.int32, device="cuda")
tot = torch.zeros(1, dtype=torch.int32, device="cuda")
assert L.lub_test_scan(ctx.h, data.data_ptr(), n, tot.data_ptr(), -1, None) == 0
out["plain_scan_exact"] = bool(torch.equal(data, torch.arange(n, dtype=torch.int32, device="cuda"))) and tot.item() == n
out["plain_scan_status"] = status(ctx)
data.fill_(1)
t0 = time.time()
assert L.lub_test_scan(ctx.h, data.data_ptr(), n, tot.data_ptr(), 3, None) == 0
out["stalled_scan_s"] = time.time() - t0
out["stalled_scan_status"] = status(ctx)
out["status_after_clear"] = status(ctx)
data.fill_(1)
assert L.lub_test_scan(ctx.h, data.data_ptr(), n, tot.data_ptr(), -1, None) == 0
out["scan_after_timeout_exact"] = bool(torch.equal(data, torch.arange(n, dtype=torch.int32, device="cuda")))

parts, dom, pi, pj = gen.pair_stream(2000, seed=81, kind="aspect", gap_range=(1e-4, 1.0), gap_scale="min_axis")
net = WarmStartMLP.load()
pl = lub.Pipeline(parts, dom, lub.default_params(precision="fp64", warm_start="mlp"))
net.install(pl.ctx)
pl.set_pairs(pi, pj)
pq = torch.zeros(4 * pl.cap, dtype=torch.float32, device="cuda")
def predict(engine):
    lub.lub_mlp_engine(pl.ctx.h, engine)
    pq.zero_()
    lub.lub_mlp_predict(pl.ctx.h, pl.P.c, pl.D, pl.pair_i, pl.pair_j, pl.d_count, pl.cap, pq)
    torch.cuda.synchronize()
    return pq.cpu().numpy().reshape(4, -1)[:, :len(pi)].copy()
ref = predict("mma_sync")
out["mma_sync_status"] = status(pl.ctx)
assert L.lub_test_skip_tc_mma(1) == 0
t0 = time.time()
predict("tcgen05")
out["stalled_tc_s"] = time.time() - t0
out["stalled_tc_status"] = status(pl.ctx)
assert L.lub_test_skip_tc_mma(0) == 0
y = predict("tcgen05")
out["tc_after_timeout_status"] = status(pl.ctx)
out["tc_after_timeout_err"] = float(np.abs(y - ref).max() / np.abs(ref).max())
print("RESULT " + json.dumps(out))
""".replace("ROOT", repr(ROOT))


@pytest.fixture(scope="module")
def result():
    from paper_1308_6482_gb300 import build
    so = build.build(testing=True)
    env = dict(os.environ, LUB_LIBRARY=so)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    return json.loads(line[7:])


def test_the_child_ran_the_test_build(result):
    assert result["library"].endswith("liblub_testing.so")


def test_scan_lookback_timeout_is_reported(result):
    import paper_1308_6482_gb300 as lub
    assert result["plain_scan_exact"] and result["plain_scan_status"] == 0
    assert result["stalled_scan_status"] == lub.LUB_ERR_TIMEOUT
    assert result["stalled_scan_s"] < 30.0
    # the record is cleared by the check, and the context works on
    assert result["status_after_clear"] == 0 and result["scan_after_timeout_exact"]


def test_tcgen05_mbarrier_timeout_is_reported(result):
    import paper_1308_6482_gb300 as lub
    assert result["mma_sync_status"] == 0
    assert result["stalled_tc_status"] == lub.LUB_ERR_TIMEOUT
    assert result["stalled_tc_s"] < 30.0
    assert result["tc_after_timeout_status"] == 0 and result["tc_after_timeout_err"] < 3e-2


def test_product_status_stays_clear():
    """A whole step of the product build leaves no timeout on record."""
    import torch

    import paper_1308_6482_gb300 as lub
    from paper_1308_6482_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    parts, dom = gen.config_mixed_suspension(N=3000, phi=0.3, seed=12)
    pl = lub.Pipeline(parts, dom, lub.default_params())
    pl.build_pairs()
    pl.step(form="merged")
    pl.apply(deterministic=1)
    lub.lub_sync_status(pl.ctx.h)
    assert np.isfinite(pl.results()["force"]).all()
