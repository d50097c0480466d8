"""The C-ABI library builds, loads without a GPU and exports every symbol the
header declares; the Python binding's structures match the C layout."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lub.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1308_6482_gb300 import build
    build.build()
    import paper_1308_6482_gb300 as lub
    return lub.load_library()


def header_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lub_[a-z_]+)\s*\(", src)))


def test_header_declares_the_four_calls():
    fns = header_functions()
    for name in ("lub_pairs_build", "lub_closest_points", "lub_resistance", "lub_apply"):
        assert name in fns


def test_library_exports_every_declared_symbol(lib):
    import paper_1308_6482_gb300._lib as L
    for name in header_functions():
        assert hasattr(lib, name), name
    assert sorted(L.EXPORTS) == sorted(header_functions())


def test_struct_layout_matches_c(lib):
    import paper_1308_6482_gb300._lib as L
    code = r"""
#include <stdio.h>
#include <stddef.h>
#include "lub.h"
int main(void) {
  printf("%zu %zu %zu\n", sizeof(lub_particles), sizeof(lub_domain), sizeof(lub_params));
  printf("%zu %zu %zu %zu\n", offsetof(lub_particles, n), offsetof(lub_particles, max_semi_axis),
         offsetof(lub_domain, wall_dir), offsetof(lub_domain, n_walls));
  printf("%zu %zu %zu %zu\n", offsetof(lub_params, precision), offsetof(lub_params, fp64_switch),
         offsetof(lub_params, newton_tol), offsetof(lub_params, warm_start));
  printf("%zu %zu %zu\n", offsetof(lub_particles, batch_offsets), offsetof(lub_particles, n_batches),
         offsetof(lub_params, model));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(code)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = subprocess.check_output([exe]).decode().split()
    vals = list(map(int, out))
    assert vals[:3] == [ctypes.sizeof(L.lub_particles), ctypes.sizeof(L.lub_domain), ctypes.sizeof(L.lub_params)]
    assert vals[3] == L.lub_particles.n.offset
    assert vals[4] == L.lub_particles.max_semi_axis.offset
    assert vals[5] == L.lub_domain.wall_dir.offset
    assert vals[6] == L.lub_domain.n_walls.offset
    assert vals[7] == L.lub_params.precision.offset
    assert vals[8] == L.lub_params.fp64_switch.offset
    assert vals[9] == L.lub_params.newton_tol.offset
    assert vals[10] == L.lub_params.warm_start.offset
    assert vals[11] == L.lub_particles.batch_offsets.offset
    assert vals[12] == L.lub_particles.n_batches.offset
    assert vals[13] == L.lub_params.model.offset


def test_default_params_are_the_papers(lib):
    import paper_1308_6482_gb300 as lub
    p = lub.default_params()
    assert p.mu == pytest.approx(1 / 6) and p.delta_n == pytest.approx(2 / 3)
    assert p.delta_t == 0.5 and p.delta_r == 0.25
    assert p.precision == lub.LUB_MIXED and p.fp64_switch == 1e-3


def test_argument_errors_without_gpu(lib):
    """Calls with invalid arguments return LUB_ERR_ARG before touching the GPU."""
    import paper_1308_6482_gb300._lib as L
    assert lib.lub_ctx_create(None) == L.LUB_ERR_ARG
    assert lib.lub_pairs_build(None, None, None, None, None, None, 0, None, None, None) == L.LUB_ERR_ARG
    assert lib.lub_apply(None, None, None, None, 0, None, None, 0, None, None, 0, 0, 0, None) == L.LUB_ERR_ARG
    assert lib.lub_last_error(None) == b"no context"


def test_no_cpu_fallback_in_the_product_package():
    """The binding never imports the oracle and has no host compute path."""
    pkg = os.path.join(ROOT, "paper_1308_6482_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            src = open(os.path.join(pkg, f)).read()
            assert "import oracle" not in src and "from oracle" not in src, f


def test_header_constants_match_the_binding():
    """Every integer constant of the header has the same value in the
    binding (return codes, modes, status bits, limits)."""
    import paper_1308_6482_gb300._lib as L
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    consts = dict(re.findall(r"^#define\s+(LUB_[A-Z0-9_]+)\s+\(?(-?\d+)\)?\s*$", src, flags=re.M))
    assert len(consts) > 30
    for name, value in consts.items():
        if name == "LUB_STATIC_SCRATCH_BYTES":
            continue  # the size of the static array: host code never passes it
        assert hasattr(L, name), name
        assert getattr(L, name) == int(value), (name, getattr(L, name), value)
