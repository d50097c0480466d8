"""Build liblub.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel with
``nvcc -gencode arch=compute_103a,code=sm_103a -O3 -lineinfo`` and linked
into ``paper_1308_6482_gb300/liblub.so`` (static CUDA runtime).  The library
has a plain C ABI (``include/lub.h``) and no PyTorch dependency.
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
SO = os.path.join(HERE, "liblub.so")
BUILD_TESTING = os.path.join(HERE, "_build_testing")
SO_TESTING = os.path.join(HERE, "liblub_testing.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["api.cu", "scan.cu", "pairs.cu", "pairs_static.cu", "closest.cu", "resistance.cu", "apply.cu", "mlp.cu", "tune.cu", "rigid.cu", "links.cu", "trace.cu"]


def nvcc():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblub")
    return p


def _stale(so=SO):
    if not os.path.exists(so):
        return True
    t = os.path.getmtime(so)
    for d in (CSRC, os.path.join(HERE, "..", "include")):
        for f in os.listdir(d):
            if os.path.getmtime(os.path.join(d, f)) > t:
                return True
    return False


def build(force=False, verbose=False, ptxas_info=False, testing=False):
    """Build liblub.so; testing=True builds liblub_testing.so instead: the same
    sources with short bounds on the device waits and the test hooks that make
    them run out (LUB_TESTING), for the tests of the timeout paths."""
    so, bdir = (SO_TESTING, BUILD_TESTING) if testing else (SO, BUILD)
    if not force and not _stale(so):
        return so
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                    "--expt-relaxed-constexpr"]
    if testing:
        flags += ["-DLUB_TESTING", "-DLUB_SCAN_SPIN_LIMIT=(1l<<14)", "-DLUB_TC_SPIN_LIMIT=(1l<<14)"]
    if ptxas_info:
        flags += ["-Xptxas", "-v"]

    def one(src):
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        cmd = [cc, "-c", os.path.join(CSRC, src), "-o", obj] + flags
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        return obj, r.stderr

    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, len(SOURCES))) as ex:
        results = list(ex.map(one, SOURCES))
    if verbose or ptxas_info:
        for _, err in results:
            if err:
                sys.stderr.write(err)
    tmp = so + ".tmp%d" % os.getpid()
    cmd = [cc, "-shared", "-o", tmp] + [o for o, _ in results] + ARCH + ["-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, so)
    return so


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(SO)
