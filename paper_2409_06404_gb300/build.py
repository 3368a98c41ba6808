"""Build libnkchem.so (the CUDA library behind include/nkchem.h) in-tree for sm_103a.

    python -m paper_2409_06404_gb300.build [--force] [--ptxas-v]

Each .cu under csrc/ is compiled by its own nvcc process (in parallel), then linked into
paper_2409_06404_gb300/_build/libnkchem.so with the CUDA runtime linked statically.  The
benchmark's pipe-throughput probe (probe/pipe_peaks.cu) is built beside it as libnkprobe.so.
"""
from __future__ import annotations

import argparse
import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libnkchem.so")
PROBE_SRC = os.path.join(HERE, "probe", "pipe_peaks.cu")
PROBE_LIB = os.path.join(OUT, "libnkprobe.so")     # pipe-throughput probe of the benchmark
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
GEN = os.path.join(OUT, "gen")
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC, "-I", GEN]


def _write_embedded_sources():
    """The run-time compiled kernel (jit.cu) includes the text of nk_math.cuh: write it as a raw
    string literal into the build directory."""
    os.makedirs(GEN, exist_ok=True)
    with open(os.path.join(CSRC, "nk_math.cuh")) as f:
        text = f.read()
    assert ")nkmathsrc" not in text
    body = 'static const char kNkMathSrc[] = R"nkmathsrc(' + text + ')nkmathsrc";\n'
    path = os.path.join(GEN, "nk_math_src.inc")
    if not os.path.exists(path) or open(path).read() != body:
        with open(path, "w") as f:
            f.write(body)


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h")) + [__file__]


def up_to_date() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(PROBE_LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps()) and os.path.getmtime(PROBE_SRC) <= os.path.getmtime(PROBE_LIB)


def build(force: bool = False, ptxas_verbose: bool = False, quiet: bool = True) -> str:
    if not force and not ptxas_verbose and up_to_date():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    _write_embedded_sources()
    cc = nvcc()
    srcs = _sources()
    extra = ["-Xptxas", "-v"] if ptxas_verbose else []

    def compile_one(src):
        obj = os.path.join(OUT, os.path.basename(src)[:-3] + ".o")
        cmd = [cc, *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        return src, obj, r

    def build_probe():
        tmp = PROBE_LIB + f".tmp{os.getpid()}"
        cmd = [cc, *ARCH, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-cudart", "static", PROBE_SRC,
               "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, PROBE_LIB)
        return r

    with ThreadPoolExecutor(max_workers=min(len(srcs) + 1, os.cpu_count() or 4)) as ex:
        probe = ex.submit(build_probe)
        results = list(ex.map(compile_one, srcs))
        rp = probe.result()
    if rp.returncode != 0:
        sys.stderr.write(rp.stdout + rp.stderr)
        raise RuntimeError(f"nvcc failed on {PROBE_SRC}")
    log = []
    for src, obj, r in results:
        log.append(f"== {os.path.basename(src)}\n{r.stdout}{r.stderr}")
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError(f"nvcc failed on {src}")
    with open(os.path.join(OUT, "build.log"), "w") as f:
        f.write("\n".join(log))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *[o for _, o, _ in results], "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("link of libnkchem.so failed")
    os.replace(tmp, LIB)
    if not quiet or ptxas_verbose:
        print("\n".join(log))
    return LIB


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--ptxas-v", action="store_true")
    a = ap.parse_args()
    print(build(force=a.force, ptxas_verbose=a.ptxas_v, quiet=False))


if __name__ == "__main__":
    main()
