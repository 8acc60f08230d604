"""Builds libfe.so in-tree with nvcc for sm_103a (no cmake, no setuptools).

Every translation unit under csrc/ is compiled in parallel into _build/, then linked into
``paper_2603_09038_gb300/libfe.so`` against the shared CUDA runtime.  Rebuilds only what changed
(source or header newer than its object).
"""
import concurrent.futures
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfe.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE,
              "--expt-relaxed-constexpr"] + ARCH


def nvcc():
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found; libfe needs the CUDA 13 toolkit")
    return cand


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _headers():
    return glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def _obj(src):
    return os.path.join(BUILD, os.path.basename(src) + ".o")


def _stale(src, newest_header):
    o = _obj(src)
    return not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(src), newest_header)


def _compile(src, extra):
    cmd = [nvcc(), "-c", src, "-o", _obj(src)] + NVCC_FLAGS + extra
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed on %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
    return r.stderr


def build(verbose=False, extra_flags=(), jobs=None):
    """Compile (if needed) and link libfe.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources()
    newest = max(os.path.getmtime(h) for h in _headers())
    todo = [s for s in srcs if _stale(s, newest)]
    if todo:
        n = jobs or min(len(todo), os.cpu_count() or 4)
        with concurrent.futures.ThreadPoolExecutor(max_workers=n) as ex:
            for src, log in zip(todo, ex.map(lambda s: _compile(s, list(extra_flags)), todo)):
                if verbose and log.strip():
                    print(os.path.basename(src), log, file=sys.stderr)
    objs = [_obj(s) for s in srcs]
    if todo or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(map(os.path.getmtime, objs)):
        cmd = [nvcc(), "-shared", "-o", LIB] + objs + ARCH + [
            "-cudart", "shared", "-Xlinker", "-rpath=/usr/local/cuda/lib64"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
