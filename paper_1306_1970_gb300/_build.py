"""Compile the CUDA library (libflr.so) in-tree for sm_103a with nvcc."""
import os
import shutil
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libflr.so")
SOURCES = ["flr_api.cu", "flr_noalloc.cu", "flr_server.cu", "flr_dense.cu"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
              "-Xcompiler", "-fPIC", "-shared"]


def _deps():
    out = [os.path.join(INCLUDE, "flr.h")]
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cuh", ".h")):
            out.append(os.path.join(CSRC, f))
    return out


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(d) > t for d in _deps())


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the FLR CUDA library cannot be built")
    return exe


def build(force: bool = False, verbose: bool = False) -> str:
    """Build libflr.so next to this file if it is missing or older than its sources."""
    if not force and not stale():
        return LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=HERE)
    os.close(fd)
    objdir = tempfile.mkdtemp(prefix="flr_build_")
    objs = [os.path.join(objdir, s + ".o") for s in SOURCES]
    # translation units compile in parallel, then one link step
    procs = []
    for s, o in zip(SOURCES, objs):
        cmd = [nvcc()] + NVCC_FLAGS[:-1] + ["-c", "-I", INCLUDE, os.path.join(CSRC, s), "-o", o]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append(subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE))
    errs = []
    for pr in procs:
        out, err = pr.communicate()
        if pr.returncode != 0:
            errs.append(err.decode(errors="replace"))
    try:
        if errs:
            raise RuntimeError("nvcc failed building libflr.so:\n" + "\n".join(errs))
        link = [nvcc(), "-shared", "-gencode", "arch=compute_103a,code=sm_103a"] + objs + ["-o", tmp]
        r = subprocess.run(link, capture_output=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc link failed:\n" + r.stderr.decode(errors="replace"))
    except Exception:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise
    finally:
        shutil.rmtree(objdir, ignore_errors=True)
    os.replace(tmp, LIB)
    return LIB
