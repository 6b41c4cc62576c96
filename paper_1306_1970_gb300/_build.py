"""Compile the CUDA library (libflr.so) in-tree for sm_103a with nvcc."""
import os
import shutil
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libflr.so")
SOURCES = ["flr_api.cu"]
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
    cmd = [nvcc()] + NVCC_FLAGS + ["-I", INCLUDE] + [os.path.join(CSRC, s) for s in SOURCES] + ["-o", tmp]
    if verbose:
        print(" ".join(cmd), flush=True)
    try:
        subprocess.run(cmd, check=True, capture_output=not verbose)
    except subprocess.CalledProcessError as e:
        os.unlink(tmp)
        msg = (e.stderr or b"").decode(errors="replace")
        raise RuntimeError(f"nvcc failed building libflr.so:\n{msg}") from None
    os.replace(tmp, LIB)
    return LIB
