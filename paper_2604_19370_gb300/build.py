"""Build libwf.so in-tree for sm_103a (GB300) with nvcc.

The CUDA sources under csrc/ are compiled in parallel to objects in
_build/ and linked into _build/libwf.so.  Nothing is installed outside the
package directory.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import json
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(OUT, "libwf.so")

SOURCES = ["wf_tables.cu", "wf_rhs.cu", "wf_rhs_stream.cu", "wf_solve.cu", "wf_linefast.cu", "wf_api.cu", "wf_server.cu", "wf_mms.cu", "wf_probe.cu", "wf_persist.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libwf")


STAMP = os.path.join(OUT, "stamp.json")
#: what the last build_library call did: "compiled" (objects rebuilt) or "up to date"
LAST_BUILD = {"mode": None}


def _digest(paths, extra: str) -> str:
    h = hashlib.sha256(extra.encode())
    for p in sorted(paths):
        h.update(os.path.basename(p).encode())
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _stamp_key(nvcc: str, headers) -> dict:
    """Per-object source hashes (source + every header + flags + nvcc + host machine)."""
    ver = subprocess.run([nvcc, "--version"], capture_output=True, text=True).stdout.strip().splitlines()[-1:]
    extra = " ".join(ARCH + FLAGS[:5]) + "|" + "".join(ver) + "|" + platform.machine()
    return {src: _digest([os.path.join(CSRC, src)] + headers, extra) for src in SOURCES}


def build_library(force: bool = False, verbose: bool = False) -> str:
    """Compile (if needed) and return the path of libwf.so.

    An object is rebuilt unless the stamp next to it records the same hash of its source, every
    header, the flags, the nvcc version and the host machine type: a _build/ folder made by
    another machine, toolkit or source tree is never reused.  LAST_BUILD["mode"] says whether this
    call compiled.
    """
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(INCLUDE, "wf.h"))
    key = _stamp_key(nvcc, headers)
    try:
        with open(STAMP) as f:
            old = json.load(f)
    except Exception:
        old = {}
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT, src.replace(".cu", ".o"))
        objs.append(o)
        if force or not os.path.exists(o) or old.get(src) != key[src]:
            jobs.append([nvcc, *ARCH, *FLAGS, "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed ({' '.join(cmd)}):\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stdout.write(r.stdout + r.stderr)

    if os.path.exists(STAMP):
        os.unlink(STAMP)  # a build interrupted below leaves no stamp behind
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        list(ex.map(run, jobs))
    if force or jobs or not os.path.exists(LIB) or old.get("lib") != key_lib(key):
        tmp = LIB + ".tmp"
        run([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, LIB)
    with open(STAMP, "w") as f:
        json.dump({**key, "lib": key_lib(key)}, f)
    LAST_BUILD["mode"] = "compiled" if jobs else "up to date"
    return LIB


def key_lib(key: dict) -> str:
    return hashlib.sha256("".join(key[s] for s in SOURCES).encode()).hexdigest()


if __name__ == "__main__":
    print(build_library(force="--force" in sys.argv, verbose=True), LAST_BUILD["mode"])
