"""Compile the GTQA CUDA library in-tree (nvcc, sm_103a only).

The shared library is written next to this file as libgtqa.so.  Sources are
the .cu files under csrc/; the public header is include/gtqa.h at the
repository root.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from typing import List, Optional

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG_DIR)
CSRC = os.path.join(PKG_DIR, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB_PATH = os.path.join(PKG_DIR, "libgtqa.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# (source, object name, extra defines): gtqa_units.cu is compiled once per precision mode
# and kernel family, so the eight instantiation sets build in parallel
_UNIT_NAMES = ("gates", "bp", "regauge", "general")
SOURCES = [("gtqa_api.cu", "gtqa_api", []), ("gtqa_diag.cu", "gtqa_diag", []),
           ("gtqa_static.cu", "gtqa_static", []), ("gtqa_plain.cu", "gtqa_plain", [])] + [
    ("gtqa_units.cu", f"gtqa_{mode.lower()[4:]}_{name}", [f"-DGTQA_UNIT_MODE={mode}", f"-DGTQA_UNIT={u}"])
    for mode in ("ModeFP64", "ModeMixed") for u, name in enumerate(_UNIT_NAMES)]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the GTQA CUDA library cannot be built")


def _deps() -> List[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))]
    files.append(os.path.join(INCLUDE, "gtqa.h"))
    return files


def needs_build() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    return any(os.path.getmtime(f) > t for f in _deps())


def build(force: bool = False, verbose: bool = False, extra: Optional[List[str]] = None) -> str:
    """Build libgtqa.so if missing or stale; returns its path."""
    if not force and not needs_build():
        return LIB_PATH
    nvcc = _nvcc()
    objs = []
    procs = []
    for src, name, defs in SOURCES:
        obj = os.path.join(PKG_DIR, "_build", name + ".o")
        os.makedirs(os.path.dirname(obj), exist_ok=True)
        cmd = [nvcc, *ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, *defs,
               "-c", os.path.join(CSRC, src), "-o", obj] + (extra or [])
        if verbose:
            print(" ".join(cmd))
        procs.append((subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT), cmd))
        objs.append(obj)
    for p, cmd in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + out.decode(errors="replace"))
    tmp = LIB_PATH + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, LIB_PATH)
    return LIB_PATH
