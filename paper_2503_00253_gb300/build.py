"""Builds the CUDA library ``libinfo_esrf.so`` in-tree for sm_103a.

Compiles every ``csrc/*.cu`` translation unit in parallel with nvcc and links
them into ``paper_2503_00253_gb300/lib/libinfo_esrf.so``.  No PyTorch is
involved; the library's C ABI is declared in ``include/info_esrf.h`` and
``include/info_esrf_stages.h``.

``build(phase_clocks=True)`` makes a second, instrumented library,
``libinfo_esrf_phase.so`` (objects in ``lib/obj_phase``), compiled with
``-DINFO_ESRF_PHASE_CLOCKS``: the 1-D band PCG kernel then records clock
counts per phase of each round (``info_esrf_band_phase_clocks``).  The
binding loads it instead of the default library when the environment has
``INFO_ESRF_PHASE_CLOCKS=1``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(PKG, "lib")
OBJDIR = os.path.join(LIBDIR, "obj")
LIBNAME = "libinfo_esrf.so"
PHASE_LIBNAME = "libinfo_esrf_phase.so"
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def library_path(phase_clocks: bool = False) -> str:
    return os.path.join(LIBDIR, PHASE_LIBNAME if phase_clocks else LIBNAME)


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return cand


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps():
    files = _sources()
    files += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return files


def up_to_date(phase_clocks: bool = False) -> bool:
    lib = library_path(phase_clocks)
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False, phase_clocks: bool = False) -> str:
    """Compiles and links the library if any source is newer; returns its path."""
    if not force and up_to_date(phase_clocks):
        return library_path(phase_clocks)
    objdir = os.path.join(LIBDIR, "obj_phase") if phase_clocks else OBJDIR
    os.makedirs(objdir, exist_ok=True)
    nvcc = _nvcc()
    flags = [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
             "-I" + INCLUDE, "-I" + CSRC, "--expt-relaxed-constexpr"]
    if phase_clocks:
        flags.append("-DINFO_ESRF_PHASE_CLOCKS")
    procs = []
    objs = []
    for src in _sources():
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        cmd = [nvcc] + flags + ["-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((src, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"), file=sys.stderr)
    if failed:
        msg = "\n".join(f"{s}:\n{o}" for s, o in failed)
        raise RuntimeError(f"nvcc failed:\n{msg}")
    tmp = library_path(phase_clocks) + ".tmp"
    cmd = [nvcc, "-shared", ARCH, "-o", tmp] + objs
    subprocess.run(cmd, check=True, capture_output=not verbose)
    os.replace(tmp, library_path(phase_clocks))
    return library_path(phase_clocks)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, phase_clocks="--phase-clocks" in sys.argv))
