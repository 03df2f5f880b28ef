"""The C-ABI library builds, loads and exports every symbol the headers declare.

CPU-only: no compute call is made.  Struct layouts of the ctypes binding are
compared with the C compiler's view of include/info_esrf.h.
"""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def _declared_functions():
    names = set()
    for f in os.listdir(INCLUDE):
        if f.endswith(".h"):
            text = open(os.path.join(INCLUDE, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names.update(re.findall(r"\b(info_esrf_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2503_00253_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


def test_binding_loads_and_reports(lib):
    from paper_2503_00253_gb300 import binding
    L = binding.library()
    assert L.info_esrf_version() >= 10000
    assert L.info_esrf_error_string(-2).decode().startswith("observation index")
    o = binding.Options()
    L.info_esrf_default_options(ctypes.byref(o))
    assert (o.precision, o.ritz_rank, o.oversample, o.max_iter) == (0, 10, 10, 1000)


def test_struct_layouts_match_c(tmp_path):
    from paper_2503_00253_gb300 import binding
    src = tmp_path / "sz.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "info_esrf.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(info_esrf_grid),"
        " sizeof(info_esrf_options), sizeof(info_esrf_stats), sizeof(info_esrf_problem),"
        " offsetof(info_esrf_options, seed), offsetof(info_esrf_problem, tol),"
        " offsetof(info_esrf_problem, max_oo)); return 0;}\n")
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", INCLUDE, str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(binding.Grid), ctypes.sizeof(binding.Options), ctypes.sizeof(binding.Stats),
            ctypes.sizeof(binding.ProblemC), binding.Options.seed.offset, binding.ProblemC.tol.offset,
            binding.ProblemC.max_oo.offset]
    assert got == want


def test_host_side_validation_without_gpu(lib):
    """Argument checks that run before any CUDA call return error codes."""
    from paper_2503_00253_gb300 import binding
    L = binding.library()
    g = binding.Grid()
    for i in range(3):
        g.shape[i] = 1
        g.half_width[i] = 1.0
    g.shape[0] = 100
    g.half_width[0] = 5.0
    o = binding.make_options()
    # workspace sizes are positive and grow with Q
    s1 = L.info_esrf_workspace_size(ctypes.byref(g), 10, 20, 4, ctypes.byref(o))
    s2 = L.info_esrf_workspace_size(ctypes.byref(g), 10, 20, 8, ctypes.byref(o))
    assert 0 < s1 < s2
    # invalid: N < 2, d > n, bad half-width, too many Ritz vectors
    assert L.info_esrf_workspace_size(ctypes.byref(g), 1, 20, 4, ctypes.byref(o)) == 0
    assert L.info_esrf_workspace_size(ctypes.byref(g), 10, 200, 4, ctypes.byref(o)) == 0
    o2 = binding.make_options(ritz_rank=40)
    assert L.info_esrf_workspace_size(ctypes.byref(g), 10, 20, 4, ctypes.byref(o2)) == 0
    # cluster sizes: 0 (chosen), -1 (band kernel off), 2, 4, 8; anything else is rejected
    for cs, ok in ((0, True), (-1, True), (2, True), (4, True), (8, True), (3, False), (16, False), (-2, False)):
        oc = binding.make_options(cluster_size=cs)
        assert (L.info_esrf_workspace_size(ctypes.byref(g), 10, 20, 4, ctypes.byref(oc)) > 0) == ok, cs
    g.half_width[0] = 0.0
    assert L.info_esrf_workspace_size(ctypes.byref(g), 10, 20, 4, ctypes.byref(o)) == 0
    # null workspace is rejected before any launch
    g.half_width[0] = 5.0
    rc = L.info_esrf_analysis(ctypes.byref(g), 10, 8, 20, 8, 8, 8, 4, 1e-8, ctypes.byref(o), None, 0,
                              None, 8, 8, None)
    assert rc == binding.ERR_WORKSPACE


def test_multishift_plan_limits_without_gpu(lib):
    """Workspace sizing runs on the host: the solver option is validated, a d whose
    full direction vector cannot fit a CTA's shared memory is unsupported (size 0),
    and shifted directions that do not fit shared memory get a scratch area."""
    from paper_2503_00253_gb300 import binding
    L = binding.library()

    def grid(n, hw):
        g = binding.Grid()
        for i in range(3):
            g.shape[i] = 1
            g.half_width[i] = 1.0
        g.shape[0] = n
        g.half_width[0] = hw
        return g

    g = grid(8192, 5.0)
    ms = dict(solver=binding.SOLVER_MULTISHIFT)
    for sv, ok in ((0, True), (1, True), (2, True), (3, False), (-1, False)):
        o = binding.make_options(solver=sv)
        assert (L.info_esrf_workspace_size(ctypes.byref(g), 10, 1024, 8, ctypes.byref(o)) > 0) == ok, sv
    # one chain's p in shared memory: about 35,000 FP32 observations at most
    big = grid(80000, 5.0)
    o32 = binding.make_options(precision=binding.PRECISION_FP32, **ms)
    assert L.info_esrf_workspace_size(ctypes.byref(big), 10, 40000, 8, ctypes.byref(o32)) == 0
    assert L.info_esrf_workspace_size(ctypes.byref(big), 10, 20000, 8, ctypes.byref(o32)) > 0
    pcg = binding.make_options(precision=binding.PRECISION_FP32)
    assert L.info_esrf_workspace_size(ctypes.byref(big), 10, 40000, 8, ctypes.byref(pcg)) > 0
    # FP64, 48 shifts: at 2 CTAs per cluster (512 rows each) the directions need scratch,
    # at 8 (128 rows) they fit in shared memory
    o2 = binding.make_options(precision=binding.PRECISION_FP64, cluster_size=2, **ms)
    o8 = binding.make_options(precision=binding.PRECISION_FP64, cluster_size=8, **ms)
    s2 = L.info_esrf_workspace_size(ctypes.byref(g), 10, 1024, 48, ctypes.byref(o2))
    s8 = L.info_esrf_workspace_size(ctypes.byref(g), 10, 1024, 48, ctypes.byref(o8))
    assert s2 >= s8 + 160 * 48 * 512 * 8, (s2, s8)
