"""The C-ABI library builds, loads without a GPU and exports every symbol that
include/pxa.h declares; argument validation answers without touching a device."""
import ctypes
import os
import re

import pytest

from paper_2004_00546_gb300 import pxa

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"^\s*(?:int|void|const char\*)\s+(pxa_\w+)\s*\(", text, flags=re.M))
    return names


def test_header_declares_the_binding_exports():
    decl = declared_functions()
    assert decl, "no declarations parsed"
    assert decl == set(pxa.EXPORTS)


def test_library_exports_every_declared_symbol(pxa_lib):
    for name in declared_functions():
        assert hasattr(pxa_lib, name), name


def test_invalid_arguments_are_rejected_without_a_device(pxa_lib):
    L = pxa_lib
    assert L.pxa_set_operator(None, None) == pxa.ERR_INVALID
    assert L.pxa_set_time(None, 1.0, 10, pxa.CN, 1) == pxa.ERR_INVALID
    assert L.pxa_gradient(None, 0, None, None) == pxa.ERR_INVALID
    L.pxa_destroy(None)  # must be a no-op
    assert L.pxa_last_error(None) == b"null context"
    h = ctypes.c_void_p()
    assert L.pxa_create(ctypes.byref(h), 4096, None) == pxa.ERR_CUDA
    assert L.pxa_create(None, 0, None) == pxa.ERR_INVALID


def test_partition_bounds_follow_the_nonequidistant_partition(pxa_lib):
    """Host logic of the overlapped direct solve: chunk boundaries are the partition of
    Eq. nonEquiP (pinned in the oracle), rounded to whole steps or subintervals."""
    from oracle import partition_nonequi
    import numpy as np

    # P == 1: chunks of steps; K large enough that rounding moves no boundary by > 1/2
    K = 1_000_000
    for r in (0.3, 0.59, 0.7, 0.9):
        b = pxa.partition_bounds(K, 1, r, 8)
        kk = r / (1.0 - r)  # k with k/(k+1) = r (the oracle takes k)
        ref = partition_nonequi(1.0, 8, kk) * K
        assert len(b) == 9 and b[0] == 0 and b[-1] == K
        assert np.all(np.abs(np.array(b) - ref) <= 0.5 + 1e-6), (r, b, ref)
    # r == 0: equal chunks
    assert pxa.partition_bounds(20000, 32, 0.0, 8) == [2500 * i for i in range(9)]
    assert pxa.partition_bounds(20000, 1, 0.0, 8) == [2500 * i for i in range(9)]
    # P > 1: whole subintervals, at least one per chunk, strictly increasing
    for P, r in ((32, 0.37), (32, 0.59), (8, 0.2), (4, 0.5), (3, 0.9)):
        K = 625 * P
        b = pxa.partition_bounds(K, P, r, 8)
        nc = min(P, 8)
        assert len(b) == nc + 1 and b[0] == 0 and b[-1] == K
        d = np.diff(b)
        assert np.all(d >= 625) and np.all(d % 625 == 0)
        if P >= 8 and r < 0.6:
            assert d[0] >= d[-1]  # the chunks shrink towards T
    # argument errors
    out = (ctypes.c_int64 * 9)()
    assert pxa_lib.pxa_partition_bounds(0, 1, 0.0, 8, out) == pxa.ERR_INVALID
    assert pxa_lib.pxa_partition_bounds(10, 3, 0.0, 8, out) == pxa.ERR_INVALID
    assert pxa_lib.pxa_partition_bounds(10, 1, 1.0, 8, out) == pxa.ERR_INVALID
    assert pxa_lib.pxa_partition_bounds(10, 1, 0.5, 8, None) == pxa.ERR_INVALID


def test_batch_entry_points_reject_bad_arguments_without_a_device(pxa_lib):
    L = pxa_lib
    h = ctypes.c_void_p()
    assert L.pxa_batch_create(ctypes.byref(h), 4096, None) == pxa.ERR_CUDA
    assert L.pxa_batch_create(None, 0, None) == pxa.ERR_INVALID
    assert L.pxa_batch_set(None, 1, None, None, 1.0, 1.0, 1.0, 16, 1) == pxa.ERR_INVALID
    assert L.pxa_batch_gradient(None, 0, None, None, None) == pxa.ERR_INVALID
    assert L.pxa_batch_sync(None) == pxa.ERR_INVALID
    assert L.pxa_batch_last_error(None) == b"null batch"
    L.pxa_batch_destroy(None)  # must be a no-op
    assert L.pxa_batch_set_power(None, 1) == pxa.ERR_INVALID
    assert L.pxa_batch_set_lane_steps(None, 4) == pxa.ERR_INVALID
    assert L.pxa_batch_set_homogeneous(None, 1.0) == pxa.ERR_INVALID


def test_setters_reject_null_contexts_and_bad_values_without_a_device(pxa_lib):
    """The configuration calls added for the multi-checkpoint scheme, the lanes' product
    bands and the propagator choice answer on the host: a null context, an interval
    count, a CN-steps-per-band value or a propagator outside their ranges."""
    L = pxa_lib
    assert L.pxa_set_checkpoints(None, 5) == pxa.ERR_INVALID
    assert L.pxa_set_lane_steps(None, 4) == pxa.ERR_INVALID
    assert L.pxa_set_propagator(None, pxa.PROP_BAND, 150) == pxa.ERR_INVALID
    assert L.pxa_set_partition(None, 0.5) == pxa.ERR_INVALID
    assert L.pxa_spmv_csr(None, 0, None, None, None, None, None) == pxa.ERR_INVALID


def test_header_is_plain_c():
    """include/pxa.h compiles on its own as C99 and as C++17 (a C ABI: no C++ types)."""
    import shutil
    import subprocess

    hdr = os.path.join(ROOT, "include", "pxa.h")
    for cc, std, lang in (("gcc", "-std=c99", "c"), ("g++", "-std=c++17", "c++")):
        if not shutil.which(cc):
            pytest.skip(f"{cc} not available")
        r = subprocess.run([cc, std, "-Wall", "-Wextra", "-Werror", "-fsyntax-only", "-x", lang, hdr],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_objective_and_precision_setters_reject_null_contexts(pxa_lib):
    L = pxa_lib
    assert L.pxa_set_objective(None, None) == pxa.ERR_INVALID
    d = pxa.ObjectiveDesc(pxa.OBJ_TERMINAL_L2, None)
    assert L.pxa_set_objective(None, ctypes.byref(d)) == pxa.ERR_INVALID
    assert L.pxa_set_precision(None, pxa.F32) == pxa.ERR_INVALID


def test_binding_structs_have_the_header_layout(tmp_path):
    """The ctypes structures of the binding have the sizes and field offsets of the C
    structures in include/pxa.h (compiled by the host C compiler)."""
    import shutil
    import subprocess

    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    fields = {"pxa_operator_desc": (pxa.OperatorDesc, ["n", "L", "u_dev", "row_ptr_dev", "col_dev", "val_dev"]),
              "pxa_objective_desc": (pxa.ObjectiveDesc, ["kind", "target_dev"]),
              "pxa_stats": (pxa.Stats, ["workspace_bytes", "prop_band_taps", "side_chunks", "ms_side_lanes"]),
              "pxa_batch_stats": (pxa.BatchStats, ["krylov_reach", "ms_total", "lane_steps"])}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{os.path.join(ROOT, "include", "pxa.h")}"',
             "int main(void) {"]
    for name, (_, fl) in fields.items():
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for f in fl:
            lines.append(f'  printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-o", str(exe), str(src)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                    check=True).stdout.splitlines())
    for name, (cls, fl) in fields.items():
        assert int(out[name]) == ctypes.sizeof(cls), name
        for f in fl:
            assert int(out[f"{name}.{f}"]) == getattr(cls, f).offset, (name, f)
