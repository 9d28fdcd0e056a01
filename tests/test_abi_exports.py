"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/rgcsr.h declares; host-only argument checks answer without a
GPU (no compute call is made here)."""
import ctypes
import os
import re

import pytest

from paper_1012_2270_gb300 import build as B
from paper_1012_2270_gb300 import _lib as L

HEADER = os.path.join(B.INCLUDE, "rgcsr.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if not n.startswith("__")))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("rgcsr_plan", "rgcsr_convert", "rgcsr_spmv", "hyb_plan", "hyb_convert", "hyb_spmv"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in L.SIGNATURES, f"binding lacks {name}"


def test_only_declared_symbols_are_exported(lib):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    ours = {s for s in exported if s.startswith(("rgcsr_", "hyb_"))}
    assert ours == set(declared_functions())


def test_status_strings_and_version(lib):
    assert lib.rgcsr_version() >= 100
    for code in range(-7, 1):
        assert lib.rgcsr_status_string(code)
    assert lib.rgcsr_status_string(L.RGCSR_ERR_COL_OOB).decode().startswith("column")


def test_workspace_sizes_host_only(lib):
    assert lib.rgcsr_plan_workspace_bytes(0, 32) > 0
    a = lib.rgcsr_plan_workspace_bytes(1_000_000, 32)
    b = lib.rgcsr_plan_workspace_bytes(1_000_000, 1)
    assert b > a > 0
    assert lib.rgcsr_plan_workspace_bytes(10, 0) == 0
    assert lib.hyb_workspace_bytes(1000, 1000) >= 8 * 1001


def _argument_checks():
    """Host-side argument checks, run by test_argument_errors_without_gpu
    in a child process that sees no GPU.  Several calls below pass small
    integers as device pointers; they are never dereferenced because the
    library rejects the call first.  Without a visible device a check that
    failed to fire would end in RGCSR_ERR_CUDA (and fail the test), never
    in a device access."""
    B.build()
    lib = L.lib()
    assert lib.rgcsr_plan(None, None, None, 0, None) == L.RGCSR_ERR_INVALID_ARG
    A = L.CSR(n_rows=-1)
    M = L.Matrix(group_size=32)
    assert lib.rgcsr_plan(ctypes.byref(A), ctypes.byref(M), None, 0, None) == L.RGCSR_ERR_INVALID_ARG
    A = L.CSR(n_rows=4, n_cols=4, nnz=0, row_ptr_type=L.I64T, value_type=L.BF16)
    assert lib.rgcsr_plan(ctypes.byref(A), ctypes.byref(M), None, 0, None) == L.RGCSR_ERR_UNSUPPORTED_DTYPE
    A = L.CSR(n_rows=2**31, n_cols=4, nnz=0, row_ptr_type=L.I64T, value_type=L.F32)
    assert lib.rgcsr_plan(ctypes.byref(A), ctypes.byref(M), None, 0, None) == L.RGCSR_ERR_INDEX_OVERFLOW
    A = L.CSR(n_rows=4, n_cols=4, nnz=0, row_ptr_type=L.I64T, value_type=L.F32, row_ptr=1)
    M = L.Matrix(group_size=32, group_ptr=1, row_lengths=1)
    assert lib.rgcsr_plan(ctypes.byref(A), ctypes.byref(M), None, 0, None) == L.RGCSR_ERR_WORKSPACE
    # an empty matrix is a no-op
    M0 = L.Matrix(n_rows=0, n_cols=0, group_size=32, value_type=L.F32)
    assert lib.rgcsr_spmv(ctypes.byref(M0), None, None, None) == L.RGCSR_OK
    M1 = L.Matrix(n_rows=4, n_cols=4, group_size=0, value_type=L.F32)
    assert lib.rgcsr_spmv(ctypes.byref(M1), None, None, None) == L.RGCSR_ERR_INVALID_ARG
    H = L.Hyb(n_rows=3, n_cols=3, value_type=L.BF16)
    assert lib.hyb_spmv(ctypes.byref(H), None, None, None) == L.RGCSR_ERR_UNSUPPORTED_DTYPE
    # a long-row schedule with segments needs every list, the arrival
    # counters included; the check comes before any device work (the
    # pointers here are never dereferenced)
    M2 = L.Matrix(n_rows=4, n_cols=4, group_size=32, n_groups=1, value_type=L.F32, group_ptr=8, row_lengths=8)
    full = dict(threshold=2, segment=4, n_segments=1, n_long_rows=1, seg_row=8, seg_start=8, long_row=8,
                long_first=8, long_count=8, partials=8, arrivals=8)
    for missing in ("arrivals", "partials", "seg_row"):
        S = L.LongRows(**{k: v for k, v in full.items() if k != missing})
        assert lib.rgcsr_spmv_long_rows(ctypes.byref(M2), ctypes.byref(S), 8, 8, None) == L.RGCSR_ERR_INVALID_ARG
    S = L.LongRows(**{k: v for k, v in full.items() if k != "arrivals"})
    assert lib.rgcsr_long_rows_build(ctypes.byref(M2), ctypes.byref(S), None, 0, None) == L.RGCSR_ERR_INVALID_ARG
    # the same for the group-tile schedule, which also needs G <= 32
    full = dict(tile=64, n_groups=1, n_extra=1, n_split=1, n_partials=2, first_extra=8, part_base=8,
                extra_group=8, arrivals=8, partials=8)
    for missing in ("arrivals", "partials", "extra_group"):
        T = L.Tiles(**{k: v for k, v in full.items() if k != missing})
        assert lib.rgcsr_spmv_tiles(ctypes.byref(M2), ctypes.byref(T), 8, 8, None) == L.RGCSR_ERR_INVALID_ARG
    T = L.Tiles(**{k: v for k, v in full.items() if k != "arrivals"})
    assert lib.rgcsr_tiles_build(ctypes.byref(M2), ctypes.byref(T), None) == L.RGCSR_ERR_INVALID_ARG
    M64 = L.Matrix(n_rows=4, n_cols=4, group_size=64, n_groups=1, value_type=L.F32, group_ptr=8, row_lengths=8)
    T = L.Tiles(**full)
    assert lib.rgcsr_spmv_tiles(ctypes.byref(M64), ctypes.byref(T), 8, 8, None) == L.RGCSR_ERR_INVALID_ARG
    # structural checks: descriptor errors come before any device work
    rep = L.CheckReport(flags=99)
    assert lib.rgcsr_check_matrix(None, ctypes.byref(rep), None) == L.RGCSR_ERR_INVALID_ARG
    assert lib.rgcsr_check_matrix(ctypes.byref(M2), None, None) == L.RGCSR_ERR_INVALID_ARG
    M3 = L.Matrix(n_rows=4, n_cols=4, group_size=32, n_groups=2, value_type=L.F32, group_ptr=8, row_lengths=8)
    assert lib.rgcsr_check_matrix(ctypes.byref(M3), ctypes.byref(rep), None) == L.RGCSR_ERR_INVALID_ARG
    M4 = L.Matrix(n_rows=4, n_cols=4, group_size=32, n_groups=1, value_type=L.I32T, group_ptr=8, row_lengths=8)
    assert lib.rgcsr_check_matrix(ctypes.byref(M4), ctypes.byref(rep), None) == L.RGCSR_ERR_UNSUPPORTED_DTYPE
    assert lib.rgcsr_check_matrix(ctypes.byref(M0), ctypes.byref(rep), None) == L.RGCSR_OK
    assert (rep.flags, rep.group, rep.row, rep.slot) == (0, -1, -1, -1)
    # the AUTO rule, host only (the pointers are only tested for alignment)
    def auto(**kw):
        base = dict(n_rows=4096, n_cols=4096, nnz=28000, group_size=32, n_groups=128, n_stored=28672,
                    max_row_len=7, value_type=L.F32, values=256, columns=512, group_ptr=8, row_lengths=1024)
        base.update(kw)
        k, v = ctypes.c_int32(-1), ctypes.c_int32(-1)
        assert lib.rgcsr_auto_kernel(ctypes.byref(L.Matrix(**base)), ctypes.byref(k), ctypes.byref(v)) == 0
        return k.value, v.value
    assert auto() == (L.KERNEL_LEAN, 1)                                  # dense, short rows: vector loads
    assert auto(value_type=L.F64) == (L.KERNEL_LEAN, 4)
    assert auto(value_type=L.BF16) == (L.KERNEL_LEAN, 1)
    assert auto(nnz=28000 * 3, n_stored=28672 * 3, max_row_len=21) == (L.KERNEL_TMA, 2)   # longer rows
    assert auto(values=260) == (L.KERNEL_LEAN, 0)                        # misaligned: thread per row
    assert auto(values=260, value_type=L.F64) == (L.KERNEL_LEAN, 0)
    assert auto(n_stored=28000 * 2) == (L.KERNEL_SPLIT, 0)              # padding > 25%: uneven rows
    assert auto(group_size=8, n_groups=512) == (L.KERNEL_LEAN, 0)
    k = ctypes.c_int32(0)
    assert lib.rgcsr_auto_kernel(ctypes.byref(M1), ctypes.byref(k), ctypes.byref(k)) == L.RGCSR_ERR_INVALID_ARG
    assert lib.rgcsr_auto_kernel(ctypes.byref(M2), None, ctypes.byref(k)) == L.RGCSR_ERR_INVALID_ARG
    assert lib.rgcsr_set_wait_limit(-1) == L.RGCSR_ERR_INVALID_ARG
    assert lib.rgcsr_set_wait_limit(0) == L.RGCSR_OK
    # checks mode: the switch returns the previous setting
    prev = lib.rgcsr_set_checks(1)
    assert lib.rgcsr_set_checks(0) == 1
    assert lib.rgcsr_set_checks(prev) == 0


def test_argument_errors_without_gpu():
    import subprocess
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    code = ("import sys; sys.path[:0] = [%r, %r]; import test_abi_exports as t; t._argument_checks()"
            % (here, os.path.dirname(here)))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr


def test_product_path_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(B, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(L, "_lib", None)
    with pytest.raises(RuntimeError, match="not found"):
        L.lib()


# ctypes mirror -> C typedef of include/rgcsr.h
STRUCTS = {"CSR": "rgcsr_csr", "Matrix": "rgcsr_matrix", "Launch": "rgcsr_launch", "Hyb": "hyb_matrix",
           "LongRows": "rgcsr_long_rows", "Tiles": "rgcsr_tiles", "BatchDesc": "rgcsr_batch_desc",
           "Batch": "rgcsr_batch", "XWindow": "rgcsr_xwindow", "CheckReport": "rgcsr_check_report"}


def declared_structs():
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return sorted(set(re.findall(r"\}\s*([a-z_][a-z0-9_]*)\s*;", src)))


def test_every_header_struct_has_a_binding():
    assert sorted(STRUCTS.values()) == declared_structs()


def test_struct_layouts_match_the_header(tmp_path):
    """Compiles a host program against the header that prints sizeof and
    offsetof of every field the binding declares; a field added, dropped or
    reordered on either side changes one of them."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "rgcsr.h"', "int main(void) {"]
    expected = []
    for py, c in STRUCTS.items():
        cls = getattr(L, py)
        lines.append(f'printf("%zu\\n", sizeof({c}));')
        expected.append(ctypes.sizeof(cls))
        for name, _ in cls._fields_:
            lines.append(f'printf("%zu\\n", offsetof({c}, {name}));')
            expected.append(getattr(cls, name).offset)
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c11", "-I", B.INCLUDE, str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got == expected


def test_c_program_links_against_the_library(tmp_path, lib):
    """A plain C program (no C++ runtime, no CUDA headers) compiles against
    the header, links against librgcsr.so and calls its host-only entry
    points, with the same answers as the binding gets."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    src = tmp_path / "use.c"
    src.write_text("\n".join([
        "#include <stdio.h>",
        '#include "rgcsr.h"',
        "int main(void) {",
        '    printf("%d\\n", rgcsr_version());',
        '    printf("%zu\\n", rgcsr_plan_workspace_bytes(1000000, 32));',
        '    printf("%s\\n", rgcsr_status_string(RGCSR_ERR_COL_OOB));',
        "    return 0;",
        "}", ""]))
    exe = tmp_path / "use"
    libdir = os.path.dirname(B.LIB_PATH)
    r = subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", B.INCLUDE, str(src), "-o", str(exe),
                        "-L", libdir, "-lrgcsr", f"-Wl,-rpath,{libdir}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()
    assert int(out[0]) == lib.rgcsr_version()
    assert int(out[1]) == lib.rgcsr_plan_workspace_bytes(1_000_000, 32)
    assert out[2] == lib.rgcsr_status_string(L.RGCSR_ERR_COL_OOB).decode()
