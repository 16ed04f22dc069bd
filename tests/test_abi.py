"""The C-ABI library builds, loads without a GPU, and exports every function
include/exact.h declares; the Python binding's struct layouts match the C
ones (checked with gcc's offsetof)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "exact.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*[a-z_][a-z_ *]*?\b(exact_[a-z_0-9]+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("exact_plan_create", "exact_forward", "exact_adjoint", "exact_operator", "exact_solve",
                     "exact_norm_estimate", "exact_plan_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_2503_19925_gb300 as ex
    lib = ex.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    from paper_2503_19925_gb300.exact import _SIGS
    bound = {n for n, _, _ in _SIGS}
    assert set(declared_functions()) <= bound
    assert lib.exact_status_string(0) == b"ok"


def test_struct_layouts_match(tmp_path):
    from paper_2503_19925_gb300 import exact as b
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "exact.h"\n'
                   'int main(void){\n'
                   'printf("%zu %zu %zu %zu\\n", sizeof(exact_geometry), offsetof(exact_geometry, pixel),'
                   ' offsetof(exact_geometry, n_bins), offsetof(exact_geometry, src_to_det));\n'
                   'printf("%zu %zu %zu %zu %zu\\n", sizeof(exact_solve_opts), offsetof(exact_solve_opts, average_tail),'
                   ' offsetof(exact_solve_opts, history), offsetof(exact_solve_opts, tv_bound),'
                   ' offsetof(exact_solve_opts, tv));\n'
                   'printf("%zu %zu %zu %zu %zu\\n", offsetof(exact_solve_opts, prox_lambda),'
                   ' offsetof(exact_solve_opts, t0), offsetof(exact_solve_opts, resume),'
                   ' offsetof(exact_solve_opts, x_last), offsetof(exact_solve_opts, launch));\n'
                   'printf("%zu %zu %zu\\n", sizeof(exact_solve_info), offsetof(exact_solve_info, status),'
                   ' offsetof(exact_solve_info, avg_change));\n'
                   'printf("%zu %zu\\n", sizeof(exact_spectrum), sizeof(exact_windows));\n'
                   'printf("%zu %zu %zu %zu\\n", sizeof(exact_job), offsetof(exact_job, opts), offsetof(exact_job, x),'
                   ' offsetof(exact_job, info));\n'
                   'printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(exact_tv_opts), offsetof(exact_tv_opts, tol_tv),'
                   ' offsetof(exact_tv_opts, lam0), sizeof(exact_tv_info), offsetof(exact_tv_info, lam),'
                   ' offsetof(exact_tv_info, status));\n'
                   'return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    g = [int(v) for v in out[0].split()]
    assert g == [ctypes.sizeof(b._Geometry), b._Geometry.pixel.offset, b._Geometry.n_bins.offset,
                 b._Geometry.src_to_det.offset]
    o = [int(v) for v in out[1].split()]
    assert o == [ctypes.sizeof(b._SolveOpts), b._SolveOpts.average_tail.offset, b._SolveOpts.history.offset,
                 b._SolveOpts.tv_bound.offset, b._SolveOpts.tv.offset]
    assert [int(v) for v in out[2].split()] == [b._SolveOpts.prox_lambda.offset, b._SolveOpts.t0.offset,
                                                 b._SolveOpts.resume.offset, b._SolveOpts.x_last.offset,
                                                 b._SolveOpts.launch.offset]
    out = out[:2] + out[3:]
    i = [int(v) for v in out[2].split()]
    assert i == [ctypes.sizeof(b._SolveInfo), b._SolveInfo.status.offset, b._SolveInfo.avg_change.offset]
    s = [int(v) for v in out[3].split()]
    assert s == [ctypes.sizeof(b._Spectrum), ctypes.sizeof(b._Windows)]
    jv = [int(v) for v in out[4].split()]
    assert jv == [ctypes.sizeof(b._Job), b._Job.opts.offset, b._Job.x.offset, b._Job.info.offset]
    tv = [int(v) for v in out[5].split()]
    assert tv == [ctypes.sizeof(b._TvOpts), b._TvOpts.tol_tv.offset, b._TvOpts.lam0.offset,
                  ctypes.sizeof(b._TvInfo), b._TvInfo.lam.offset, b._TvInfo.status.offset]


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2503_19925_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "exact_oracle" not in text and "liboracle" not in text, f
