"""The C-ABI library builds for sm_103a, loads, and exports every symbol of include/polfed.h.

No compute calls: this runs without a GPU.
"""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "polfed.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(polfed_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2005_09534_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = header_symbols()
    for name in ["polfed_basis_build", "polfed_h_apply", "polfed_cheb_filter", "polfed_block_lanczos",
                 "polfed_eigs", "polfed_ctx_create", "polfed_ctx_destroy", "polfed_last_error"]:
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    for name in header_symbols():
        assert hasattr(lib, name), name


def test_binding_loads_and_reports_errors_without_gpu(lib):
    import paper_2005_09534_gb300 as pf
    pf.load()
    o = pf.opts_default()
    assert abs(o.p - 0.17) < 1e-15 and o.precision == pf.DF64
    # dimension query touches no device memory
    assert pf.basis_build(22, 11) == 705432
    assert pf.basis_build(24, 12) == 2704156
    with pytest.raises(pf.PolfedError) as e:
        pf.basis_build(33, 1)
    assert e.value.code == pf.POLFED_EINVAL


def test_struct_layouts_match_header(tmp_path):
    """Every field of the ctypes mirrors sits at the offset the C compiler gives it."""
    import subprocess
    import paper_2005_09534_gb300 as pf
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    structs = [("polfed_model", pf.CModel), ("polfed_opts", pf.COpts), ("polfed_stats", pf.CStats),
               ("polfed_batch_info", pf.CBatchInfo), ("polfed_counters", pf.CCounters),
               ("polfed_conv_point", pf.CConvPoint)]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "polfed.h"', "int main(void) {"]
    for cname, cls in structs:
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                 text=True).stdout.splitlines())
    for cname, cls in structs:
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(cls, f).offset, f"{cname}.{f}"
