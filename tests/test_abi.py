"""CPU checks of the C ABI: the library builds, loads and exports every declared entry point.

No compute call is made here (there is no GPU in the CPU test environment).
"""
import ctypes
import os
import re

import pytest

from paper_1503_03004_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include"))) if f.endswith(".h")]


def _declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(sfr_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    if not os.path.exists(binding.LIB_PATH):
        from paper_1503_03004_gb300 import build_lib
        build_lib.build()
    return binding.LIB_PATH


def test_header_declares_the_boundary():
    names = _declared_functions()
    for n in ("sfr_create", "sfr_solve", "sfr_submit", "sfr_poll", "sfr_destroy", "sfr_last_error", "sfr_version"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for n in _declared_functions():
        assert hasattr(lib, n), n


def test_binding_signatures_cover_the_header():
    bound = {name for name, _, _ in binding.SIGNATURES}
    assert set(_declared_functions()) <= bound


def test_struct_layouts_match_the_header():
    # field order and sizes of the ctypes mirrors against the C declarations
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "sfr.h")).read(), flags=re.S)
    for struct, py in (("sfr_config", binding.Config), ("sfr_problem", binding.Problem), ("sfr_result", binding.Result),
                       ("sfr_kernel_stat", binding.KernelStat), ("sfr_opt_full_problem", binding.OptFullProblem),
                       ("sfr_opt_full_result", binding.OptFullResult)):
        body = re.search(r"typedef struct \{([^}]*)\}\s*" + struct + ";", text).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            for part in decl.split(","):
                fields.append(re.findall(r"[A-Za-z_][A-Za-z0-9_]*", part)[-1])
        assert fields == [f for f, _ in py._fields_], struct


def test_version_string(libpath):
    lib = binding.load(libpath)
    assert lib.sfr_version().decode().startswith("libsfr")


def test_create_without_a_gpu_fails_cleanly(libpath):
    # On a machine without a usable GPU, sfr_create must return an error code, not crash.
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = binding.load(libpath)
    h = ctypes.c_void_p()
    cfg = binding.Config(device=0, hbm_budget_bytes=0, max_slots=0, cuda_stream=None)
    st = lib.sfr_create(ctypes.byref(h), ctypes.byref(cfg))
    assert st < 0
    assert lib.sfr_last_error(None)


def test_struct_offsets_match_the_c_compiler(tmp_path):
    # the ctypes mirrors' sizes and field offsets against what a C compiler lays out for the header
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = (("sfr_config", binding.Config), ("sfr_problem", binding.Problem), ("sfr_result", binding.Result),
               ("sfr_kernel_stat", binding.KernelStat), ("sfr_opt_full_problem", binding.OptFullProblem),
               ("sfr_opt_full_result", binding.OptFullResult))
    lines = ['#include <stdio.h>', '#include "sfr.h"', "int main(void) {"]
    for name, py in structs:
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = str(tmp_path / "layout")
    r = subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", exe],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    got = {}
    for line in subprocess.run([exe], capture_output=True, text=True, timeout=60).stdout.splitlines():
        parts = line.split()
        got[(parts[0], parts[1])] = int(parts[-1])
    for name, py in structs:
        assert got[(name, "size")] == ctypes.sizeof(py), name
        for f, _ in py._fields_:
            assert got[(name, f)] == getattr(py, f).offset, (name, f)
