"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/pv3d.h; the Python binding's structs match the C layout."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_1410_5780_gb300 import build as B
from paper_1410_5780_gb300 import pv3d

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pv3d.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pv3d_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc") and not os.path.exists(B.LIB):
        pytest.skip("no nvcc and no prebuilt library")
    B.build()
    return pv3d.load()


def test_header_declares_the_abi():
    names = declared_functions()
    assert set(names) == set(pv3d.EXPORTED), names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (pv3d_[a-z_]+)", out))
    assert exported == set(declared_functions())


def test_struct_layouts_match_c(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    prog = tmp_path / "sz.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "pv3d.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(pv3d_opts), '
                    'sizeof(pv3d_module), sizeof(pv3d_layout), sizeof(pv3d_tracker), sizeof(pv3d_eval_opts), '
                    'sizeof(pv3d_result), offsetof(pv3d_eval_opts, stream), offsetof(pv3d_result, tests));'
                    'printf("%zu %zu\\n", sizeof(pv3d_profile), offsetof(pv3d_profile, sample_tests));'
                    'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), str(prog), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    exp = [ctypes.sizeof(pv3d.pv3d_opts), ctypes.sizeof(pv3d.pv3d_module), ctypes.sizeof(pv3d.pv3d_layout),
           ctypes.sizeof(pv3d.pv3d_tracker), ctypes.sizeof(pv3d.pv3d_eval_opts), ctypes.sizeof(pv3d.pv3d_result),
           pv3d.pv3d_eval_opts.stream.offset, pv3d.pv3d_result.tests.offset,
           ctypes.sizeof(pv3d.pv3d_profile), pv3d.pv3d_profile.sample_tests.offset]
    assert got == exp


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(pv3d, "_lib", None)
    monkeypatch.setattr(B, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        pv3d.load()


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1410_5780_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "pv3d_oracle" not in text, f


def test_noalloc_wrapper_rejects_bad_buffers():
    """The binding checks the buffers of pv3d_module_shade_noalloc before the
    call: the kernels read 9 float32 per triangle and write cells_u * cells_v
    32-bit counts, so host, wrong-dtype, non-contiguous or short tensors are
    refused with ValueError (the checks run before any device access)."""
    import torch
    module = dict(origin=(0.0, 0.0, 0.0), u=(1.0, 0.0, 0.0), v=(0.0, 1.0, 0.0), pitch=0.156, cells_u=6,
                  cells_v=10)
    tri = torch.zeros(4, 9, dtype=torch.float32)
    counts = torch.zeros(60, dtype=torch.int32)
    with pytest.raises(ValueError):
        pv3d.pv3d_module_shade_noalloc(tri, module, (0.0, 0.0, 1.0), 2, 256, counts)  # host tensors
    with pytest.raises(ValueError):
        pv3d.pv3d_module_shade_noalloc(tri.half(), module, (0.0, 0.0, 1.0), 2, 256, counts)
    with pytest.raises(ValueError):
        pv3d.pv3d_module_shade_noalloc(tri.t(), module, (0.0, 0.0, 1.0), 2, 256, counts)
    with pytest.raises(ValueError):
        pv3d.pv3d_module_shade_noalloc(tri, module, (0.0, 0.0, 1.0), 2, 256, counts[:10])
