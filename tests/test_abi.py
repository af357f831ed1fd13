"""The C ABI library builds, loads and exports what include/*.h declare.

These tests run without a GPU: they launch no compute.  Calls that need a
device must fail cleanly with a status code.
"""
import ctypes
import os
import re

import pytest

import paper_1705_09366_gb300 as pkg
from paper_1705_09366_gb300 import build as pkg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libstkde():
    pkg_build.build()
    return pkg.lib()


def declared_symbols():
    inc = os.path.join(ROOT, "include")
    text = ""
    for name in sorted(os.listdir(inc)):
        if name.endswith(".h"):
            with open(os.path.join(inc, name)) as f:
                text += f.read()
    return sorted(set(re.findall(r"STKDE_API\s+[\w\s\*]*?\b(stkde_\w+)\s*\(", text)))


def exported_symbols(path):
    import subprocess
    r = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                       check=True)
    return sorted({ln.split()[-1] for ln in r.stdout.splitlines() if " T " in ln})


def test_header_declares_the_boundary():
    names = declared_symbols()
    assert set(names) == set(pkg.EXPORTED_SYMBOLS)


def test_library_exports_every_declared_symbol(libstkde):
    exported = exported_symbols(pkg.lib_path)
    for name in declared_symbols():
        assert name in exported, name
        assert hasattr(libstkde, name)
    # nothing but the C ABI is exported
    assert all(s.startswith("stkde_") for s in exported), exported


def test_status_strings(libstkde):
    assert pkg.stkde_status_string(0) == "ok"
    assert "invalid" in pkg.stkde_status_string(1)
    assert pkg.stkde_status_string(99) == "unknown status"


def test_default_options(libstkde):
    o = pkg.stkde_default_options()
    assert o.form == pkg.FORM_TENSOR_BF16X3
    assert o.kernel_constants == pkg.KERNEL_PRINTED
    assert o.device == 0 and not o.stream and o.profile == 0


def test_null_arguments_are_rejected_without_a_device(libstkde):
    g = pkg.make_grid(4, 4, 4)
    assert libstkde.stkde_compute(None, None, 0, ctypes.byref(g), 1.0, 1.0, None) == pkg.ERR_INVALID_ARGUMENT
    assert libstkde.stkde_create(None, None) == pkg.ERR_INVALID_ARGUMENT
    assert libstkde.stkde_synchronize(None) == pkg.ERR_INVALID_ARGUMENT
    assert libstkde.stkde_phase_times(None, None, 0) == 0
    assert libstkde.stkde_reserve(None, 1 << 20) == pkg.ERR_INVALID_ARGUMENT
    assert libstkde.stkde_inject_fault(None, pkg.FAULT_ALLOC, 1) == pkg.ERR_INVALID_ARGUMENT
    libstkde.stkde_destroy(None)


def test_bad_options_are_rejected(libstkde):
    h = ctypes.c_void_p()
    o = pkg.stkde_default_options()
    o.form = 17
    assert libstkde.stkde_create(ctypes.byref(h), ctypes.byref(o)) == pkg.ERR_INVALID_ARGUMENT
    for tb in (24, 64):  # reserved field: only 0 is accepted
        o = pkg.stkde_default_options()
        o.t_block = tb
        assert libstkde.stkde_create(ctypes.byref(h), ctypes.byref(o)) == pkg.ERR_INVALID_ARGUMENT


def test_create_without_gpu_fails_cleanly(libstkde):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = libstkde.stkde_create(ctypes.byref(h), None)
    assert st in (pkg.ERR_UNSUPPORTED, pkg.ERR_CUDA, pkg.ERR_INVALID_ARGUMENT)
    assert not h.value


def test_binding_raises_without_library(tmp_path, monkeypatch):
    monkeypatch.setattr(pkg, "lib_path", str(tmp_path / "missing.so"))
    monkeypatch.setattr(pkg, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        pkg.lib()
