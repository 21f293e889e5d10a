"""The C-ABI library builds, loads and exports every entry point declared in
include/fastcod.h; host-side argument checks that need no GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "fastcod.h")) as f:
        txt = f.read()
    return sorted(set(re.findall(r"FASTCOD_API\s+[\w\s\*]+?\b(fastcod_\w+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2302_09247_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("fastcod_create", "fastcod_set_volumes", "fastcod_add_streamlines", "fastcod_connectivity",
                 "fastcod_endpoint_connectivity", "fastcod_destroy"):
        assert want in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(lib, name), name
    # and nothing of the internals leaks into the dynamic symbol table
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    fastcod = {s for s in exported if s.startswith("fastcod_")}
    assert fastcod == set(_declared())


def test_binding_names_match_header(lib_path):
    from paper_2302_09247_gb300 import fastcod
    assert sorted(fastcod.EXPORTED) == _declared()
    for name in _declared():
        assert callable(getattr(fastcod, name))


def test_null_and_state_errors_without_gpu(lib_path):
    from paper_2302_09247_gb300 import fastcod as fc
    L = fc.lib
    assert L.fastcod_create(None, 0, 0) == fc.FASTCOD_EINVAL
    assert L.fastcod_destroy(None) == fc.FASTCOD_OK
    assert L.fastcod_set_volumes(None, None, None, 1, 1, 1, 0, 0) == fc.FASTCOD_EINVAL
    assert L.fastcod_add_streamlines(None, None, 0, None, 0) == fc.FASTCOD_EINVAL
    assert L.fastcod_get_shape(None, None, None) == fc.FASTCOD_EINVAL
    assert L.fastcod_restore(None, None, None, None) == fc.FASTCOD_EINVAL
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if not has_gpu:
        out = ctypes.c_void_p()
        assert L.fastcod_create(ctypes.byref(out), 0, 0) == fc.FASTCOD_EINVAL
        assert out.value is None
        assert fc.fastcod_last_error(None) != ""


def test_checked_build_exports_the_same_symbols(lib_path):
    # the bounds-checked variant (FASTCOD_CHECKED=1) builds and exports the
    # same boundary
    from paper_2302_09247_gb300 import build
    checked = build.build(checked=True)
    out = subprocess.run(["nm", "-D", "--defined-only", checked], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln and ln.split()[-1].startswith("fastcod_")}
    assert exported == set(_declared())
