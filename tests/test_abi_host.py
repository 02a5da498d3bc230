"""CPU checks of the C-ABI library: it builds, loads without a GPU, exports every entry
point include/dog.h declares, and its host-side parameter validation and workspace sizing
behave as documented (no kernel is launched)."""
import ctypes as C
import os
import re

import pytest

from paper_1605_02406_b300 import build, native as N, scene

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return N.lib()


def declared_symbols():
    hdr = ""
    for name in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if name.endswith(".h"):
            hdr += open(os.path.join(ROOT, "include", name)).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(dog_[a-z0-9_]+)\s*\(", hdr)))


def test_header_declarations_match_binding():
    assert declared_symbols() == sorted(N.SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_error_strings(lib):
    for code in [0, -1, -2, -3, -4, -5, -6, -7]:
        assert N.dog_error_string(code)
    assert N.dog_error_string(-99) == "unknown error"


def test_workspace_bytes_and_validation(lib):
    cfg = scene.CONFIGS["automotive_1024"]
    p = N.make_params(scene.filter_params(cfg))
    n = N.dog_workspace_bytes(p)
    # every particle array, the sort buffers and the cell arrays fit, and nothing absurd
    assert 4 * 16 * cfg["nu"] < n < 8 * 64 * cfg["nu"] + 256 * cfg["width"] * cfg["height"]
    small = N.make_params(scene.filter_params(scene.CONFIGS["plain_128"]))
    assert N.dog_workspace_bytes(small) < n
    bad = N.make_params(dict(scene.filter_params(cfg), p_S=1.5))
    with pytest.raises(N.DogError) as e:
        N.dog_workspace_bytes(bad)
    assert e.value.code == -1
    for w, h in [(8192, 4096), (4096, 4096)]:  # C = 2^25, and C = 2^24 just past the limit
        huge = N.make_params(dict(scene.filter_params(cfg), width=w, height=h))
        with pytest.raises(N.DogError) as e:
            N.dog_workspace_bytes(huge)
        assert e.value.code == -7
    assert N.dog_workspace_bytes(N.make_params(dict(scene.filter_params(cfg), width=4095, height=4096))) > 0
    zero = N.make_params(dict(scene.filter_params(cfg), nu=0))
    with pytest.raises(N.DogError):
        N.dog_workspace_bytes(zero)


def test_create_rejects_small_or_unaligned_workspace(lib):
    p = N.make_params(scene.filter_params(scene.CONFIGS["plain_128"]))
    n = N.dog_workspace_bytes(p)
    h = C.c_void_p()
    assert lib.dog_create(C.byref(p), C.c_void_p(256), n - 1, None, C.byref(h)) == -2
    assert lib.dog_create(C.byref(p), C.c_void_p(257), n, None, C.byref(h)) == -1
    assert lib.dog_create(C.byref(p), None, n, None, C.byref(h)) == -1
