"""CPU checks of the C ABI boundary: the library builds for sm_103a, loads,
and exports every entry point include/*.h declares; the product code never
reaches the oracle."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    inc = os.path.join(ROOT, "include")
    names = set()
    for fn in sorted(os.listdir(inc)):
        if fn.endswith(".h"):
            txt = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, fn)).read(), flags=re.S)
            names.update(re.findall(r"\b(kitc_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def libkitc():
    from paper_1902_02250_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_four_calls():
    names = _declared()
    for n in ("kitc_build_tree", "kitc_modified_weights", "kitc_evaluate", "kitc_direct"):
        assert n in names


def test_library_exports_every_declared_symbol(libkitc):
    for name in _declared():
        assert hasattr(libkitc, name), name


def test_binding_lists_every_declared_symbol():
    from paper_1902_02250_gb300 import kitc
    assert sorted(kitc.SYMBOLS) == _declared()


def test_status_strings_without_gpu(libkitc):
    libkitc.kitc_status_string.restype = ctypes.c_char_p
    assert libkitc.kitc_status_string(0) == b"ok"
    assert libkitc.kitc_status_string(4) == b"device-side wait timed out"
    assert libkitc.kitc_kernel_win(2) == 6 and libkitc.kitc_kernel_wout(1) == 6
    assert libkitc.kitc_kernel_win(7) == -1


def test_product_code_does_not_touch_the_oracle():
    pkg = os.path.join(ROOT, "paper_1902_02250_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, fn)).read()
                assert not re.search(r"\bimport\s+oracle|from\s+oracle|kitc_oracle|or_tree", txt), fn


def test_build_is_for_sm_103a_only():
    from paper_1902_02250_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_binding_raises_without_the_library(tmp_path, monkeypatch):
    """No CPU fallback: without the built library every call fails loudly."""
    from paper_1902_02250_gb300 import build, kitc
    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing" / "libkitc.so"))
    monkeypatch.setattr(kitc, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        kitc.lib()
