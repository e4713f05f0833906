"""The C-ABI library loads and exports every entry point that include/*.h declares (no device
work), and host-side argument checks reject bad calls without touching a GPU."""
import ctypes as C
import glob
import os
import re

import pytest

from paper_2307_14302_gb300 import build as B
from paper_2307_14302_gb300 import dgswe as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(?:int|void|int64_t|const\s+char\s*\*)\s+(dgswe_\w+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    B.build()
    return D.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 25
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert set(D.EXPORTS) == names


def test_host_side_errors_without_device_work(lib):
    h = C.c_void_p()
    rc = lib.dgswe_create(None, 0, None)
    assert rc == -1 and b"null" in lib.dgswe_last_error()
    rc = lib.dgswe_set_params(None, None)
    assert rc == -1
    assert lib.dgswe_launch_count(None) == 0
    lib.dgswe_destroy(None)  # NULL is ignored
    import torch
    if not torch.cuda.is_available():
        rc = lib.dgswe_create(C.byref(h), 0, None)
        assert rc == -8 and h.value is None  # ENOLIB: no device here
        with pytest.raises(D.DgsweError) as ei:
            D.Solver()
        assert ei.value.code == -8


def test_binding_fails_loudly_when_library_missing(monkeypatch, tmp_path):
    monkeypatch.setattr(D, "LIB_PATH", str(tmp_path / "libdgswe.so"))
    monkeypatch.setattr(D, "_lib", None)
    with pytest.raises(D.DgsweUnavailable):
        D.lib()


def test_every_declaration_names_its_passage():
    """Each entry point's own comment names the passage of the paper that defines what it does
    (a section or equation), or says that the paper has no counterpart."""
    src = open(os.path.join(ROOT, "include", "dgswe.h")).read()
    documented = {}
    for m in re.finditer(r"(/\*(?:.|\n)*?\*/)\s*(?:int|void|int64_t|const\s+char\s*\*)\s+(dgswe_\w+)\s*\(", src):
        documented[m.group(2)] = m.group(1)
    assert set(documented) == _declared()
    for name, comment in documented.items():
        assert re.search(r"Sec\. \d|Eq\. \w|no counterpart in the paper|paper has no counterpart", comment, re.I), name
