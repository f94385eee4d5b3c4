"""CPU-side checks of the C ABI: the library builds, loads and exports every
entry point that include/emri_fd.h declares; pure host-side argument checks
return their status codes without touching a device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "emri_fd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(emri_fd_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    from paper_2307_12585_gb300 import api, build
    build.build()
    return api.lib()


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert set(names) >= {"emri_fd_plan", "emri_fd_sum_modes", "emri_fd_sync", "emri_fd_stats",
                          "emri_fd_plan_destroy", "emri_fd_strerror"}
    for nme in names:
        assert hasattr(L, nme), nme


def test_binding_names_match_header():
    from paper_2307_12585_gb300 import api
    for nme in _declared():
        assert hasattr(api, nme), nme


def test_strerror_and_null_arguments(L):
    from paper_2307_12585_gb300 import api
    for code in range(11):
        assert L.emri_fd_strerror(code)
    assert L.emri_fd_plan(None, None, None) == 1            # EMRI_FD_ERR_ARG, no device touched
    h = C.c_void_p()
    d = api.emri_fd_desc()
    d.precision = 7
    assert L.emri_fd_plan(C.byref(h), C.byref(d), None) == 1
    assert L.emri_fd_sync(None) == 1
    assert L.emri_fd_sum_modes(None, 1, *[None] * 18) == 1
    L.emri_fd_plan_destroy(None)


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2307_12585_gb300")
    for fn in os.listdir(pkg):
        if fn.endswith(".py"):
            src = open(os.path.join(pkg, fn)).read()
            assert not re.search(r"^\s*(from\s+oracle|import\s+oracle)", src, flags=re.M), fn
    for fn in os.listdir(os.path.join(pkg, "csrc")):
        assert "oracle" not in open(os.path.join(pkg, "csrc", fn)).read(), fn


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2307_12585_gb300 import api
    monkeypatch.setattr(api, "_lib", None)
    monkeypatch.setattr(api, "library_path", lambda: str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError):
        api.lib()
