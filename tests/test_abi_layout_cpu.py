"""The ctypes binding agrees with include/emri_fd.h.  A small C program compiled
against the header prints the descriptor's size and field offsets and the values
of the status, precision, SPA-form and window enums, and the binding's
definitions must match them; and every prototype, parsed from the preprocessed
header, matches the binding's argtypes and restype.  CPU only (gcc, no CUDA)."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_2307_12585_gb300 import api

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FIELDS = [f[0] for f in api.emri_fd_desc._fields_]
STATUS_NAMES = [api.STATUS[k] for k in sorted(api.STATUS)]

PROBE = r"""
#include <stdio.h>
#include <stddef.h>
#include "emri_fd.h"
int main(void) {
  printf("sizeof %zu\n", sizeof(emri_fd_desc));
@OFFSETS@
@STATUS@
  printf("EMRI_FD_FP64 %d\nEMRI_FD_MIXED %d\nEMRI_FD_FP64X %d\n", EMRI_FD_FP64, EMRI_FD_MIXED, EMRI_FD_FP64X);
  printf("EMRI_FD_SPA_STANDARD %d\nEMRI_FD_SPA_EXTENDED %d\n", EMRI_FD_SPA_STANDARD, EMRI_FD_SPA_EXTENDED);
  printf("EMRI_FD_WINDOW_NONE %d\nEMRI_FD_WINDOW_HANN %d\n", EMRI_FD_WINDOW_NONE, EMRI_FD_WINDOW_HANN);
  return 0;
}
"""


@pytest.fixture(scope="module")
def header_values(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    d = tmp_path_factory.mktemp("abi")
    offs = "\n".join('  printf("off_%s %%zu\\n", offsetof(emri_fd_desc, %s));' % (f, f) for f in FIELDS)
    stats = "\n".join('  printf("%s %%d\\n", (int)%s);' % (n, n) for n in STATUS_NAMES)
    src = d / "probe.c"
    src.write_text(PROBE.replace("@OFFSETS@", offs).replace("@STATUS@", stats))
    exe = d / "probe"
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                           "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True)
    return {k: int(v) for k, v in (line.split() for line in out.strip().splitlines())}


def test_descriptor_layout(header_values):
    assert header_values["sizeof"] == C.sizeof(api.emri_fd_desc)
    for f in FIELDS:
        assert header_values["off_" + f] == getattr(api.emri_fd_desc, f).offset, f


def test_enum_values(header_values):
    for code, name in api.STATUS.items():
        assert header_values[name] == code, name
    assert (header_values["EMRI_FD_FP64"], header_values["EMRI_FD_MIXED"], header_values["EMRI_FD_FP64X"]) == \
        (api.EMRI_FD_FP64, api.EMRI_FD_MIXED, api.EMRI_FD_FP64X)
    assert header_values["EMRI_FD_SPA_STANDARD"] == api.SPA_FORMS["standard"]
    assert header_values["EMRI_FD_SPA_EXTENDED"] == api.SPA_FORMS["extended"]
    assert header_values["EMRI_FD_WINDOW_NONE"] == api.WINDOWS[None]
    assert header_values["EMRI_FD_WINDOW_HANN"] == api.WINDOWS["hann"]


def _c_kind(node):
    """Class of a pycparser type node: "ptr", "int", "ll", "double", "void"."""
    from pycparser import c_ast
    if isinstance(node, c_ast.PtrDecl):
        return "ptr"
    if isinstance(node, c_ast.TypeDecl) and isinstance(node.type, c_ast.IdentifierType):
        names = node.type.names
        if names in (["emri_fd_plan_t"], ["emri_fd_graph_t"]):
            return "ptr"   # typedefs of pointers
        if names in (["int"], ["emri_fd_status"]):
            return "int"
        if names == ["long", "long"]:
            return "ll"
        if names == ["double"]:
            return "double"
        if names == ["void"]:
            return "void"
    raise AssertionError("unhandled type %r" % node)


def _ctypes_kind(t):
    if t is None:
        return "void"
    if t in (C.c_void_p, C.c_char_p) or (isinstance(t, type) and issubclass(t, C._Pointer)):
        return "ptr"
    return {C.c_int: "int", C.c_longlong: "ll", C.c_double: "double"}[t]


def test_function_signatures_match_argtypes():
    """Every exported prototype in the header against the binding's argtypes and
    restype, parameter by parameter (pointer / int / long long / double)."""
    pycparser = pytest.importorskip("pycparser")
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    try:
        L = api.lib()
    except (OSError, RuntimeError) as e:
        pytest.skip("library not built: %s" % e)
    text = subprocess.check_output(["gcc", "-E", "-P", "-std=c11", os.path.join(ROOT, "include", "emri_fd.h")],
                                   text=True)
    ast = pycparser.CParser().parse(text)
    protos = {}
    for ext in ast.ext:
        if type(ext).__name__ == "Decl" and type(ext.type).__name__ == "FuncDecl":
            f = ext.type
            params = [] if f.args is None else [p.type for p in f.args.params]
            if len(params) == 1 and _c_kind(params[0]) == "void":
                params = []
            protos[ext.name] = (_c_kind(f.type), [_c_kind(p) for p in params])
    assert set(protos) == set(api.EXPORTS)
    for name, (ret, params) in protos.items():
        fn = getattr(L, name)
        assert [_ctypes_kind(t) for t in fn.argtypes] == params, name
        assert _ctypes_kind(fn.restype) == ret, name
