"""The C ABI library builds for sm_103a, loads, and exports every entry point that
include/rs_gb300.h declares (no GPU needed: no compute call is made)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"\b(rs_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2412_18629_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_four_calls():
    names = _declared()
    for n in ("rs_fof3d", "rs_fof6d", "rs_unbind", "rs_halo_props"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2412_18629_gb300 as rs
    monkeypatch.setattr(rs, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(rs, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        rs.load_library()


def test_invalid_config_is_rejected(lib):
    import paper_2412_18629_gb300 as rs
    cfg = rs.rs_config()
    cfg.box_L, cfg.link_len = -1.0, 0.2
    h = ctypes.c_void_p()
    lib.rs_ctx_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(rs.rs_config),
                                  ctypes.c_int]
    assert lib.rs_ctx_create(ctypes.byref(h), ctypes.byref(cfg), 0) == 1  # RS_ERR_INVALID_ARG


def _c_layout(tmp_path, struct, fields):
    """sizeof and offsetof of a header struct, from a C program compiled with gcc."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    body = "".join(f'  printf("%zu\\n", offsetof({struct}, {f}));\n' for f in fields)
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "rs_gb300.h"\n'
                   f'int main(void) {{\n  printf("%zu\\n", sizeof({struct}));\n{body}  return 0;\n}}\n')
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True,
                                           text=True).stdout.split()]
    return vals[0], vals[1:]


@pytest.mark.parametrize("name", ("rs_config", "rs_snapshot"))
def test_ctypes_structs_match_the_header(tmp_path, name):
    import paper_2412_18629_gb300 as rs
    cls = getattr(rs, name)
    fields = [f[0] for f in cls._fields_]
    size, offs = _c_layout(tmp_path, name, fields)
    assert ctypes.sizeof(cls) == size
    assert [getattr(cls, f).offset for f in fields] == offs
