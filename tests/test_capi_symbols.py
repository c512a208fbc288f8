"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function include/expdg.h declares.  No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "expdg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(expdg_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2011_01316_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("expdg_create", "expdg_destroy", "expdg_residual", "expdg_jv", "expdg_phi",
                     "expdg_step", "expdg_advance", "expdg_last_error", "expdg_set_stream"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    from paper_2011_01316_gb300 import expdg
    assert "sm_103a" in expdg.version()
    cfg = expdg.default_config()
    assert cfg.dim == 2 and cfg.p == 4 and cfg.eq == expdg.EXPDG_EULER
    assert cfg.m_max <= 64 and cfg.krylov_tol == 1e-10


def test_binding_matches_header_structs():
    """The ctypes mirrors of the C structs have the field order of the header."""
    from paper_2011_01316_gb300 import expdg
    text = open(HEADER).read()
    body = text[text.index("typedef struct {\n  int dim;"):text.index("} expdg_config;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = re.findall(r"\b([a-z_0-9]+)(?:\[3\])?[,;]", body)
    fields = [f for f, _ in expdg.expdg_config._fields_]
    assert [n for n in names if n in fields] == fields


def test_binding_constants_match_header():
    from paper_2011_01316_gb300 import expdg
    text = open(HEADER).read()
    for name in ("EXPDG_MAX_ORDER", "EXPDG_MAX_KRYLOV", "EXPDG_MAX_PHI", "EXPDG_MAX_IOP"):
        m = re.search(r"#define\s+" + name + r"\s+(\d+)", text)
        assert m, name
        assert getattr(expdg, name) == int(m.group(1)), name


def test_config_layout_matches_c(tmp_path):
    """sizeof and field offsets of expdg_config as the C compiler lays it out
    equal the ctypes mirror's (host C compiler, no GPU)."""
    import shutil
    import subprocess
    from paper_2011_01316_gb300 import expdg
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    fields = [f for f, _ in expdg.expdg_config._fields_]
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "expdg.h"\nint main(void) {\n'
                   '  printf("%zu\\n", sizeof(expdg_config));\n'
                   + "".join(f'  printf("%zu\\n", offsetof(expdg_config, {f}));\n' for f in fields)
                   + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert out[0] == ctypes.sizeof(expdg.expdg_config)
    assert out[1:] == [getattr(expdg.expdg_config, f).offset for f in fields]
