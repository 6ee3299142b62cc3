"""The C-ABI library loads and exports every entry point include/awe.h
declares, and the binding covers exactly those (no compute calls: CPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "awe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(awe_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libawe():
    from paper_2211_13295_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_library_exports_every_declared_symbol(libawe):
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(libawe, n), n


def test_binding_covers_the_header():
    from paper_2211_13295_gb300 import awe
    assert sorted(awe.exported_symbols()) == declared_symbols()


def test_config_struct_layout_matches_header(libawe):
    """The ctypes mirror of awe_config has the C layout: compile a probe of
    offsetof() with the header and compare."""
    import subprocess
    import tempfile
    from paper_2211_13295_gb300.awe import AweConfig
    fields = [f[0] for f in AweConfig._fields_]
    code = "#include <stdio.h>\n#include <stddef.h>\n#include \"awe.h\"\nint main(){"
    code += "".join(f'printf("%zu\\n", offsetof(awe_config, {f}));' for f in fields)
    code += 'printf("%zu\\n", sizeof(awe_config)); return 0;}'
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        open(c, "w").write(code)
        exe = os.path.join(d, "p")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = [int(x) for x in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    assert out[:-1] == [getattr(AweConfig, f).offset for f in fields]
    assert out[-1] == ctypes.sizeof(AweConfig)


def test_binding_fails_loudly_without_the_library(tmp_path, monkeypatch):
    from paper_2211_13295_gb300 import awe
    monkeypatch.setattr(awe, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(awe, "_lib", None)
    with pytest.raises(RuntimeError):
        awe.lib()
