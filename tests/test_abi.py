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


BAD_CONFIGS = {
    "dim": lambda c: setattr(c, "dim", 1),
    "order_high": lambda c: setattr(c, "order", 5),
    "order_low": lambda c: setattr(c, "order", 1),
    "gate_at_order_2": lambda c: (setattr(c, "order", 2), setattr(c, "gate", 1)),
    "prec": lambda c: setattr(c, "prec", 7),
    "too_few_zones": lambda c: c.n.__setitem__(1, 2),
    "empty_domain": lambda c: c.hi.__setitem__(0, c.lo[0]),
    "boundary": lambda c: c.bc.__setitem__(3, 99),
    "gamma": lambda c: setattr(c, "gamma", 1.0),
    "picard": lambda c: setattr(c, "picard", 9),
    "slab": lambda c: setattr(c, "slab", -1),
    "riemann": lambda c: setattr(c, "riemann", 9),
    "scheme": lambda c: setattr(c, "scheme", 5),
    "rk_stages": lambda c: (setattr(c, "scheme", 1), setattr(c, "rk_stages", 4)),
    "grid_too_large": lambda c: [c.n.__setitem__(d, 1 << 11) for d in range(3)],
}


@pytest.mark.parametrize("case", sorted(BAD_CONFIGS))
def test_create_rejects_a_bad_config_before_touching_the_device(libawe, case):
    """awe_create validates the whole configuration before any CUDA call, so
    every rejection (AWE_ERR_ARG with a message, no handle) runs on a machine
    without a GPU."""
    from paper_2211_13295_gb300 import awe
    from paper_2211_13295_gb300 import problems as P
    c = awe.make_config(P.tgv3d(n=8, order=4))
    BAD_CONFIGS[case](c)
    h = ctypes.c_void_p(1234)
    libawe.awe_last_error.restype = ctypes.c_char_p
    rc = libawe.awe_create(ctypes.byref(c), None, ctypes.byref(h))
    assert rc == -1
    assert h.value is None
    assert libawe.awe_last_error(None)


def test_create_reports_a_forced_allocation_failure(libawe, monkeypatch):
    """AWE_FAIL_ALLOC=1 makes awe_create fail as if the device allocation had
    (AWE_ERR_OOM, no handle), after the configuration checks, before any CUDA
    call: the out-of-memory path of a caller can be exercised without a GPU."""
    from paper_2211_13295_gb300 import awe
    from paper_2211_13295_gb300 import problems as P
    monkeypatch.setenv("AWE_FAIL_ALLOC", "1")
    c = awe.make_config(P.tgv3d(n=8, order=4))
    h = ctypes.c_void_p(1234)
    libawe.awe_last_error.restype = ctypes.c_char_p
    assert libawe.awe_create(ctypes.byref(c), None, ctypes.byref(h)) == -3
    assert h.value is None
    assert b"AWE_FAIL_ALLOC" in libawe.awe_last_error(None)
