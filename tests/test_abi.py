"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/sign.h declares (no compute calls: runs without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sign.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sign_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2210_03356_gb300 import build
    lib = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (sign_\w+)", out))
    declared = _declared()
    assert declared, "no functions found in include/sign.h"
    missing = [d for d in declared if d not in exported]
    assert not missing, missing


def test_binding_covers_header_and_loads():
    import paper_2210_03356_gb300 as sg
    from paper_2210_03356_gb300 import _native
    assert sorted(_native.SIGNATURES) == _declared()
    sg.load()
    o = sg.default_opts()
    assert (o.tol, o.filter, o.c4, o.switch_resid, o.max_iter) == (1e-8, 1, 1e-4, 1e-6, 100)
    assert (o.prec, o.fp32_until, o.scale_1norm, o.dense_frac, o.dense64_min_n) == (0, 1e-4, 1, 0.25, 1024)
    assert (o.fp32_band, o.filter_t, o.budget_norm, o.method) == (1, 0, 0, 0)
    assert (o.band_min_eff, o.group_margin, o.pair_rows) == (0.08, 0.05, 1)
    assert sg.last_error() == ""


def test_library_is_built_for_sm103a_only():
    from paper_2210_03356_gb300 import build
    lib = build.build()
    out = subprocess.run(["cuobjdump", "--list-elf", lib], capture_output=True, text=True).stdout
    arches = set(re.findall(r"sm_(\d+a?)", out))
    assert arches == {"103a"}, arches


def test_no_oracle_on_the_product_path():
    """The package never imports the oracle and has no CPU compute fallback."""
    pkg = os.path.join(ROOT, "paper_2210_03356_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "oracle.h" not in text, f


def test_missing_library_fails_loudly(tmp_path):
    from paper_2210_03356_gb300 import _native
    saved = _native._lib
    try:
        _native._lib = None
        with pytest.raises(RuntimeError):
            _native.load(str(tmp_path / "nope.so"))
    finally:
        _native._lib = saved


def _prototypes():
    """{name: (return type, parameter count)} of every function in include/sign.h."""
    src = open(os.path.join(ROOT, "include", "sign.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    protos = {}
    for ret, name, params in re.findall(r"([A-Za-z_][\w\s\*]*?)\s*\b(sign_[a-z0-9_]+)\s*\(([^)]*)\)\s*;",
                                        src):
        params = " ".join(params.split())
        count = 0 if params in ("", "void") else params.count(",") + 1
        protos[name] = (" ".join(ret.split()), count)
    return protos


def test_binding_arity_and_return_types_match_the_header():
    """Each ctypes signature takes as many arguments as the C prototype and
    returns the same kind of value (a wrong count would corrupt the call)."""
    import ctypes as C
    from paper_2210_03356_gb300 import _native
    protos = _prototypes()
    assert sorted(protos) == _declared()
    kinds = {"void": None, "sign_status": C.c_int, "int": C.c_int, "int64_t": C.c_int64,
             "double": C.c_double, "const char *": C.c_char_p}
    for name, (ret, count) in protos.items():
        restype, argtypes = _native.SIGNATURES[name]
        assert len(argtypes) == count, (name, len(argtypes), count)
        assert restype is kinds[ret], (name, ret, restype)
