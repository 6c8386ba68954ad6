"""The C-ABI library builds for sm_103a, loads, exports exactly what
include/rsnegf.h declares, and validates arguments on the host (no GPU
compute is issued in these tests)."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1401_0782_gb300 import binding, build
    path = build.build()
    return binding.load(path)


def _declared():
    src = open(os.path.join(ROOT, "include", "rsnegf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rsn_[a-z_]+)\s*\(", src)))


def test_header_declarations_are_exported(lib):
    from paper_1401_0782_gb300 import binding
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(binding.exported_symbols()) == names


def test_default_opts(lib):
    from paper_1401_0782_gb300 import binding as B
    o = B.default_opts(B.RSN_MIXED)
    assert o.precision == 1 and o.tol == 1e-10 and o.tol_inner == 1e-1 and o.use_graph == 1
    o = B.default_opts(B.RSN_FP64)
    assert o.precision == 0 and o.tol == 1e-13 and o.max_outer >= 2 and o.max_iter == 20000
    assert o.tol_adjoint == 0.0 and o.tol_T == 3e-11
    assert B.default_opts(B.RSN_MIXED).tol_T == 1e-7


def test_null_context_and_create_errors(lib):
    from paper_1401_0782_gb300 import binding as B
    assert lib.rsn_set_grid(None, 4, 4, 4, 0.5, 1) == B.RSN_EINVAL
    assert lib.rsn_set_potential(None, None) == B.RSN_EINVAL
    assert lib.rsn_destroy(None) == B.RSN_OK
    assert lib.rsn_create(None, 0, None) == B.RSN_EINVAL
    assert b"NULL" in lib.rsn_last_error(None)
    h = ct.c_void_p()
    rc = lib.rsn_create(ct.byref(h), 10_000, None)  # no such device on any machine
    assert rc in (B.RSN_ECUDA, B.RSN_EINVAL)
    assert h.value is None
    assert len(lib.rsn_last_error(None)) > 0
    # the batched entry point checks its arrays before touching a device
    assert lib.rsn_batch_transmission(0, None, None, None, None, None, None, None, None) == B.RSN_OK
    assert lib.rsn_batch_transmission(-1, None, None, None, None, None, None, None, None) == B.RSN_EINVAL
    assert lib.rsn_batch_transmission(2, None, None, None, None, None, None, None, None) == B.RSN_EINVAL
    assert B.batch_transmission([], [], []) == []


def test_package_import_loads_nothing():
    import subprocess
    import sys
    code = ("import sys; import paper_1401_0782_gb300; "
            "assert 'paper_1401_0782_gb300.binding' not in sys.modules; "
            "assert 'oracle' not in sys.modules; print('ok')")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)
    assert out.stdout.strip() == "ok", out.stderr


def test_product_code_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1401_0782_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, re.M), f
                assert "negf_oracle" not in txt, f


def test_missing_library_fails_loudly(tmp_path):
    from paper_1401_0782_gb300 import binding
    with pytest.raises(RuntimeError, match="not built"):
        binding.load(str(tmp_path / "librsnegf.so"))
