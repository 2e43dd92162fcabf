"""The C-ABI library loads and exports every function include/askit.h declares
(CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "askit.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_][a-z_0-9]*\s*\*?\s*(askit_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1410_0260_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_api():
    names = declared_functions()
    for n in ["askit_setup", "askit_set_weights", "askit_evaluate", "askit_evaluate_targets",
              "askit_evaluate_host", "askit_get_info", "askit_get_structure", "askit_sync", "askit_destroy"]:
        assert n in names


def test_library_exports_every_declared_function(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_binding_lists_every_export():
    from paper_1410_0260_gb300 import askit
    assert sorted(askit.EXPORTS) == declared_functions()


def test_host_only_calls(lib):
    lib.askit_status_string.restype = ctypes.c_char_p
    assert lib.askit_status_string(0) == b"ok"
    assert lib.askit_status_string(4) == b"device wait timed out"

    from paper_1410_0260_gb300.askit import Params   # layout checked in test_abi_layout.py
    p = Params()
    lib.askit_default_params(ctypes.byref(p))
    assert p.leaf_size == 128 and p.kappa == 16 and p.ell_extra == 20 and p.kernel_scale == 0.5
    assert p.batch_entries == 0 and p.prune == 1
    # invalid arguments are rejected before any device work
    out = ctypes.c_void_p()
    lib.askit_setup.restype = ctypes.c_int
    rc = lib.askit_setup(ctypes.c_void_p(16), ctypes.c_int64(0), 3, ctypes.c_int64(3), None, None,
                         ctypes.byref(p), None, ctypes.byref(out))
    assert rc == 1 and not out.value
    # a leaf or skeleton longer than 16 sub-blocks of 128 rows cannot be
    # indexed by the work lists: refused (UNSUPPORTED) before any device work
    for field, val in (("leaf_size", 4096), ("s_max", 2049)):
        q = Params()
        lib.askit_default_params(ctypes.byref(q))
        setattr(q, field, val)
        rc = lib.askit_setup(ctypes.c_void_p(16), ctypes.c_int64(3000), 3, ctypes.c_int64(3), None, None,
                             ctypes.byref(q), None, ctypes.byref(out))
        assert rc == 6 and not out.value, field
    q = Params()
    lib.askit_default_params(ctypes.byref(q))
    q.leaf_size, q.kappa = 2, 1                      # 2^30 points in leaves of 2: depth 29 > 25
    rc = lib.askit_setup(ctypes.c_void_p(16), ctypes.c_int64(1 << 30), 3, ctypes.c_int64(3), None, None,
                         ctypes.byref(q), None, ctypes.byref(out))
    assert rc == 6 and not out.value


def test_oracle_and_product_share_no_code():
    pkg = os.path.join(ROOT, "paper_1410_0260_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "askit_oracle" not in txt, f
