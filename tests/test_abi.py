"""The C-ABI library loads without a GPU and exports every function include/*.h declares.

No compute call is made here; the library is built first if it is missing (nvcc
cross-compiles sm_103a without a device).
"""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(hdr).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]+?\b(sl_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    import paper_1605_04821_gb300 as slp
    from paper_1605_04821_gb300 import build
    if not os.path.exists(slp.LIB_PATH):
        build.build()
    return ctypes.CDLL(slp.LIB_PATH)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("sl_hjb_create", "sl_hjb_step", "sl_hjb_solve", "sl_hjb_destroy",
                     "sl_hjb_last_error", "sl_opts_default"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_symbol():
    import paper_1605_04821_gb300 as slp
    assert set(slp.EXPORTED) == _declared()


def test_opts_default_without_gpu(lib):
    import paper_1605_04821_gb300 as slp
    o = slp.default_opts()
    assert o.nu1 == 2 and o.nu2 == 2 and abs(o.omega - 0.8) < 1e-15
    assert o.krylov_tol == 1e-12 and o.tie_rel == 1e-12 and o.precision == 0
