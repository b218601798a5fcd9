"""The C-ABI library builds, loads without a GPU and exports every entry point
the public headers declare (no compute calls)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(lbm_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2501_00620_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_headers_declare_the_boundary():
    names = declared_functions()
    for required in ("lbm_create", "lbm_init", "lbm_step", "lbm_moments", "lbm_diagnostics",
                     "lbm_save", "lbm_load", "lbm_destroy", "lbm_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    lib.lbm_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.lbm_version()
    from paper_2501_00620_gb300 import lbm
    o = lbm.lbm_default_opts()
    assert o.dtype == lbm.LBM_F64 and o.tile == -1 and o.diagnostics == 1 and o.use_graphs == 1


def test_argument_validation_needs_no_gpu(lib):
    """Invalid arguments are rejected before any CUDA call."""
    from paper_2501_00620_gb300 import lbm
    for args in [(4, 8, 1, 1, 0.8, 0.3), (1, 8, 2, 1, 0.8, 0.3), (2, 8, 8, 1, -1.0, 0.3),
                 (2, 8, 8, 1, 0.8, 0.0), (3, 0, 4, 4, 0.8, 0.3)]:
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_create(*args, bc=lbm.LBM_BC_PERIODIC)
        assert e.value.status == lbm.LBM_EINVAL
