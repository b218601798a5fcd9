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


def test_noalloc_step_rejects_before_any_cuda_call(lib):
    """The no-allocation step validates its sizes on the host first: a lattice
    needing more diagnostics scratch than the fixed array holds is refused
    with a message, before the buffers are touched."""
    from paper_2501_00620_gb300 import lbm
    buf = [16 * (k + 1) for k in range(4)]  # placeholders, never dereferenced on these paths
    cases = [
        ((0, 8, 1, 1, 0.8, 0.3, 0), "extents"),
        ((2, 8, 8, 2, 0.8, 0.3, 0), "extents"),
        ((2, 8, 8, 1, 0.0, 0.3, 0), "tau"),
        ((1, 43681 * 256, 1, 1, 0.8, 0.3, 0), "too large"),
        ((2, 128 * 182, 64 * 181, 1, 0.8, 0.3, 0), "too large"),
        ((3, 32 * 100, 8 * 100, 64 * 3, 0.52, 0.05, 0), "too large"),
    ]
    for args, msg in cases:
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_step_noalloc(*args, *buf)
        assert e.value.status == lbm.LBM_EINVAL
        assert msg in str(e.value)
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_step_noalloc(1, 8, 1, 1, 0.8, 0.3, 0, buf[0], buf[1], buf[0], buf[3])
    assert "differ" in str(e.value)
