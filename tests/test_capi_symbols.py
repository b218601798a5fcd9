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


def test_boundary_model_and_setting_validation_needs_no_gpu(lib):
    """Walls need dim 2 or 3; the comparator model runs on periodic lattices
    with ny, nz <= 65535; unknown boundaries and models are refused; the
    force, wall-velocity and MRT setters refuse a NULL simulation -- all on
    the host, before any CUDA call."""
    from paper_2501_00620_gb300 import lbm
    bad = [((1, 64, 1, 1, 0.8, 0.3), dict(bc=lbm.LBM_BC_WALLS)),
           ((2, 8, 8, 1, 0.8, 0.3), dict(bc=7))]
    o = lbm.lbm_default_opts()
    o.model = lbm.LBM_MODEL_STANDARD
    bad += [((2, 8, 8, 1, 0.8, 0.3), dict(bc=lbm.LBM_BC_WALLS, opts=o)),
            ((2, 8, 8, 1, 0.8, 0.3), dict(bc=lbm.LBM_BC_FIXED_STATE, opts=o)),
            ((2, 8, 70000, 1, 0.8, 0.3), dict(bc=lbm.LBM_BC_PERIODIC, opts=o))]
    o2 = lbm.lbm_default_opts()
    o2.model = 5
    bad.append(((2, 8, 8, 1, 0.8, 0.3), dict(bc=lbm.LBM_BC_PERIODIC, opts=o2)))
    for args, kw in bad:
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_create(*args, **kw)
        assert e.value.status == lbm.LBM_EINVAL
    for call in (lambda: lbm.lbm_set_force(None, [1e-4, 0.0]),
                 lambda: lbm.lbm_set_wall_velocity(None, [0.01, 0.0], [0.0, 0.0]),
                 lambda: lbm.lbm_set_mrt(None, 1.2, 1.2),
                 lambda: lbm.lbm_set_debug(None, lbm.LBM_DEBUG_MISSING_COPY),
                 lambda: lbm.lbm_set_small_t(None, 1.0)):
        with pytest.raises(lbm.LBMError) as e:
            call()
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
    # D1Q3, 8 sites: f planes 3 x 64 bytes, b plane 64 bytes
    fb, bb = 3 * 8 * 8, 8 * 8
    base = 1 << 20
    f_in, b_in, f_out, b_out = base, base + 4096, base + 8192, base + 12288
    overlapping = [
        (f_in, b_in, f_in, b_out),                 # output = input
        (f_in, b_in, f_out, b_in + 8),             # b_out partly over b_in
        (f_in, b_in, f_in + fb - 8, b_out),        # f_out starts inside f_in
        (f_in, b_in, f_out, f_in + 16),            # a b plane inside an f buffer
        (f_in, b_in, f_out, f_out + fb - bb // 2),  # the two outputs overlap
    ]
    for ptrs in overlapping:
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_step_noalloc(1, 8, 1, 1, 0.8, 0.3, 0, *ptrs)
        assert e.value.status == lbm.LBM_EINVAL and "overlap" in str(e.value), ptrs


def test_binding_structs_match_the_headers(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets
    the C compiler gives the header's struct (gcc on the host)."""
    from paper_2501_00620_gb300 import lbm
    structs = [lbm.lbm_opts, lbm.lbm_fields_in, lbm.lbm_fields_out, lbm.lbm_server_opts,
               lbm.lbm_request, lbm.lbm_server_stats]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lbm_serve.h"', "int main(void) {"]
    for st in structs:
        name = st.__name__
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for f in st._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, f[0], name, f[0]))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    import subprocess
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(ln.split() for ln in subprocess.check_output([str(exe)], text=True).splitlines())
    for st in structs:
        name = st.__name__
        assert int(got[name]) == ctypes.sizeof(st), name
        for f in st._fields_:
            assert int(got["%s.%s" % (name, f[0])]) == getattr(st, f[0]).offset, (name, f[0])
