"""The C-ABI library loads on a machine without a GPU and exports every
entry point that include/sda.h declares (no compute calls here)."""
import ctypes
import os
import re

from paper_1709_04794_gb300 import _build, sda

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sda.h")).read()
    return sorted(set(re.findall(r"SDA_API\s+[\w\s\*]+?\b(sda_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("sda_build_operator", "sda_solve_shifts", "sda_project", "sda_destroy_operator"):
        assert n in names


def test_library_loads_and_exports_every_declared_symbol():
    _build.build_libsda()
    lib = ctypes.CDLL(_build.LIBSDA)
    for name in _declared():
        assert hasattr(lib, name), name
    # the Python binding wraps exactly the declared entry points
    assert sda.exported_symbols() == _declared()


def test_status_strings_without_gpu():
    lib = sda.load()
    assert lib.sda_status_string(0) == b"SDA_OK"
    assert lib.sda_status_string(-8) == b"SDA_ERR_BREAKDOWN"
    o = sda.sda_default_opts()
    assert o.max_iter == 10000 and abs(o.tol - 1e-6) < 1e-18 and o.target_count == -1


def test_struct_layouts_match_header():
    # offsets the C side relies on (x86-64 and aarch64 share this ABI)
    assert ctypes.sizeof(sda.sda_csr) == 56
    assert ctypes.sizeof(sda.sda_shift_report) == 24
    assert sda.sda_solve_opts.rhs.offset == 24
    assert ctypes.sizeof(sda.sda_solve_opts) == 104
    assert sda.sda_solve_opts.shift_form.offset == 96
    assert ctypes.sizeof(sda.sda_solve_stats) == 112
    assert ctypes.sizeof(sda.sda_operator_info) == 128
    assert sda.sda_operator_info.exact_x_passes.offset == 120


def test_heldout_logistic_rejects_bad_arguments_without_gpu():
    """The selection call checks its sizes and offsets on the host, before any
    device work: no targets is a no-op; offsets that do not start at 0 or that
    decrease, no shifts, and missing outputs are INVALID_ARG."""
    import numpy as np
    lib = sda.load()

    def call(n, ns, off, out=True):
        o = np.ascontiguousarray(off, dtype=np.int64)
        p = ctypes.c_void_p(8) if out else None            # never dereferenced: the checks come first
        return lib.sda_heldout_logistic(n, ns, o.ctypes.data, None, None, p, p, None, None)

    assert call(0, 4, [0]) == sda.SDA_OK
    assert call(2, 4, [1, 2, 3]) == sda.SDA_ERR_INVALID_ARG
    assert call(2, 4, [0, 3, 2]) == sda.SDA_ERR_INVALID_ARG
    assert call(2, 0, [0, 1, 2]) == sda.SDA_ERR_INVALID_ARG
    assert call(-1, 4, [0]) == sda.SDA_ERR_INVALID_ARG
    assert call(1, 4, [0, 0], out=False) == sda.SDA_ERR_INVALID_ARG
    assert call(1, 4, [0, 5]) == sda.SDA_ERR_INVALID_ARG        # rows but no scores, y or g
