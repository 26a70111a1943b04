"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads,
exports every entry point declared in include/amgt.h, and rejects bad calls
without touching a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2010_04559_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def _declared():
    src = open(os.path.join(ROOT, "include", "amgt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(amgt_[A-Za-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    assert "amgt_solve" in names and "amgt_op_sweep" in names and "amgt_op_scatter" in names
    from paper_2010_04559_gb300 import EXPORTS
    assert sorted(EXPORTS) == names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_null_context_is_rejected(lib):
    lib.amgt_set_angular_uniform.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
    lib.amgt_set_angular_uniform.restype = ctypes.c_int
    assert lib.amgt_set_angular_uniform(None, 1, 2) == -1
    lib.amgt_last_error.argtypes = [ctypes.c_void_p]
    lib.amgt_last_error.restype = ctypes.c_char_p
    assert lib.amgt_last_error(None) == b"null context"
    lib.amgt_create.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    lib.amgt_create.restype = ctypes.c_int
    assert lib.amgt_create(None, 0, None) == -1


def test_batch_calls_reject_bad_arguments(lib):
    """The batch entry points refuse a null list, a negative count, null
    members and a context listed twice before any thread or device work (no
    member is dereferenced: the repeated one below is a zeroed host buffer,
    not a context); an empty batch succeeds."""
    P = ctypes.c_void_p
    lib.amgt_setup_batch.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.c_int]
    lib.amgt_setup_batch.restype = ctypes.c_int
    assert lib.amgt_setup_batch(None, 1, 0) == -1
    empty = (P * 1)(None)
    assert lib.amgt_setup_batch(empty, -1, 0) == -1
    assert lib.amgt_setup_batch(empty, 1, 0) == -1        # a null context in the list
    assert lib.amgt_setup_batch(empty, 0, 0) == 0
    fake = ctypes.create_string_buffer(1 << 16)
    twice = (P * 2)(ctypes.addressof(fake), ctypes.addressof(fake))
    assert lib.amgt_setup_batch(twice, 2, 0) == -1
    lib.amgt_solve_batch.argtypes = [ctypes.POINTER(P), ctypes.c_int, P, ctypes.POINTER(P),
                                     ctypes.POINTER(P), P, ctypes.c_int]
    lib.amgt_solve_batch.restype = ctypes.c_int
    opts = ctypes.create_string_buffer(256)
    bufs = (P * 2)(ctypes.addressof(fake), ctypes.addressof(fake))
    assert lib.amgt_solve_batch(twice, 2, ctypes.addressof(opts), bufs, None, None, 0) == -1
    assert lib.amgt_solve_batch(empty, 1, ctypes.addressof(opts), bufs, None, None, 0) == -1
    assert lib.amgt_solve_batch(empty, 0, ctypes.addressof(opts), bufs, None, None, 0) == 0


def _header_constants():
    src = open(os.path.join(ROOT, "include", "amgt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {name: int(val) for name, val in re.findall(r"#define\s+(AMGT_[A-Z_0-9]+)\s+(-?\d+)", src)}
    for name, val in re.findall(r"\b(AMGT_[A-Z_0-9]+)\s*=\s*(-?\d+)", src):
        out[name] = int(val)
    return out


def test_binding_constants_match_the_header():
    """The tuning keys, kernel-timer classes, dtypes, modes and error codes
    the header defines are exported by the package with the same values."""
    import paper_2010_04559_gb300 as pkg
    from paper_2010_04559_gb300 import _capi
    consts = _header_constants()
    assert len(consts) > 30
    for name, val in consts.items():
        assert hasattr(_capi, name), name
        assert getattr(_capi, name) == val, name
        if name.startswith(("AMGT_TUNE_", "AMGT_KT_", "AMGT_F", "AMGT_MODE_", "AMGT_PREC_",
                            "AMGT_KRYLOV_")) and name != "AMGT_KT_COUNT":
            assert getattr(pkg, name) == val, name


def test_without_a_gpu_the_library_fails_loudly(lib):
    """No CUDA device (this CPU host): context creation returns
    AMGT_ERR_CUDA and leaves no handle, and the Python binding raises
    instead of computing anything on the CPU (there is no CPU fallback)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is visible")
    from paper_2010_04559_gb300 import AMGT_ERR_CUDA, AmgtError, context_from_problem
    h = ctypes.c_void_p(1)
    lib.amgt_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p]
    lib.amgt_create.restype = ctypes.c_int
    assert lib.amgt_create(ctypes.byref(h), 0, None) == AMGT_ERR_CUDA
    assert not h.value
    import workloads as W
    with pytest.raises(AmgtError) as e:
        context_from_problem(W.random_problem(2, (3, 3), 1, 4, 1), device=0)
    assert e.value.code == AMGT_ERR_CUDA
