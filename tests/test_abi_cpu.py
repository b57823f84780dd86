"""Host-side checks of the native library: it builds for sm_103a, loads
without a GPU, exports every function include/mpkrylov.h declares, and the
binding's struct layouts match the header.  No compute call is made."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mpkrylov.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mp_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1411_2377_gb300 import _lib, build

    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("mp_csr_create", "mp_csr_create_f64", "mp_csr_destroy", "mp_spmv", "mp_spmv_t",
                 "mp_dot", "mp_axpy", "mp_bicg", "mp_gpbicg", "mp_check", "mp_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib):
    from paper_1411_2377_gb300 import _lib

    assert set(declared_functions()) <= set(_lib.SIGNATURES)


def test_status_strings_without_gpu(lib):
    assert lib.mp_status_string(0) == b"ok"
    assert b"span" in lib.mp_status_string(5)
    assert lib.mp_status_string(99) == b"unknown status"


def test_struct_layouts():
    from paper_1411_2377_gb300 import _lib

    assert ctypes.sizeof(_lib.MpVec) == 32
    assert _lib.MpVec.ld.offset == 16 and _lib.MpVec.data.offset == 24
    assert ctypes.sizeof(_lib.MpSolveOpts) == 32 + 32 + 8
    assert ctypes.sizeof(_lib.MpSolveInfo) == 32


def test_library_is_built_for_sm_103a(lib):
    """The device code in the library targets sm_103a (cuobjdump lists the
    embedded ELF architectures; nothing is disassembled)."""
    import shutil
    import subprocess

    tool = shutil.which("cuobjdump") or "/usr/local/cuda/bin/cuobjdump"
    if not os.path.exists(tool):
        pytest.skip("cuobjdump not available")
    from paper_1411_2377_gb300 import _lib

    out = subprocess.run([tool, "--list-elf", _lib.LIB_PATH], capture_output=True, text=True)
    assert "sm_103a" in out.stdout


def test_config_calls_reject_bad_arguments_without_gpu(lib):
    """Argument checks of the launch-configuration calls run before any
    device work."""
    from paper_1411_2377_gb300 import _lib

    t = ctypes.c_int32()
    assert lib.mp_csr_set_config(None, 0, 128, -1, -1) == _lib.MP_ERR_ARG
    assert lib.mp_csr_get_config(None, 0, ctypes.byref(t), None, None) == _lib.MP_ERR_ARG
    assert lib.mp_csr_tune(None, 1, 3, None, None, None, None, None) == _lib.MP_ERR_ARG


def test_precision_sets_without_gpu(lib):
    """p = 2048 / 4096 / 8192 pass the precision checks of the calls that
    support them (and then stop at the missing device), other p and the
    calls kept at p <= 1024 refuse them before any device work."""
    import numpy as np

    from paper_1411_2377_gb300 import _lib

    rowptr = np.array([0, 1], np.int64)
    col = np.array([0], np.int32)
    v = np.array([2.0])
    out = ctypes.c_void_p()

    def create(p):
        return lib.mp_csr_create_f64(1, rowptr.ctypes.data, col.ctypes.data, v.ctypes.data, p, 0,
                                     None, ctypes.byref(out))

    for p in (2048, 4096, 8192):
        assert create(p) == _lib.MP_ERR_CUDA, p
    for p in (64, 3000, 16384):
        assert create(p) == _lib.MP_ERR_PREC, p
    buf = np.zeros(33 * 4, np.uint64)
    x = _lib.MpVec(4, 2048, 4, buf.ctypes.data)
    o = _lib.MpVec(1, 2048, 1, buf.ctypes.data)
    assert lib.mp_dot(x, x, o, None) == _lib.MP_ERR_CUDA
    assert lib.mp_ewise(0, x, x, x, None) == _lib.MP_ERR_PREC
    assert lib.mp_gemv(2, 2, x, _lib.MpVec(2, 2048, 2, buf.ctypes.data),
                       _lib.MpVec(2, 2048, 2, buf.ctypes.data), None) == _lib.MP_ERR_PREC
    bad = _lib.MpVec(4, 3000, 4, buf.ctypes.data)
    assert lib.mp_dot(bad, bad, bad, None) == _lib.MP_ERR_PREC


def test_autotune_leaves_the_wide_precisions_alone():
    """At 2048-8192 bits the products have one fixed form: the tuner reports
    it without touching the device or the cache."""
    from paper_1411_2377_gb300 import tune

    class Wide:
        prec = 2048

        def tune(self, *a):
            raise AssertionError("no timing at the wide precisions")

    out = tune.autotune(Wide(), cache=None)
    assert set(out) == {"ordered", "exact"}
    assert all(v["fixed"] and v["variant"] == -1 for v in out.values())


def test_noalloc_dot_refusals_without_gpu(lib):
    """mp_dot_noalloc and mp_dot refuse, on the host and before any CUDA
    call, vectors longer than MP_DOT_MAX_N (a length-2^31 view of a
    4-element host buffer: nothing reads it); mp_dot_noalloc also refuses
    the wide precisions, which only mp_dot takes."""
    import numpy as np

    from paper_1411_2377_gb300 import _lib

    buf = np.zeros(3 * 4, np.uint64)
    n = 2 ** 31
    big = _lib.MpVec(n, 128, n, buf.ctypes.data)
    out = _lib.MpVec(1, 128, 1, buf.ctypes.data)
    assert lib.mp_dot_noalloc(big, big, out, None) == _lib.MP_ERR_ARG
    assert b"maximum" in lib.mp_last_error()
    assert lib.mp_dot(big, big, out, None) == _lib.MP_ERR_ARG  # the same bound
    assert b"maximum" in lib.mp_last_error()
    wbig = _lib.MpVec(n, 2048, n, buf.ctypes.data)
    wout = _lib.MpVec(1, 2048, 1, buf.ctypes.data)
    assert lib.mp_dot(wbig, wbig, wout, None) == _lib.MP_ERR_ARG
    wide = np.zeros(33 * 4, np.uint64)
    x = _lib.MpVec(4, 2048, 4, wide.ctypes.data)
    o = _lib.MpVec(1, 2048, 1, wide.ctypes.data)
    assert lib.mp_dot_noalloc(x, x, o, None) == _lib.MP_ERR_PREC
    assert lib.mp_dot(x, x, o, None) == _lib.MP_ERR_CUDA  # accepted, then no device


def test_fault_hook_arguments_without_gpu(lib):
    from paper_1411_2377_gb300 import _lib

    assert lib.mp_debug_fail(b"x" * 80, 0) == _lib.MP_ERR_ARG
    assert lib.mp_debug_fail(b"solver poll", -1) == _lib.MP_ERR_ARG
    assert lib.mp_debug_fail(None, 0) == _lib.MP_OK


def test_binding_checks_array_lengths_without_gpu(lib):
    """The binding refuses host arrays shorter or longer than the lengths the
    library reads from them (rowptr[-1] column indices and values) and
    tensors that are not a vector's planes, before any library call."""
    import numpy as np
    import torch

    import paper_1411_2377_gb300 as mpk

    p = 128
    rowptr = np.array([0, 2, 3], np.int64)
    planes = np.zeros((p // 64 + 1, 3), np.uint64)
    with pytest.raises(ValueError, match="column indices"):
        mpk.CSR(rowptr, np.array([0, 1], np.int32), planes[:, :2], p)
    with pytest.raises(ValueError, match="column indices"):
        mpk.CSR(rowptr, np.array([0, 1, 1, 0], np.int32), planes, p)
    with pytest.raises(ValueError, match="double values"):
        mpk.CSR(rowptr, np.array([0, 1, 1], np.int32), np.array([1.0, 2.0]), p)
    with pytest.raises(ValueError, match="planes"):
        mpk.CSR(rowptr, np.array([0, 1, 1], np.int32), planes[:2], p)
    with pytest.raises(ValueError, match="offsets"):
        mpk.CSR(np.zeros(0, np.int64), np.zeros(0, np.int32), np.zeros(0), p)
    with pytest.raises(ValueError, match="column indices"):
        mpk.Batch([(rowptr, np.array([0, 1, 1], np.int32), np.ones(3)),
                   (rowptr, np.array([0, 1], np.int32), np.ones(2))], p)
    with pytest.raises(ValueError, match="double values"):
        mpk.Batch([(rowptr, np.array([0, 1, 1], np.int32), np.ones(4))], p)
    with pytest.raises(ValueError, match="shape"):
        mpk.Vec(torch.zeros((p // 64, 4), dtype=torch.int64), p)
    with pytest.raises(ValueError, match="CUDA tensor"):
        mpk.Vec(torch.zeros((p // 64 + 1, 4), dtype=torch.int64), p)


def test_host_argument_checks_without_gpu(lib):
    """Argument errors are found on the host and returned before any CUDA
    call (MP_ERR_ARG, with the offending item in mp_last_error), so they
    behave the same on a machine without a GPU: matrix creation, products,
    solvers, refinement, batches, ILU(0) and the vector calls."""
    import numpy as np

    from paper_1411_2377_gb300 import _lib

    ARG = _lib.MP_ERR_ARG
    out = ctypes.c_void_p()
    col = np.array([0, 1, 1], np.int32)
    v = np.ones(3)

    def create(n, rowptr, colidx=col, values=v, flags=0, p=128, dst=ctypes.byref(out)):
        rp = rowptr.ctypes.data if rowptr is not None else None
        ci = colidx.ctypes.data if colidx is not None else None
        va = values.ctypes.data if values is not None else None
        return lib.mp_csr_create_f64(n, rp, ci, va, p, flags, None, dst)

    good = np.array([0, 2, 3], np.int64)
    assert create(2, good, dst=None) == ARG
    assert create(-1, good) == ARG
    assert create(1 << 31, good) == ARG and b"out of range" in lib.mp_last_error()
    assert create(2, None) == ARG
    assert create(2, np.array([1, 2, 3], np.int64)) == ARG and b"rowptr[0]" in lib.mp_last_error()
    assert create(2, np.array([0, 2, 1], np.int64)) == ARG
    assert b"row 1: rowptr decreases" in lib.mp_last_error()
    assert create(2, good, colidx=None) == ARG
    assert create(2, good, values=None) == ARG
    assert create(2, good, flags=4) == ARG and b"flags" in lib.mp_last_error()
    assert out.value is None  # nothing was created

    buf = np.zeros(3 * 8, np.uint64)
    vec = lambda n, p=128: _lib.MpVec(n, p, max(n, 1), buf.ctypes.data)  # noqa: E731
    opts = _lib.MpSolveOpts(1e-30, 0.0, 100, 0, 8, _lib.MpVec(0, 128, 1, None), 0, 0)
    info = _lib.MpSolveInfo()
    for f in (lib.mp_spmv, lib.mp_spmv_t):
        assert f(None, vec(2), vec(2), 0, None) == ARG
    assert lib.mp_residual(None, vec(2), vec(2), vec(2), None) == ARG
    for f in (lib.mp_bicg, lib.mp_gpbicg, lib.mp_cgs, lib.mp_bicgstab):
        assert f(None, vec(2), vec(2), ctypes.byref(opts), ctypes.byref(info), None) == ARG
    ropts = _lib.MpRefineOpts(1e-30, 10, 1e-10, 1000, 1, 8)
    assert lib.mp_refine(None, vec(2), vec(2), ctypes.byref(ropts), None, None) == ARG
    assert lib.mp_batch_gpbicg(None, vec(2), vec(2), ctypes.byref(opts), None, None) == ARG
    assert lib.mp_ilu0_create(None, None, ctypes.byref(out)) == ARG
    assert lib.mp_ilu0_factor(None, vec(2), None) == ARG
    assert lib.mp_ilu0_apply(None, vec(2), vec(2), None) == ARG
    assert lib.mp_csr_grad(None, vec(2), vec(2), vec(2), None) == ARG
    # vector calls: lengths, precisions and the op code
    assert lib.mp_axpy(vec(1), vec(3), vec(2), None) == ARG
    assert lib.mp_axpy(vec(1), vec(2), vec(2, 256), None) == ARG
    assert lib.mp_dot(vec(2), vec(3), vec(1), None) == ARG
    assert lib.mp_dot(vec(2), vec(2), vec(2), None) == ARG  # out is a scalar
    assert lib.mp_ewise(9, vec(2), vec(2), vec(2), None) == ARG
    assert lib.mp_gemv(-1, 2, vec(0), vec(2), vec(0), None) == ARG
    assert lib.mp_gemv(2, 2, vec(3), vec(2), vec(2), None) == ARG  # A holds m*n values
    short_ld = _lib.MpVec(4, 128, 2, buf.ctypes.data)
    assert lib.mp_dot(short_ld, short_ld, vec(1), None) == ARG and b"ld" in lib.mp_last_error()
