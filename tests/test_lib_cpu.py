"""Host-only checks of the C-ABI library: it builds for sm_103a, loads, and
exports every function include/spgemm.h declares.  No GPU work is done."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(spgemm_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1510_00844_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("spgemm_plan", "spgemm_symbolic", "spgemm_numeric", "spgemm_merge_symbolic",
                     "spgemm_merge_numeric", "spgemm_kslice_bounds", "spgemm_plan_destroy",
                     "spgemm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_pure_host_entry_points(lib):
    lib.spgemm_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.spgemm_version()
    lib.spgemm_plan_workspace_size.restype = ctypes.c_size_t
    lib.spgemm_plan_workspace_size.argtypes = [ctypes.c_int64]
    a = lib.spgemm_plan_workspace_size(1000)
    b = lib.spgemm_plan_workspace_size(2000)
    assert b > a > 0 and a % 256 == 0


def test_argument_errors_need_no_gpu(lib):
    from paper_1510_00844_gb300 import spgemm as sg
    plan = ctypes.c_void_p()
    # NULL A -> INVALID_ARG before any device work
    st = sg._lib.spgemm_plan(None, None, None, None, None, 0, ctypes.byref(plan))
    assert st == 1
    assert b"NULL" in sg._lib.spgemm_last_error()
    A = sg._Csr(4, 5, 0, 1, None, None, None, 0, 0)
    B = sg._Csr(6, 3, 0, 1, None, None, None, 0, 0)   # 5 != 6
    st = sg._lib.spgemm_plan(ctypes.byref(A), ctypes.byref(B), None, None, None, 0,
                             ctypes.byref(plan))
    assert st == 1 and b"inner dimensions" in sg._lib.spgemm_last_error()
    B = sg._Csr(5, 3, 0, 1, None, None, None, 0, 0)
    st = sg._lib.spgemm_plan(ctypes.byref(A), ctypes.byref(B), None, None, None, 0,
                             ctypes.byref(plan))
    assert st == 4   # plan workspace missing
    Bbad = sg._Csr(5, 3, 0, 1, None, None, None, 0, 9)
    st = sg._lib.spgemm_plan(ctypes.byref(A), ctypes.byref(Bbad), None, None, None, 0,
                             ctypes.byref(plan))
    assert st == 1 and b"value_type" in sg._lib.spgemm_last_error()


def test_merge_argument_errors(lib):
    from paper_1510_00844_gb300 import spgemm as sg
    arr = (sg._Csr * 1)()
    nnz = ctypes.c_int64()
    st = sg._lib.spgemm_merge_symbolic(0, arr, None, None, None, 0, None, ctypes.byref(nnz))
    assert st == 1 and b"c <= 32" in sg._lib.spgemm_last_error()
    st = sg._lib.spgemm_merge_symbolic(33, arr, None, None, None, 0, None, ctypes.byref(nnz))
    assert st == 1


def test_kernels_are_compiled_for_sm103a():
    from paper_1510_00844_gb300 import build
    assert ["-gencode", "arch=compute_103a,code=sm_103a"] == build.ARCH
    assert "-fmad=false" in build.FLAGS


def test_sizer_record_checks_need_no_gpu(lib):
    """spgemm_sizer_save answers its size query and spgemm_sizer_load rejects
    malformed records before touching the device."""
    P, S, I32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32
    lib.spgemm_sizer_save.argtypes = [P, I32, P, P, S, ctypes.POINTER(S)]
    lib.spgemm_sizer_load.argtypes = [P, S, I32, P, P]
    lib.spgemm_sizer_param_count.argtypes = [I32]
    need = S()
    assert lib.spgemm_sizer_save(None, 6, None, None, 0, ctypes.byref(need)) == 0
    count = lib.spgemm_sizer_param_count(6)
    assert need.value == 8 + 24 + 4 * count + 8
    rec = ctypes.create_string_buffer(b"NOTSIZER" + bytes(need.value - 8))
    assert lib.spgemm_sizer_load(rec, need.value, 6, None, None) == 1          # wrong magic
    head = b"SGSIZER\x00" + (2).to_bytes(4, "little") + bytes(need.value - 12)
    rec = ctypes.create_string_buffer(head)
    assert lib.spgemm_sizer_load(rec, need.value, 6, None, None) == 7          # other version
    import struct
    head = b"SGSIZER\x00" + struct.pack("<6I", 1, 6, 32, 1, 1, count)
    rec = ctypes.create_string_buffer(head + bytes(4 * count + 8))
    assert lib.spgemm_sizer_load(rec, need.value - 1, 6, None, None) == 1      # truncated
    assert lib.spgemm_sizer_load(rec, need.value, 6, None, None) == 1          # hash mismatch
    assert lib.spgemm_sizer_load(rec, need.value, 7, None, None) == 1          # another F


def test_chain_argument_errors_need_no_gpu(lib):
    """spgemm_chain_create rejects bad arguments before any device access
    (the workspace address below is never dereferenced)."""
    from paper_1510_00844_gb300 import spgemm as sg
    L = sg._lib
    L.spgemm_chain_workspace_size.restype = ctypes.c_size_t
    need = L.spgemm_chain_workspace_size(1)
    assert need >= 256 and need % 256 == 0
    steps = (sg._ChainStep * 1)()
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(1 << 20)            # 256-byte aligned, not memory
    ok_opts = sg._ChainOpts(0.0, -1, 0, None)
    # no steps
    assert L.spgemm_chain_create(0, steps, ctypes.byref(ok_opts), fake, need, ctypes.byref(h)) == 1
    # workspace too small / not aligned
    assert L.spgemm_chain_create(1, steps, ctypes.byref(ok_opts), fake, need - 1,
                                 ctypes.byref(h)) == 4
    assert L.spgemm_chain_create(1, steps, ctypes.byref(ok_opts), ctypes.c_void_p((1 << 20) + 8),
                                 need, ctypes.byref(h)) == 1
    # negative timeout, unsupported block size, missing plan
    bad_t = sg._ChainOpts(-1.0, -1, 0, None)
    assert L.spgemm_chain_create(1, steps, ctypes.byref(bad_t), fake, need, ctypes.byref(h)) == 1
    bad_b = sg._ChainOpts(0.0, -1, 512, None)
    assert L.spgemm_chain_create(1, steps, ctypes.byref(bad_b), fake, need, ctypes.byref(h)) == 1
    assert b"block_threads" in L.spgemm_last_error()
    assert L.spgemm_chain_create(1, steps, ctypes.byref(ok_opts), fake, need, ctypes.byref(h)) == 1
    assert b"plan" in L.spgemm_last_error()
