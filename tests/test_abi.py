"""C ABI checks that need no GPU: the library builds, loads, exports every function
include/ftlm.h declares, and rejects invalid arguments before touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2605_26261_gb300 import _build
from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "ftlm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ftlm_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_api():
    names = declared_functions()
    for n in ("ftlm_basis_create", "ftlm_hv", "ftlm_lanczos", "ftlm_thermo", "ftlm_ritz"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    lib.ftlm_status_string.restype = ctypes.c_char_p
    for s in range(7):
        assert lib.ftlm_status_string(s).startswith(b"FTLM_")
    assert lib.ftlm_status_string(6).startswith(b"FTLM_ENOCONV")


def _create(lib, N, two_sz, bonds, mode=0):
    bi = np.ascontiguousarray([b[0] for b in bonds], dtype=np.int32)
    bj = np.ascontiguousarray([b[1] for b in bonds], dtype=np.int32)
    J = np.ascontiguousarray([b[2] for b in bonds], dtype=np.float64)
    out = ctypes.c_void_p()
    lib.ftlm_basis_create.restype = ctypes.c_int
    st = lib.ftlm_basis_create(N, two_sz, len(J), ctypes.c_void_p(bi.ctypes.data),
                               ctypes.c_void_p(bj.ctypes.data), ctypes.c_void_p(J.ctypes.data), mode,
                               None, ctypes.byref(out))
    return st, out


@pytest.mark.parametrize("N,two_sz,bonds,mode,want", [
    (0, 0, [], 0, 1),                                  # N < 1
    (37, 1, [], 0, 1),                                 # N > FTLM_MAX_SITES
    (4, 1, [(0, 1, 1.0)], 0, 1),                       # parity of two_sz
    (4, 6, [(0, 1, 1.0)], 0, 1),                       # |two_sz| > N
    (4, 0, [(0, 0, 1.0)], 0, 1),                       # self bond
    (4, 0, [(0, 4, 1.0)], 0, 1),                       # site out of range
    (4, 0, [(0, 1, 1.0), (1, 0, 2.0)], 0, 1),          # duplicate pair
    (4, 0, [(0, 1, float("nan"))], 0, 1),              # non-finite J
    (4, 0, [(0, 1, 1.0)], 7, 1),                       # bad mode
    (34, 0, [(0, 1, 1.0)], 1, 3),                      # CLT needs N <= 32
    (36, 0, [(0, 1, 1.0)], 2, 3),                      # D = C(36, 18) >= 2^32
])
def test_create_rejects_bad_arguments(lib, N, two_sz, bonds, mode, want):
    st, out = _create(lib, N, two_sz, bonds, mode)
    assert st == want
    assert not out.value
    lib.ftlm_last_error.restype = ctypes.c_char_p
    assert len(lib.ftlm_last_error()) > 0


def test_too_many_bonds_unsupported(lib):
    bonds = [(i, j, 1.0) for i in range(24) for j in range(i + 1, 24)]  # 276 > 256
    st, _ = _create(lib, 24, 0, bonds)
    assert st == 3


def test_null_handles_rejected(lib):
    assert lib.ftlm_hv(None, 1, None, None, None) == 1
    assert lib.ftlm_basis_labels(None, ctypes.c_uint64(0), ctypes.c_uint64(1), None, None) == 1
    assert lib.ftlm_lanczos_workspace_bytes(None, 1, 10, 1, None) == 1
    assert lib.ftlm_ritz(-1, 10, None, None, None, None, None, None) == 1
    assert lib.ftlm_ritz(1, 0, None, None, None, None, None, None) == 1
    assert lib.ftlm_thermo(0, None, None, 1, 1, None, None, None, 1, ctypes.c_double(2.0),
                           ctypes.c_double(0.0), 1, None, None, None, None, None, None) == 1
    lib.ftlm_basis_destroy(None)  # ignored


def test_profile_toggle_without_gpu(lib):
    assert lib.ftlm_profile_enable(1) == 0
    a, v, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    b, d = ctypes.c_double(), ctypes.c_double()
    assert lib.ftlm_profile_read(ctypes.byref(a), ctypes.byref(v), ctypes.byref(b), ctypes.byref(c),
                                 ctypes.byref(d)) == 0
    assert a.value == 0 and v.value == 0 and c.value == 0
    assert lib.ftlm_profile_enable(0) == 0


def _create_spin(lib, N, two_s, two_sz, bonds):
    bi = np.ascontiguousarray([b[0] for b in bonds], dtype=np.int32)
    bj = np.ascontiguousarray([b[1] for b in bonds], dtype=np.int32)
    J = np.ascontiguousarray([b[2] for b in bonds], dtype=np.float64)
    out = ctypes.c_void_p()
    lib.ftlm_basis_create_spin.restype = ctypes.c_int
    st = lib.ftlm_basis_create_spin(N, two_s, two_sz, len(J), ctypes.c_void_p(bi.ctypes.data),
                                    ctypes.c_void_p(bj.ctypes.data), ctypes.c_void_p(J.ctypes.data), None,
                                    ctypes.byref(out))
    return st, out


@pytest.mark.parametrize("N,two_s,two_sz,bonds,want", [
    (6, 0, 0, [(0, 1, 1.0)], 1),                 # two_s < 1
    (6, 2, 1, [(0, 1, 1.0)], 1),                 # parity of two_sz
    (6, 2, 14, [(0, 1, 1.0)], 1),                # |two_sz| > N two_s
    (6, 8, 0, [(0, 1, 1.0)], 3),                 # s = 4 > 7/2
    (17, 2, 0, [(0, 1, 1.0)], 3),                # N > 16 at s > 1/2
    (6, 2, 0, [(0, 0, 1.0)], 1),                 # self bond
    (6, 2, 0, [(0, 1, 1.0), (1, 0, 1.0)], 1),    # duplicate pair
    (6, 2, 0, [(0, 6, 1.0)], 1),                 # site out of range
    (6, 1, 1, [(0, 1, 1.0)], 1),                 # two_s = 1: the spin-1/2 checks (parity)
])
def test_create_spin_rejects_bad_arguments(lib, N, two_s, two_sz, bonds, want):
    st, out = _create_spin(lib, N, two_s, two_sz, bonds)
    assert st == want and not out.value


def test_new_entry_points_validate_without_a_device(lib):
    P = ctypes.c_void_p
    lib.ftlm_lanczos_set_block.restype = ctypes.c_int
    assert lib.ftlm_lanczos_set_block(3) == 1
    assert lib.ftlm_lanczos_set_block(0) == 0
    assert lib.ftlm_launch_count(None) == 1
    n = ctypes.c_uint64()
    assert lib.ftlm_launch_count(ctypes.byref(n)) == 0
    assert lib.ftlm_basis_destroy_async(None, None) == 0
    assert lib.ftlm_batch_destroy_async(None, None) == 0
    lib.ftlm_ghosts.argtypes = [ctypes.c_int, ctypes.c_int] + [P] * 5 + [ctypes.c_double] * 2 + [P] * 6
    assert lib.ftlm_ghosts(-1, 10, *([None] * 5), 1.0, 1e-7, *([None] * 6)) == 1
    assert lib.ftlm_ghosts(1, 0, *([None] * 5), 1.0, 1e-7, *([None] * 6)) == 1
    assert lib.ftlm_ghosts(1, 10, *([None] * 5), -1.0, 1e-7, *([None] * 6)) == 1
    assert lib.ftlm_ghosts(0, 10, *([None] * 5), 1.0, 1e-7, *([None] * 6)) == 0  # nothing to do
    assert lib.ftlm_sigma_emp(0, 5, None, None, None, None) == 1
    assert lib.ftlm_sigma_emp(2, 0, None, None, None, None) == 0
    lib.ftlm_partition.argtypes = [ctypes.c_int, P, P, ctypes.c_int, ctypes.c_int, P, P, P, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_int, P, P, P, P]
    assert lib.ftlm_partition(0, None, None, 1, 1, None, None, None, 1, 0.0, 1, None, None, None, None) == 1
    lib.ftlm_batch_create.argtypes = [ctypes.c_int, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, P, ctypes.POINTER(P)]
    out = P()
    assert lib.ftlm_batch_create(0, None, 10, 0, 1, 0, 0, None, ctypes.byref(out)) == 1  # empty batch
