"""The C-ABI library loads without a GPU and exports what include/part.h
declares; the host-only entry points validate their arguments.  No compute
call is made here."""
import ctypes as C

import pytest

from paper_2602_23434_b300 import _lib as P
from paper_2602_23434_b300.build import build


@pytest.fixture(scope="module")
def L():
    build()
    return P.lib()


def test_exports_every_declared_symbol(L):
    names = P.header_functions()
    assert "part_gather_push" in names and "spec_update" in names and len(names) >= 16
    for nm in names:
        assert hasattr(L, nm), nm


def test_brick_dims_and_key_space(L):
    b = (C.c_int * 3)()
    nk = C.c_int64()
    g = P.make_grid(3, 128)
    assert L.part_brick_dims(C.byref(g), b, C.byref(nk)) == 0
    assert tuple(b) == (8, 8, 8) and nk.value == 128 ** 3
    g = P.make_grid(3, (20, 20, 20))
    assert L.part_brick_dims(C.byref(g), b, C.byref(nk)) == 0
    assert nk.value == 27 * 512                    # partial bricks keep full key blocks
    g = P.make_grid(2, 64)
    assert L.part_brick_dims(C.byref(g), b, C.byref(nk)) == 0
    assert tuple(b) == (16, 16, 1) and nk.value == 64 * 64


def test_workspace_size_and_validation(L):
    sz = C.c_size_t()
    g = P.make_grid(3, 128)
    assert L.part_workspace_size(C.byref(g), P.FP64, P.BORIS, 1 << 24, 0, C.byref(sz)) == 0
    # incl. the alternate particle buffers and the fields' x quadratics (192 B per cell)
    assert 1.6e9 < sz.value < 2.5e9
    assert L.part_workspace_size(C.byref(g), P.FP64, P.LP_RK2, 1 << 22, 128, C.byref(sz)) == 0
    bad = P.make_grid(3, 16)
    bad.dim = 4
    assert L.part_workspace_size(C.byref(bad), P.FP64, P.BORIS, 10, 0, C.byref(sz)) == 1
    opn = P.make_grid(3, 16)
    opn.periodic[1] = 0                     # an open (outflow) axis is accepted
    assert L.part_workspace_size(C.byref(opn), P.FP64, P.BORIS, 10, 0, C.byref(sz)) == 0
    bad = P.make_grid(3, 16)
    bad.dx[0] = 0.0
    assert L.part_workspace_size(C.byref(bad), P.FP64, P.BORIS, 10, 0, C.byref(sz)) == 1
    # LP mode keeps FP64 spectra
    assert L.part_workspace_size(C.byref(g), P.MIXED, P.LP_RK2, 10, 128, C.byref(sz)) == 6
    assert L.part_workspace_size(C.byref(g), P.FP64, P.LP_RK2, 10, 0, C.byref(sz)) == 1
    assert b"nbins" in L.part_last_error(None)
    # part_init refuses a NULL / misaligned workspace before touching CUDA
    ctx = C.c_void_p()
    assert L.part_init(C.byref(ctx), C.byref(g), 0, 2, 0, 10, 0, None, 0, None) == 1
    assert L.part_init(C.byref(ctx), C.byref(g), 0, 2, 0, 10, 0, C.c_void_p(0x1001), 1 << 30,
                       None) == 1


def test_size_limits(L):
    """The largest accepted sizes and the first refused ones: capacity below
    2^31 (particle slots are 32-bit), at most 2^30 cells (keys are 32-bit),
    spectra of 1..4096 bins; the workspace of the largest case is computed
    without overflow."""
    sz = C.c_size_t()
    g = P.make_grid(3, 1024)                               # 2^30 cells
    assert L.part_workspace_size(C.byref(g), P.FP64, P.BORIS, (1 << 31) - 1, 0,
                                 C.byref(sz)) == 0
    assert (1 << 31) * 24 < sz.value < 1 << 45             # state copies + sort buffers
    assert L.part_workspace_size(C.byref(g), P.FP64, P.BORIS, 1 << 31, 0, C.byref(sz)) == 1
    assert L.part_workspace_size(C.byref(g), P.FP64, P.BORIS, -1, 0, C.byref(sz)) == 1
    big = P.make_grid(3, (1024, 1024, 1025))
    assert L.part_workspace_size(C.byref(big), P.FP64, P.BORIS, 10, 0, C.byref(sz)) == 1
    assert b"2^30" in L.part_last_error(None)
    for nb, ok in ((1, 0), (4096, 0), (4097, 1)):
        assert L.part_workspace_size(C.byref(P.make_grid(3, 16)), P.FP64, P.LP_RK2, 10, nb,
                                     C.byref(sz)) == ok
    b = (C.c_int * 3)()
    nk = C.c_int64()
    assert L.part_brick_dims(C.byref(g), b, C.byref(nk)) == 0 and nk.value == 1 << 30


def test_multirank_and_probe_entry_points_refuse_bad_arguments(L):
    """The several-rank helpers and the FP64 probe check their arguments on
    the host before any device call (PART_EINVAL = 1)."""
    I3 = C.c_int * 3
    dims, lo, ext = I3(4, 4, 4), I3(0, 0, 0), I3(4, 4, 1)
    src = C.c_void_p(0x1000)
    assert L.part_box_pack(None, 3, dims, lo, ext, src, None) == 1            # NULL source
    assert L.part_box_pack(src, 0, dims, lo, ext, src, None) == 1             # ncomp < 1
    assert L.part_box_add(src, 3, dims, I3(0, 0, 3), I3(4, 4, 2), src, None) == 1  # outside
    assert b"outside" in L.part_last_error(None)
    assert L.part_box_pack(C.c_void_p(0x1004), 3, dims, lo, ext, src, None) == 1   # unaligned
    assert L.part_sum_ordered(None, src, 10, 2, None) == 1
    assert L.part_sum_ordered(src, src, 10, 0, None) == 1
    assert L.part_sum_ordered(src, src, -1, 2, None) == 1
    sz = C.c_size_t()
    assert L.part_exchange_bytes(None, 10, C.byref(sz)) == 1
    n = C.c_int64 * 2
    sh = P.XShift(0.0, 0, 4)
    assert L.part_exchange_pack(None, 0, 1, 2, C.byref(sh), C.byref(sh), None, 0, None, 0,
                                None, n()) == 1
    assert L.part_exchange_unpack(None, 1, None, 0) == 1
    tf, ms = C.c_double(), C.c_double()
    assert L.part_probe_fp64_fma(None, None, 4, 8192, 5, C.byref(tf), C.byref(ms)) == 1
    assert L.part_probe_fp64_fma(None, src, 9, 8192, 5, C.byref(tf), C.byref(ms)) == 1
    assert L.part_probe_fp64_fma(None, src, 4, 0, 5, C.byref(tf), C.byref(ms)) == 1
