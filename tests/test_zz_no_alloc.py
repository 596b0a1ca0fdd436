"""part_sort_fp64_noalloc, the sort entry point that allocates nothing.

Some callers cannot allocate device memory at the point where they sort:
a plug-in whose host code owns every device byte through its own pool, or a
latency-critical loop that cannot afford an allocation that may synchronise
the device.  For them the library
keeps a fixed scratch array inside libpart.so.  These tests call that entry
point through the C ABI and check that it gives bit for bit what part_sort
(the workspace-based entry point) gives on the same particles, twice in a
row with different inputs, so that leftovers in the shared scratch from the
first call cannot leak into the second.

The file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2602_23434_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2602_23434_b300 import _lib as P  # noqa: E402


def _noalloc():
    L = P.lib()
    f = L.part_sort_fp64_noalloc
    f.restype = C.c_int
    f.argtypes = [C.POINTER(P.Grid), C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                  C.c_void_p, C.c_void_p, C.c_void_p]
    return L, f


def _reference_sort(grid, x, u, w, ids):
    """part_sort through a context with a workspace; returns the sorted copies."""
    N = x.shape[1]
    p = P.Part(grid, P.FP64, P.TSC, P.BORIS, capacity=max(N, 1))
    xr, ur, wr, ir = x.clone(), u.clone(), w.clone(), ids.clone()
    p.bind(N, xr, u=ur, w=wr, ids=ir)
    p.sort()
    cs = p.cell_start().clone()
    p.sync()
    return xr, ur, wr, ir, cs, p.nkeys


def _noalloc_sort(grid, x, u, w, ids, nkeys):
    L, f = _noalloc()
    N = x.shape[1]
    xs, us, ws, is_ = x.clone(), u.clone(), w.clone(), ids.clone()
    cs = torch.full((nkeys + 1,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    rc = f(C.byref(grid), N, xs.data_ptr(), us.data_ptr(), ws.data_ptr(), is_.data_ptr(),
           cs.data_ptr(), stream.cuda_stream)
    assert rc == 0, L.part_last_error(None)
    torch.cuda.synchronize()
    return xs, us, ws, is_, cs.to(torch.int64) & 0xFFFFFFFF


def _particles(n_cells, N, seed, dim=3):
    x, u, w, ids = synth.particles(dim, None, N, seed)
    w = np.random.default_rng(seed).uniform(0.5, 2.0, N)
    dev = torch.device("cuda")
    return (torch.as_tensor(x).to(dev), torch.as_tensor(u).to(dev),
            torch.as_tensor(w).to(dev), torch.as_tensor(ids.astype(np.int64)).to(dev))


def test_noalloc_sort_matches_part_sort_twice():
    # first call: 20^3 grid (partial bricks), ragged particle count
    g1 = P.make_grid(3, 20)
    a = _particles(20, 20 ** 3 * 8 + 13, 101)
    ref = _reference_sort(g1, *a)
    got = _noalloc_sort(g1, *a, ref[5])
    for r, q in zip(ref[:5], got):
        assert torch.equal(r, q)
    # second call, straight after: other grid, fewer particles, other seed
    g2 = P.make_grid(3, 16)
    b = _particles(16, 16 ** 3 * 3 + 5, 202)
    ref2 = _reference_sort(g2, *b)
    got2 = _noalloc_sort(g2, *b, ref2[5])
    for r, q in zip(ref2[:5], got2):
        assert torch.equal(r, q)


def test_noalloc_sort_rejects_more_than_its_scratch_holds():
    L, f = _noalloc()
    g = P.make_grid(3, 16)
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    cs = torch.zeros(16 ** 3 + 1, dtype=torch.int32, device="cuda")
    rc = f(C.byref(g), 1048577, dummy.data_ptr(), dummy.data_ptr(), None, None,
           cs.data_ptr(), None)
    assert rc == 1
    assert b"1048576" in L.part_last_error(None)


def test_noalloc_sort_allocates_nothing():
    """After a first call on the device (which loads the library's kernels
    and looks up the scratch address), a call changes neither the device's
    free memory nor what torch's allocator holds."""
    L, f = _noalloc()
    g = P.make_grid(3, 16)
    a = _particles(16, 16 ** 3 * 4 + 7, 303)
    nkeys = 16 ** 3  # 16^3: two whole bricks per axis, no key gaps
    cs = torch.zeros(nkeys + 1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def call():
        rc = f(C.byref(g), a[0].shape[1], a[0].data_ptr(), a[1].data_ptr(), a[2].data_ptr(),
               a[3].data_ptr(), cs.data_ptr(), stream.cuda_stream)
        assert rc == 0, L.part_last_error(None)
        torch.cuda.synchronize()

    call()
    free0, held0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    call()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == held0
