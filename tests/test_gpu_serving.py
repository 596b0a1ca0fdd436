"""Continuous-batching server: a request's result is the same alone and in a
mix (bitwise: test particles never interact and every slice runs the same
per-particle arithmetic), equals part_gather_push with nsteps fused steps,
admission respects the device-memory budget, bad work items are refused on
the host, and latency statistics are reported."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2602_23434_b300 import _lib as P  # noqa: E402
from paper_2602_23434_b300 import serving as S  # noqa: E402


@pytest.fixture(scope="module")
def snaps():
    return [S.make_snapshot(torch, 32, 501, capacity=20000),
            S.make_snapshot(torch, 48, 502, capacity=20000)]


def _state(r):
    c, o, u = r.result()
    return c.clone(), o.clone(), u.clone()


def _same(a, b):
    return all(torch.equal(x, y) for x, y in zip(a, b))


def test_request_alone_equals_mixed_and_fused_push(snaps):
    budget = 1 << 30
    # A alone, 50-step slices
    s1 = S.Server(torch, snaps, budget, chunk=2048, slice_steps=50)
    a1 = s1.submit(1, 5000, 137, seed=11, dt=0.02)
    s1.run_until_idle()
    alone = _state(a1)
    assert a1.latency is not None and a1.latency > 0
    s1.close()
    # A in a mix: other requests before, alongside and after it; 20-step slices
    s2 = S.Server(torch, snaps, budget, chunk=1024, slice_steps=20)
    s2.submit(0, 12000, 300, seed=21, dt=0.03)
    s2.round()
    a2 = s2.submit(1, 5000, 137, seed=11, dt=0.02)
    s2.submit(1, 3000, 40, seed=31, dt=0.01)
    s2.round()
    s2.submit(0, 999, 7, seed=41, dt=0.05)
    s2.run_until_idle()
    assert _same(_state(a2), alone)
    st = s2.stats()
    assert st["completed"] == 4 and st["p50_s"] is not None and st["p99_s"] >= st["p50_s"]
    s2.close()
    # A in the same mix under a work budget per round (every request an equal
    # share of 2e5 particle-steps per round: other slicings, same bits)
    s3 = S.Server(torch, snaps, budget, chunk=1024, round_psteps=2e5)
    s3.submit(0, 12000, 300, seed=21, dt=0.03)
    s3.round()
    a3 = s3.submit(1, 5000, 137, seed=11, dt=0.02)
    s3.submit(1, 3000, 40, seed=31, dt=0.01)
    s3.round()
    s3.submit(0, 999, 7, seed=41, dt=0.05)
    s3.run_until_idle()
    assert _same(_state(a3), alone)
    assert s3.stats()["completed"] == 4
    s3.close()
    # the same request through part_gather_push (fused nsteps, one launch)
    n = 48
    p = P.Part(P.make_grid(3, n), P.MIXED, P.TSC, P.BORIS, capacity=5000)
    p.set_fields(snaps[1].fields)
    cell = torch.empty(5000, dtype=torch.int32, device="cuda")
    off = torch.empty((3, 5000), dtype=torch.float32, device="cuda")
    u = torch.empty((6, 5000), dtype=torch.float32, device="cuda")   # compensated pair
    p.bind(5000, cell, off=off, u=u)
    p.init_particles(11, 0.1)
    p.sort()
    p.gather_push(1.0, 0.02, 137)
    p.sync()
    assert _same((cell, off, u), alone)


def test_admission_by_memory_budget(snaps):
    per = 4000 * S.STATE_BYTES_PER_PARTICLE
    srv = S.Server(torch, snaps, mem_budget_bytes=per + 10, chunk=1024, slice_steps=10)
    rs = [srv.submit(i % 2, 4000, 30, seed=100 + i) for i in range(3)]
    srv.round()
    assert len(srv.active) == 1 and len(srv.queue) == 2       # only one fits
    srv.run_until_idle()
    assert [r.rid for r in srv.finished] == [r.rid for r in rs]   # FIFO completion
    assert all(r.admitted >= rs[0].admitted for r in rs)
    with pytest.raises(P.PartError) as e:
        srv.submit(0, 100000, 5, seed=1)                     # larger than the budget
    assert e.value.name == "PART_ENOMEM"
    srv.close()


def test_bad_work_item_refused_on_host(snaps):
    srv = S.Server(torch, snaps, 1 << 26, chunk=1024)
    r = srv.submit(0, 2000, 5, seed=3)
    srv.round()                                               # admits and runs one round
    srv.drain()              # that round's work list is read by the GPU: let it finish first
    w = srv.items[0]
    w.cell, w.off, w.u = r.cell.data_ptr(), r.off.data_ptr(), r.u.data_ptr()
    w.stride, w.first, w.count, w.nsteps = 2000, 1500, 1000, 1   # slice past the end
    w.snapshot, w.q_over_m, w.dt = 0, 1.0, 0.01
    assert srv.L.part_server_run(srv.h, 1) == 1
    assert b"bad slice" in srv.L.part_last_error(None)
    w.count, w.snapshot = 10, 7                               # snapshot out of range
    assert srv.L.part_server_run(srv.h, 1) == 1
    srv.close()


def test_server_refuses_default_stream(snaps):
    """A round is captured into a CUDA graph, which a default stream cannot
    hold: the server refuses it before capturing anything."""
    L = P.lib()
    db, hb = C.c_size_t(), C.c_size_t()
    assert L.part_server_sizes(2, 16, C.byref(db), C.byref(hb)) == 0
    ws = torch.empty(db.value, dtype=torch.uint8, device="cuda")
    stage = torch.empty(hb.value, dtype=torch.uint8, pin_memory=True)
    arr = (C.c_void_p * 2)(snaps[0].part.ctx.value, snaps[1].part.ctx.value)
    h = C.c_void_p()
    rc = L.part_server_init(C.byref(h), arr, 2, 16, C.c_void_p(ws.data_ptr()), db.value,
                            C.c_void_p(stage.data_ptr()), hb.value, None, 256, 4)
    assert rc == 1 and b"created stream" in L.part_last_error(None)
