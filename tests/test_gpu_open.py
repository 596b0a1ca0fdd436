"""Open (outflow) axes on the GPU against the oracle: zero-gradient ghost
fields, sampling clamped to the domain, no wrap, the outflow mask, deposits
folded onto the edge cells, and removal of the particles that left by
part_compact.  Tolerances as in the periodic parity tests (FP64: 1e-12
relative per step; outflow flags bit-exact; mixed form: 1e-6 cell).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2602_23434_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2602_23434_b300 import _lib as P  # noqa: E402


def _host(t):
    return t.detach().cpu().numpy()


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype).cuda()


def _pdiff(a, b):
    d = a - b
    return d - 2.0 * np.round(d / 2.0)


def _near_faces(dim, N, seed, opn):
    """Particles crowded near the open faces, moving fast (|v| close to 1)."""
    x, u, w, ids = synth.particles(dim, None, N, seed, u_th=2.0)
    rng = np.random.default_rng(seed)
    for a in range(dim):
        if opn[a]:
            k = rng.random(N) < 0.5
            x[a, k] = np.where(rng.random(k.sum()) < 0.5, rng.uniform(-1.0, -0.9, k.sum()),
                               rng.uniform(0.9, 0.999999, k.sum()))
    w = rng.uniform(0.5, 2.0, N)
    return x, u, w, ids


@pytest.mark.parametrize("dim,n,opn", [(3, 20, (1, 0, 1)), (2, 40, (1, 1, 0)), (3, 16, (0, 1, 0))])
@pytest.mark.parametrize("shape", [P.TSC, P.CIC])
def test_open_boris_step_deposit_and_outflow(dim, n, opn, shape):
    og = O.make_grid(dim, (n, n, n), open_axes=opn)
    pg = P.make_grid(dim, n, open_axes=opn)
    N = n ** dim * 4 + 3
    x, u, w, ids = _near_faces(dim, N, 17 + n, opn)
    f = synth.em_fields(dim, n, 19, v_rms=0.05).reshape(6, -1)
    p = P.Part(pg, P.FP64, shape, P.BORIS, capacity=N)
    p.set_fields(_dev(f))
    xd, ud, wd = _dev(x), _dev(u), _dev(w)
    idd = torch.as_tensor(ids.astype(np.int64)).cuda()
    out = torch.full((N,), 7, dtype=torch.uint8, device="cuda")
    p.bind(N, xd, u=ud, w=wd, ids=idd)
    p.set_outflow(out)
    p.enable_deposit(True)
    p.sort()
    p.sync()
    x0, u0, w0 = _host(xd), _host(ud), _host(wd)
    dt = 0.9 * 2.0 / n
    p.gather_push(1.0, dt, 1)
    dep = torch.empty((3, f.shape[1]), dtype=torch.float64, device="cuda")
    p.deposit(dep)
    p.sync()
    xr, ur, F, xo = O.boris_step(og, shape, f, x0, u0, w0, 1.0, dt, True)
    assert np.max(np.abs(_pdiff(_host(xd), xr))) <= 2e-12
    assert np.max(np.abs(_host(ud) - ur) / np.maximum(np.abs(ur), 1e-3)) <= 1e-12
    flags = O.outside(og, xr)
    assert 0 < int(flags.sum()) < N
    assert np.array_equal(_host(out), flags)
    dref = O.deposit(og, shape, xo, F)
    dabs = O.deposit(og, shape, xo, np.abs(F))
    assert np.max(np.abs(_host(dep) - dref) / np.maximum(dabs, 1e-300)) <= 1e-12
    assert np.allclose(_host(dep).sum(axis=1), F.sum(axis=1), rtol=1e-12, atol=1e-12)


def test_open_fused_steps_stop_at_the_face():
    """Particle-order kernel, 6 fused steps: a particle that leaves is not
    advanced further (oracle stepped once per step, freezing the same way)."""
    dim, n, opn = 3, 16, (1, 1, 0)
    og = O.make_grid(dim, (n, n, n), open_axes=opn)
    pg = P.make_grid(dim, n, open_axes=opn)
    N = 3001
    x, u, w, ids = _near_faces(dim, N, 5, opn)
    f = synth.em_fields(dim, n, 6, v_rms=0.05).reshape(6, -1)
    p = P.Part(pg, P.FP64, P.TSC, P.BORIS, capacity=N)
    p.set_fields(_dev(f))
    xd, ud = _dev(x), _dev(u)
    out = torch.zeros(N, dtype=torch.uint8, device="cuda")
    p.bind(N, xd, u=ud)
    p.set_outflow(out)
    dt = 0.4 * 2.0 / n
    p.gather_push(1.0, dt, 6)
    p.sync()
    xr, ur = x.copy(), u.copy()
    for _ in range(6):
        live = O.outside(og, xr) == 0
        xn, un, _, _ = O.boris_step(og, P.TSC, f, xr[:, live], ur[:, live], None, 1.0, dt)
        xr[:, live], ur[:, live] = xn, un
    assert np.max(np.abs(_pdiff(_host(xd), xr))) <= 1e-11
    assert np.array_equal(_host(out), O.outside(og, xr))
    assert int(_host(out).sum()) > 50


def test_open_outflow_then_compact_then_resort():
    """Push, remove the particles that left (part_compact with the mask),
    sort the survivors and push again, against the oracle doing the same."""
    dim, n, opn = 3, 16, (1, 0, 0)
    og = O.make_grid(dim, (n, n, n), open_axes=opn)
    pg = P.make_grid(dim, n, open_axes=opn)
    N = n ** 3 * 3 + 1
    x, u, w, ids = _near_faces(dim, N, 8, opn)
    f = synth.em_fields(dim, n, 2, v_rms=0.05).reshape(6, -1)
    p = P.Part(pg, P.FP64, P.TSC, P.BORIS, capacity=N)
    p.set_fields(_dev(f))
    xd, ud = _dev(x), _dev(u)
    idd = torch.as_tensor(ids.astype(np.int64)).cuda()
    out = torch.zeros(N, dtype=torch.uint8, device="cuda")
    p.bind(N, xd, u=ud, ids=idd)
    p.set_outflow(out)
    dt = 0.8 * 2.0 / n
    xr, ur, ir = x.copy(), u.copy(), ids.astype(np.int64)
    for _ in range(3):
        p.sort()
        perm = O.stable_sort(O.keys(og, p.brick, xr))
        xr, ur, ir = xr[:, perm], ur[:, perm], ir[perm]
        p.gather_push(1.0, dt, 1)
        xr, ur, _, _ = O.boris_step(og, P.TSC, f, xr, ur, None, 1.0, dt)
        p.sync()
        m = O.outside(og, xr)
        assert np.array_equal(_host(out)[: xr.shape[1]], m)
        nn = p.compact(out)
        k, src = O.compact_map(m)
        assert nn == k
        xr, ur, ir = xr[:, src], ur[:, src], ir[src]
        p.set_outflow(out)                     # the mask stays bound; re-set for clarity
    p.sync()
    k = xr.shape[1]
    assert k < N
    assert np.array_equal(_host(idd)[:k], ir)
    xg = _host(xd).reshape(-1)[: 3 * k].reshape(3, k)
    assert np.max(np.abs(_pdiff(xg, xr))) <= 1e-11
    assert np.all(O.outside(og, xg) == 0)


def test_open_mixed_step_and_outflow():
    """Mixed form on an open-x grid: one sorted step with deposit; position
    within 1e-6 cell of the FP64 oracle, outflow flags equal except within
    1e-5 cell of a face (the flag is decided in f32 there)."""
    dim, n, opn = 3, 20, (1, 0, 0)
    og = O.make_grid(dim, (n, n, n), open_axes=opn)
    pg = P.make_grid(dim, n, open_axes=opn)
    N = n ** 3 * 4 + 3
    x, u, _, ids = _near_faces(dim, N, 23, opn)
    dx = 2.0 / n
    j = np.minimum(np.floor((x + 1.0) / dx), n - 1).astype(np.int64)
    off = ((x + 1.0) / dx - j - 0.5).astype(np.float32)
    x = -1.0 + (j + 0.5 + off.astype(np.float64)) * dx        # exactly representable
    cell = ((j[2] * n + j[1]) * n + j[0]).astype(np.int32)
    uf = np.concatenate([u.astype(np.float32), np.zeros((3, N), dtype=np.float32)])  # hi, lo
    f = synth.em_fields(dim, n, 29, v_rms=0.05).reshape(6, -1)
    p = P.Part(pg, P.MIXED, P.TSC, P.BORIS, capacity=N)
    p.set_fields(torch.as_tensor(f.astype(np.float32)).cuda())
    cd, od, ud = (torch.as_tensor(a).cuda() for a in (cell, off, uf))
    out = torch.zeros(N, dtype=torch.uint8, device="cuda")
    p.bind(N, cd, off=od, u=ud)
    p.set_outflow(out)
    p.sort()
    p.sync()
    c0, o0, u0 = _host(cd), _host(od), _host(ud)
    jj = np.stack([c0 % n, (c0 // n) % n, c0 // (n * n)])
    x0 = -1.0 + (jj + 0.5 + o0.astype(np.float64)) * dx
    dt = 0.9 * dx
    p.gather_push(1.0, dt, 1)
    p.sync()
    xr, ur, _, _ = O.boris_step(og, P.TSC, f.astype(np.float32).astype(np.float64), x0,
                                u0[:3].astype(np.float64) + u0[3:].astype(np.float64), None,
                                1.0, dt)
    flags = O.outside(og, xr)
    got = _host(out)
    near = np.abs(np.minimum(np.abs(xr[0] - 1.0), np.abs(xr[0] + 1.0))) < 1e-5 * dx
    assert np.array_equal(got[~near], flags[~near]) and flags.sum() > 0
    live = (flags == 0) & ~near
    c1, o1 = _host(cd), _host(od)
    j1 = np.stack([c1 % n, (c1 // n) % n, c1 // (n * n)])
    xg = -1.0 + (j1 + 0.5 + o1.astype(np.float64)) * dx
    assert np.max(np.abs(_pdiff(xg[:, live], xr[:, live])) / dx) <= 1e-6


def test_open_shock_test_with_outflow_and_removal():
    """Sec. 4.1.2 with its outflow x boundary: LPs advected through the shock;
    those leaving at x = +1 are removed each step; flags, positions and
    spectra against the oracle doing the same."""
    n, N, nb = 40, 400, 32
    r = 40.0 / 11.0
    og = O.make_grid(2, (n, n, n), open_axes=(1, 0, 0))
    pg = P.make_grid(2, n, open_axes=(1, 0, 0))
    xc = -1.0 + (np.arange(n) + 0.5) * (2.0 / n)
    down = np.broadcast_to(xc[None, :] > 0.0, (n, n)).reshape(-1)
    f7 = np.zeros((7, n * n))
    f7[0] = np.where(down, 0.1 / r, 0.1)
    f7[3] = np.where(down, 50.0 * r, 50.0)
    f7[4] = 1.0
    rng = np.random.default_rng(9)
    x = np.zeros((3, N))
    x[0] = rng.uniform(0.3, 0.99, N)            # downstream, drifting out through x = +1
    x[1] = rng.uniform(-1.0, 1.0, N)
    e1, c1 = O.init_spectrum(nb, 1e2, 1e4, 9.0, 1e-6)
    eng, chi = np.repeat(e1[:, None], N, 1), np.repeat(c1[:, None], N, 1)
    no = np.array([O.gather(og, P.TSC, f7[3:4], x[:, i])[0] for i in range(N)])
    p = P.Part(pg, P.FP64, P.TSC, P.LP_RK2, capacity=N, nbins=nb)
    p.set_fields(_dev(f7))
    xd, chid, engd, nod = _dev(x), _dev(chi), _dev(eng), _dev(no)
    idd = torch.as_tensor(np.arange(N, dtype=np.int64)).cuda()
    out = torch.zeros(N, dtype=torch.uint8, device="cuda")
    p.bind(N, xd, ids=idd, chi=chid, eng=engd, n_old=nod)
    p.set_outflow(out)
    ir = np.arange(N)
    dt = 2.0 * (2.0 / n) / (0.1 / r)                # two cells of downstream flow per step
    for _ in range(6):
        p.gather_push(0.0, dt, 1)
        p.spec_update(dt, 1e-6, 0.0)
        x, nn, b2, gm = O.lp_rk2_step(og, P.TSC, f7[:3], f7[3:4], f7[4:], x, dt)
        chi, eng, no = O.spec_update(chi, eng, no, nn, b2, gm, dt, 1e-6)
        p.sync()
        m = O.outside(og, x)
        assert np.array_equal(_host(out)[: x.shape[1]], m)
        k = p.compact(out)
        kk, src = O.compact_map(m)
        assert k == kk
        x, chi, eng, no, ir = x[:, src], chi[:, src], eng[:, src], no[src], ir[src]
    p.sync()
    k = x.shape[1]
    assert 0 < k < N
    assert np.array_equal(_host(idd)[:k], ir)
    assert np.max(np.abs(_host(xd).reshape(-1)[: 3 * k].reshape(3, k) - x)) <= 1e-12
    cg = _host(chid).reshape(-1)[: nb * k].reshape(nb, k)
    assert np.max(np.abs(cg - chi) / np.abs(chi)) <= 1e-11


def test_open_errors():
    pg = P.make_grid(3, 8)
    p = P.Part(pg, P.FP64, P.TSC, P.BORIS, capacity=4)
    m = torch.zeros(4, dtype=torch.uint8, device="cuda")
    with pytest.raises(P.PartError):
        p.set_outflow(m)                         # periodic grid: no open axis
    import ctypes as C
    po = P.Part(P.make_grid(3, 8, open_axes=(1, 0, 0)), P.MIXED, P.TSC, P.BORIS, capacity=4)
    po.set_fields(torch.zeros((6, 512), dtype=torch.float32, device="cuda"))
    L = P.lib()
    db, hb = C.c_size_t(), C.c_size_t()
    assert L.part_server_sizes(1, 16, C.byref(db), C.byref(hb)) == 0
    ws = torch.empty(db.value, dtype=torch.uint8, device="cuda")
    stage = torch.empty(hb.value, dtype=torch.uint8, pin_memory=True)
    arr = (C.c_void_p * 1)(po.ctx.value)
    h = C.c_void_p()
    s = torch.cuda.Stream()
    rc = L.part_server_init(C.byref(h), arr, 1, 16, C.c_void_p(ws.data_ptr()), db.value,
                            C.c_void_p(stage.data_ptr()), hb.value, C.c_void_p(s.cuda_stream),
                            256, 4)
    assert rc == 6 and b"periodic" in L.part_last_error(None)   # PART_EUNSUPPORTED


def test_open_inflow_injection_and_outflow_removal():
    """An open-x run whose particle count is kept up at run time (Sec. 3.2):
    every step new particles are injected at the inflow face, the set is
    sorted and pushed, and those that left through any open face are removed
    by part_compact with the outflow mask.  The oracle does the same
    (concatenate, stable sort, Boris step, outside flags, compaction map);
    flags and ids bit-exact, positions within 1e-12 per step."""
    dim, n, opn = 3, 16, (1, 0, 0)
    og = O.make_grid(dim, (n, n, n), open_axes=opn)
    pg = P.make_grid(dim, n, open_axes=opn)
    C = n ** 3 * 3
    N0, K = n ** 3 * 2, 900
    x, u, _, ids = _near_faces(dim, N0, 31, opn)
    f = synth.em_fields(dim, n, 4, v_rms=0.05).reshape(6, -1)
    p = P.Part(pg, P.FP64, P.TSC, P.BORIS, capacity=C)
    p.set_fields(_dev(f))
    xb = torch.zeros(3 * C, dtype=torch.float64, device="cuda")
    ub = torch.zeros(3 * C, dtype=torch.float64, device="cuda")
    ib = torch.zeros(C, dtype=torch.int64, device="cuda")
    xb[: 3 * N0] = _dev(x).reshape(-1)
    ub[: 3 * N0] = _dev(u).reshape(-1)
    ib[:N0] = torch.as_tensor(ids.astype(np.int64)).cuda()
    out = torch.zeros(C, dtype=torch.uint8, device="cuda")
    p.bind(N0, xb, u=ub, ids=ib)
    p.set_outflow(out)
    dt = 0.8 * 2.0 / n
    xr, ur, ir = x.copy(), u.copy(), ids.astype(np.int64)
    rng = np.random.default_rng(37)
    next_id = N0
    for step in range(4):
        # inflow: K particles in the first cell layer, moving in +x
        xn = np.stack([rng.uniform(-1.0, -1.0 + 2.0 / n, K), rng.uniform(-1.0, 1.0, K),
                       rng.uniform(-1.0, 1.0, K)])
        un = rng.normal(0.0, 0.5, (3, K))
        un[0] = np.abs(un[0])
        idn = np.arange(next_id, next_id + K, dtype=np.int64)
        next_id += K
        p.inject(K, _dev(xn), u=_dev(un), ids=torch.as_tensor(idn).cuda())
        xr, ur, ir = np.concatenate([xr, xn], 1), np.concatenate([ur, un], 1), \
            np.concatenate([ir, idn])
        p.sort()
        perm = O.stable_sort(O.keys(og, p.brick, xr))
        xr, ur, ir = xr[:, perm], ur[:, perm], ir[perm]
        p.gather_push(1.0, dt, 1)
        xr, ur, _, _ = O.boris_step(og, P.TSC, f, xr, ur, None, 1.0, dt)
        p.sync()
        m = O.outside(og, xr)
        assert np.array_equal(_host(out)[: xr.shape[1]], m)
        nn = p.compact(out)
        k, src = O.compact_map(m)
        assert nn == k and 0 < m.sum()
        xr, ur, ir = xr[:, src], ur[:, src], ir[src]
        p.sync()
        assert np.array_equal(_host(ib)[:k], ir)
        xg = _host(xb)[: 3 * k].reshape(3, k)
        assert np.max(np.abs(_pdiff(xg, xr))) <= 1e-12 * 2.0 * (step + 1)
