"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (FP64 path): cell keys, sort permutation and cell_start bit-exact;
particle state 1e-12 relative per step, max(|ref|, scale) normalised;
deposit 1e-12 relative to the sum of |contributions| to the cell; deposit
run-to-run bitwise.  Differences come only from FMA contraction and the
order of sums, so 1e-12 leaves three orders of magnitude of margin.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2602_23434_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2602_23434_b300 import _lib as P  # noqa: E402  (loads libpart.so lazily)


def _grids(dim, n):
    return O.make_grid(dim, (n, n, n)), P.make_grid(dim, n)


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype).cuda()


def _host(t):
    return t.detach().cpu().numpy()


def _pdiff(a, b, L=2.0):
    d = a - b
    return d - L * np.round(d / L)


def _rel(gpu, ref, scale):
    return np.max(np.abs(gpu - ref) / np.maximum(np.abs(ref), scale)) if gpu.size else 0.0


CASES = [(3, 20, 8), (2, 40, 16)]     # (dim, n, particles per cell): partial bricks


@pytest.mark.parametrize("dim,n,ppc", CASES + [(3, 8, 3), (3, 5, 2)])
def test_sort_bit_exact(dim, n, ppc):
    og, pg = _grids(dim, n)
    G = n ** dim
    N = G * ppc + 7                         # ragged tail
    x, u, w, ids = synth.particles(dim, None, N, 11 + n)
    p = P.Part(pg, P.FP64, P.TSC, P.BORIS, capacity=N)
    xd, ud, wd, idd = _dev(x), _dev(u), _dev(w), torch.as_tensor(ids.astype(np.int64)).cuda()
    p.bind(N, xd, u=ud, w=wd, ids=idd)
    p.sort()
    cs = _host(p.cell_start())
    p.sync()
    keys = O.keys(og, p.brick, x)
    perm = O.stable_sort(keys)
    assert np.array_equal(_host(idd), ids[perm].astype(np.int64))
    assert np.array_equal(_host(xd), x[:, perm])
    assert np.array_equal(_host(ud), u[:, perm])
    assert np.array_equal(cs, O.cell_start(p.nkeys, keys[perm]).astype(np.int64))


def _face_positions(rng, N, n, xmin, dx):
    """Coordinates on the cell faces xmin + j dx (j = 0..n, in FP64) moved by
    -3..3 ulp, at the upper domain edge minus one ulp, and inside cells."""
    j = rng.integers(0, n + 1, N)
    x = xmin + j * dx
    k = rng.integers(-3, 4, N)
    for _ in range(3):
        up, dn = k > 0, k < 0
        x = np.where(up, np.nextafter(x, np.inf), np.where(dn, np.nextafter(x, -np.inf), x))
        k = k - up + dn
    xmax = xmin + n * dx
    x = np.where(x >= xmax, np.nextafter(xmax, -np.inf), x)
    x = np.where(x < xmin, xmin, x)
    inside = rng.random(N) < 0.3
    return np.where(inside, xmin + rng.uniform(0.0, n, N) * dx, x)


@pytest.mark.parametrize("n,xmin", [(16, (-1.0, -1.0, -1.0)), (20, (-1.0, -1.0, -1.0)),
                                    (24, (3.7, -10.25, 0.5))])
def test_sort_keys_at_cell_faces(n, xmin):
    """Cell keys of positions on and a few ulp around every cell face (dx = 0.125
    exact, 0.1 inexact, an offset domain): the full sort's keys and, after a
    push that leaves the positions where they are, the incremental sort's,
    both bit-exact against the oracle.  The key passes take the floor from an
    f32 image and fall back to the FP64 expression near faces, so this is
    where they could differ."""
    dim, L = 3, 2.0
    og = O.make_grid(dim, (n, n, n), xmin=xmin, dx=(L / n,) * 3)
    pg = P.make_grid(dim, n, xmin=xmin, L=(L,) * 3)
    rng = np.random.default_rng(n)
    N = 20000
    x = np.stack([_face_positions(rng, N, n, xmin[a], L / n) for a in range(3)])
    u = np.zeros((3, N))
    ids = np.arange(N, dtype=np.int64)
    p = P.Part(pg, P.FP64, P.TSC, P.BORIS, capacity=N)
    p.set_fields(_dev(np.zeros((6, n ** 3))))
    xd, ud, idd = _dev(x), _dev(u), torch.as_tensor(ids).cuda()
    p.bind(N, xd, u=ud, ids=idd)
    p.sort()
    cs = _host(p.cell_start())
    p.sync()
    keys = O.keys(og, p.brick, x)
    perm = O.stable_sort(keys)
    assert np.array_equal(_host(idd), ids[perm])
    assert np.array_equal(cs, O.cell_start(p.nkeys, keys[perm]).astype(np.int64))
    # u = 0: the push leaves every position as it is; the next sort is incremental
    p.gather_push(1.0, 0.5 * L / n, 1)
    p.sync()
    xb, ib = _host(xd).copy(), _host(idd).copy()
    assert np.array_equal(xb, x[:, perm])
    p.sort()
    cs = _host(p.cell_start())
    p.sync()
    keys = O.keys(og, p.brick, xb)
    perm = O.stable_sort(keys)
    assert np.array_equal(_host(idd), ib[perm])
    assert np.array_equal(cs, O.cell_start(p.nkeys, keys[perm]).astype(np.int64))


@pytest.mark.parametrize("N", [0, 1, 31, 33, 4096, 4097])
def test_sort_edge_counts(N):
    og, pg = _grids(3, 16)
    x, u, w, ids = synth.particles(3, None, max(N, 1), 5)
    x, u, ids = x[:, :N].copy(), u[:, :N].copy(), ids[:N].copy()
    p = P.Part(pg, P.FP64, P.TSC, P.BORIS, capacity=max(N, 1))
    xd, ud = _dev(x if N else np.zeros((3, 1))), _dev(u if N else np.zeros((3, 1)))
    idd = torch.as_tensor(ids.astype(np.int64) if N else np.zeros(1, np.int64)).cuda()
    p.bind(N, xd, u=ud, ids=idd)
    p.sort()
    cs = _host(p.cell_start())
    p.sync()
    keys = O.keys(og, p.brick, x) if N else np.zeros(0, np.uint32)
    perm = O.stable_sort(keys)
    if N:
        assert np.array_equal(_host(idd)[:N], ids[perm].astype(np.int64))
    assert np.array_equal(cs, O.cell_start(p.nkeys, keys[perm]).astype(np.int64))


def _boris_case(dim, n, ppc, shape, seed, turbulent=True):
    og, pg = _grids(dim, n)
    G = n ** dim
    N = G * ppc + 13
    if turbulent:
        f = synth.em_fields(dim, n, seed, v_rms=0.05)
    else:
        f = synth.uniform_em_fields(dim, n, B=(0.0, 0.0, 1.0))
    x, u, w, ids = synth.particles(dim, None, N, seed + 1, u_th=0.3)
    w = np.random.default_rng(seed).uniform(0.5, 2.0, N)
    return og, pg, f.reshape(6, -1), x, u, w, ids, N


@pytest.mark.parametrize("dim,n,ppc", CASES)
@pytest.mark.parametrize("shape", [P.TSC, P.CIC])
def test_boris_push_and_deposit_fp64(dim, n, ppc, shape):
    og, pg, f, x, u, w, ids, N = _boris_case(dim, n, ppc, shape, 21)
    qm, dt = 1.0, 0.5 * (2.0 / n)
    p = P.Part(pg, P.FP64, shape, P.BORIS, capacity=N)
    p.set_fields(_dev(f))
    xd, ud, wd = _dev(x), _dev(u), _dev(w)
    idd = torch.as_tensor(ids.astype(np.int64)).cuda()
    p.bind(N, xd, u=ud, w=wd, ids=idd)
    p.enable_deposit(True)
    p.sort()
    p.sync()
    xs, us, ws = _host(xd), _host(ud), _host(wd)      # sorted input state
    p.gather_push(qm, dt, 1)
    out = torch.empty((3, og.n[0] * og.n[1] * og.n[2]), dtype=torch.float64, device="cuda")
    p.deposit(out)
    p.sync()
    xr, ur, F, xo = O.boris_step(og, shape, f, xs, us, ws, qm, dt, True)
    assert np.max(np.abs(_pdiff(_host(xd), xr))) <= 1e-12 * 2.0
    assert _rel(_host(ud), ur, np.max(np.abs(ur))) <= 1e-12
    dref = O.deposit(og, shape, xo, F)
    dabs = O.deposit(og, shape, xo, np.abs(F))
    dg = _host(out)
    assert np.max(np.abs(dg - dref) / np.maximum(dabs, 1e-300)) <= 1e-12
    # bitwise reproducible: same inputs, same bits
    xd2, ud2 = _dev(xs), _dev(us)
    p.bind(N, xd2, u=ud2, w=_dev(ws))
    p.sort()
    p.gather_push(qm, dt, 1)
    out2 = torch.empty_like(out)
    p.deposit(out2)
    p.sync()
    assert torch.equal(out, out2)
    assert torch.equal(xd, xd2) and torch.equal(ud, ud2)


def test_boris_uniform_field_config_shape():
    """2D 64^2, B = z, E = 0, fused multi-step particle-order kernel vs 20
    oracle steps (the 2D uniform-field workload, scaled down in steps)."""
    og, pg, f, x, u, w, ids, N = _boris_case(2, 64, 16, P.TSC, 31, turbulent=False)
    qm, dt, steps = 1.0, 0.1, 20
    p = P.Part(pg, P.FP64, P.TSC, P.BORIS, capacity=N)
    p.set_fields(_dev(f))
    xd, ud = _dev(x), _dev(u)
    p.bind(N, xd, u=ud)
    p.gather_push(qm, dt, steps)
    p.sync()
    xr, ur = x, u
    for _ in range(steps):
        xr, ur, _, _ = O.boris_step(og, P.TSC, f, xr, ur, None, qm, dt)
    assert np.max(np.abs(_pdiff(_host(xd), xr))) <= 1e-12 * 2.0 * steps
    assert _rel(_host(ud), ur, np.max(np.abs(ur))) <= 1e-12 * steps
    # |u| conserved by the rotation (E = 0)
    assert np.max(np.abs(np.linalg.norm(_host(ud), axis=0) / np.linalg.norm(u, axis=0) - 1)) \
        < 1e-13


@pytest.mark.parametrize("dim,n", [(3, 20), (2, 40)])
def test_lp_step_and_spectra(dim, n):
    og, pg = _grids(dim, n)
    vel, rho, B = synth.fluid_snapshot(dim, n, 41, v_rms=0.05)
    f7 = np.concatenate([vel, rho, B]).reshape(7, -1)
    N = n ** dim * 2 + 5
    nb = 128
    p = P.Part(pg, P.FP64, P.TSC, P.LP_RK2, capacity=N, nbins=nb)
    p.set_fields(_dev(f7))
    xd = torch.zeros((3, N), dtype=torch.float64, device="cuda")
    chi = torch.zeros((nb, N), dtype=torch.float64, device="cuda")
    eng = torch.zeros_like(chi)
    nold = torch.zeros(N, dtype=torch.float64, device="cuda")
    p.bind(N, xd, chi=chi, eng=eng, n_old=nold)
    p.init_particles(77, 0.0, 1.0, 1e6, 2.2, 1e-6)
    p.sync()
    # initialisation vs the oracle
    xo, _, _, _ = O.init_particles(og, N, 77, 0.0)
    assert np.array_equal(_host(xd), xo)
    e1, c1 = O.init_spectrum(nb, 1.0, 1e6, 2.2, 1e-6)
    assert _rel(_host(eng), e1[:, None] * np.ones(N), 0) <= 1e-14
    assert _rel(_host(chi), c1[:, None] * np.ones(N), 0) <= 1e-13
    r0 = np.array([O.gather(og, P.TSC, rho.reshape(1, -1), xo[:, i])[0] for i in range(N)])
    assert _rel(_host(nold), r0, 0) <= 1e-13
    # one RK2 step + spectral update
    dt, c0 = 0.5 * 2.0 / n, 2e-3
    x0, ch0, en0, no0 = _host(xd), _host(chi), _host(eng), _host(nold)
    p.gather_push(0.0, dt, 1)
    p.spec_update(dt, c0, 0.1)
    p.sync()
    xr, n_new, b2m, gam = O.lp_rk2_step(og, P.TSC, vel.reshape(3, -1), rho.reshape(1, -1),
                                        B.reshape(3, -1), x0, dt)
    assert np.max(np.abs(_pdiff(_host(xd), xr))) <= 1e-12 * 2.0
    chr_, enr, nor = O.spec_update(ch0, en0, no0, n_new, b2m, gam, dt, c0, 0.1)
    assert _rel(_host(eng), enr, 0) <= 1e-12
    assert _rel(_host(chi), chr_, 0) <= 1e-12
    assert _rel(_host(nold), nor, 0) <= 1e-12


def test_lp_spectra_across_flushes_and_injection():
    """Several LP steps with no sync in between (the spectra stay in the
    library's 1/eps, chi eps^2 form), a flush in the middle, then an injection
    (which brings them back first) and more steps: chi and eps after the final
    sync against the oracle's (chi, eps) steps, 1e-12 relative."""
    dim, n, nb = 3, 16, 32
    og, pg = _grids(dim, n)
    vel, rho, B = synth.fluid_snapshot(dim, n, 43, v_rms=0.05)
    f7 = np.concatenate([vel, rho, B]).reshape(7, -1)
    N0, K = 3000, 200
    p = P.Part(pg, P.FP64, P.TSC, P.LP_RK2, capacity=N0 + K, nbins=nb)
    p.set_fields(_dev(f7))
    xd = torch.zeros((3, N0 + K), dtype=torch.float64, device="cuda")
    chi = torch.zeros((nb, N0 + K), dtype=torch.float64, device="cuda")
    eng = torch.zeros_like(chi)
    nold = torch.zeros(N0 + K, dtype=torch.float64, device="cuda")
    p.bind(N0, xd, chi=chi, eng=eng, n_old=nold)
    p.init_particles(5, 0.0, 1.0, 1e6, 2.2, 1e-6)
    p.sync()

    def plain(N):
        v = lambda t, r: _host(t).reshape(-1)[: r * N].reshape(r, N).copy()  # noqa: E731
        return v(xd, 3), v(chi, nb), v(eng, nb), _host(nold)[:N].copy()

    x, ch, en, no = plain(N0)
    dt, c0 = 0.5 * 2.0 / n, 3e-3

    def steps(k, x, ch, en, no):
        for _ in range(k):
            p.gather_push(0.0, dt, 1)
            p.spec_update(dt, c0, 0.05)
            x, nn, b2, gm = O.lp_rk2_step(og, P.TSC, vel.reshape(3, -1), rho.reshape(1, -1),
                                          B.reshape(3, -1), x, dt)
            ch, en, no = O.spec_update(ch, en, no, nn, b2, gm, dt, c0, 0.05)
        return x, ch, en, no

    x, ch, en, no = steps(3, x, ch, en, no)
    p.flush()
    x, ch, en, no = steps(2, x, ch, en, no)
    rng = np.random.default_rng(9)
    xn = rng.uniform(-1.0, 1.0, (3, K))
    e1, c1 = O.init_spectrum(nb, 1.0, 1e6, 2.2, 1e-6)
    cn = np.repeat(c1[:, None], K, 1) * rng.uniform(0.5, 2.0, (1, K))
    en_ = np.repeat(e1[:, None], K, 1)
    nn0 = np.array([O.gather(og, P.TSC, rho.reshape(1, -1), xn[:, i])[0] for i in range(K)])
    p.inject(K, x=_dev(xn), chi=_dev(cn), eng=_dev(en_), n_old=_dev(nn0))
    N = N0 + K
    x, ch = np.concatenate([x, xn], 1), np.concatenate([ch, cn], 1)
    en, no = np.concatenate([en, en_], 1), np.concatenate([no, nn0])
    x, ch, en, no = steps(3, x, ch, en, no)
    p.sync()
    xg, cg, eg, ng = plain(N)
    assert np.max(np.abs(_pdiff(xg, x))) <= 1e-12 * 2.0
    assert _rel(eg, en, 0) <= 1e-12
    assert _rel(cg, ch, 0) <= 1e-12
    assert _rel(ng, no, 0) <= 1e-12


def test_init_particles_fp64_and_mixed():
    og, pg = _grids(3, 24)
    N = 50001
    p = P.Part(pg, P.FP64, P.TSC, P.BORIS, capacity=N)
    xd = torch.zeros((3, N), dtype=torch.float64, device="cuda")
    ud = torch.zeros_like(xd)
    wd = torch.zeros(N, dtype=torch.float64, device="cuda")
    idd = torch.zeros(N, dtype=torch.int64, device="cuda")
    p.bind(N, xd, u=ud, w=wd, ids=idd)
    p.init_particles(1235, 0.1)
    p.sync()
    xo, uo, wo, io = O.init_particles(og, N, 1235, 0.1)
    assert np.array_equal(_host(xd), xo)           # positions decide cells: bit-exact
    assert _rel(_host(ud), uo, 0.1) <= 1e-14
    assert np.array_equal(_host(wd), wo) and np.array_equal(_host(idd), io.astype(np.int64))
    pm = P.Part(pg, P.MIXED, P.TSC, P.BORIS, capacity=N)
    cell = torch.zeros(N, dtype=torch.int32, device="cuda")
    off = torch.zeros((3, N), dtype=torch.float32, device="cuda")
    uf = torch.zeros((6, N), dtype=torch.float32, device="cuda")   # compensated pair
    pm.bind(N, cell, off=off, u=uf)
    pm.init_particles(1235, 0.1)
    pm.sync()
    c = _host(cell).astype(np.int64)
    j = np.stack([c % 24, (c // 24) % 24, c // 576])
    pos = -1.0 + (j + 0.5 + _host(off)) * (2.0 / 24)
    assert np.max(np.abs(pos - xo)) <= 2.0 / 24 * 6e-8
    assert np.all(np.abs(_host(off)) <= 0.5)
    assert _rel(_host(uf)[:3].astype(np.float64), uo, 0.1) <= 1e-6
    # the pair carries the draw beyond f32: hi + lo is u to ~2^-48 relative
    u_pair = _host(uf)[:3].astype(np.float64) + _host(uf)[3:].astype(np.float64)
    assert _rel(u_pair, uo, 0.1) <= 1e-13


def test_bounded_wait_times_out_and_the_context_survives():
    """Failure detection without a fault: a device wait that nothing
    completes gives up after its limit, the next part_sync reports
    PART_ETIMEOUT (and clears it), and the same context then steps and
    deposits like a fresh one."""
    import time
    og, pg, f, x, u, w, ids, N = _boris_case(3, 16, 4, P.TSC, 5)
    qm, dt = 1.0, 0.5 * (2.0 / 16)
    p = P.Part(pg, P.FP64, P.TSC, P.BORIS, capacity=N)
    p.selftest_wait(10_000_000, True)                 # completed wait: no error
    p.sync()
    t0 = time.perf_counter()
    p.selftest_wait(20_000_000, False)                # nothing arrives: 20 ms limit
    with pytest.raises(P.PartError) as e:
        p.sync()
    assert e.value.name == "PART_ETIMEOUT"
    assert time.perf_counter() - t0 >= 0.02
    p.sync()                                          # latched once, then cleared
    for bad in (0, -1, 10 ** 11):
        with pytest.raises(P.PartError):
            p.selftest_wait(bad, False)
    p.set_fields(_dev(f))
    xd, ud, wd = _dev(x), _dev(u), _dev(w)
    p.bind(N, xd, u=ud, w=wd)
    p.enable_deposit(True)
    p.sort()
    p.sync()
    xs, us, ws = _host(xd), _host(ud), _host(wd)
    p.gather_push(qm, dt, 1)
    out = torch.empty((3, 16 ** 3), dtype=torch.float64, device="cuda")
    p.deposit(out)
    p.sync()
    xr, ur, F, xo = O.boris_step(og, P.TSC, f, xs, us, ws, qm, dt, True)
    assert np.max(np.abs(_pdiff(_host(xd), xr))) <= 1e-12 * 2.0
    assert _rel(_host(ud), ur, np.max(np.abs(ur))) <= 1e-12
    dref = O.deposit(og, P.TSC, xo, F)
    dabs = O.deposit(og, P.TSC, xo, np.abs(F))
    assert np.max(np.abs(_host(out) - dref) / np.maximum(dabs, 1e-300)) <= 1e-12


def test_misaligned_arrays_refused_on_the_host():
    """A caller array not aligned to its element size would fault in a
    kernel; every entry point that takes one refuses it before any launch."""
    import ctypes as C
    og, pg = _grids(3, 8)
    N = 100
    p = P.Part(pg, P.FP64, P.TSC, P.BORIS, capacity=N)
    raw = torch.zeros(8 * 6 * N + 64, dtype=torch.uint8, device="cuda")
    good = raw.data_ptr() + 64 - raw.data_ptr() % 64
    L = P.lib()
    bad = C.c_void_p(good + 4)
    ok = C.c_void_p(good)
    l0 = p.launches()
    assert L.part_bind_particles(p.ctx, N, bad, None, ok, None, None, None, None, None) != 0
    assert L.part_bind_particles(p.ctx, N, ok, None, bad, None, None, None, None, None) != 0
    assert L.part_set_fields(p.ctx, bad, 6, P.FP64) != 0
    assert L.part_sort_fp64_noalloc(C.byref(pg), N, bad, ok, None, None, ok, None) != 0
    assert p.launches() == l0
    p.sync()


def test_pinned_host_fields_and_output_and_pageable_refused():
    """Fields read from pinned host memory and the deposit written into pinned
    host memory give the same bits as device buffers.  Pageable host memory is
    refused on the host before any launch: first through bind (which launches
    nothing on the arrays in any case), then the fields and the output."""
    og, pg, f, x, u, w, ids, N = _boris_case(3, 16, 4, P.TSC, 9)
    qm, dt = 1.0, 0.5 * (2.0 / 16)
    outs = []
    for host in (False, True):
        p = P.Part(pg, P.FP64, P.TSC, P.BORIS, capacity=N)
        ft = torch.as_tensor(f).pin_memory() if host else _dev(f)
        p.set_fields(ft)
        xd, ud, wd = _dev(x), _dev(u), _dev(w)
        p.bind(N, xd, u=ud, w=wd)
        p.enable_deposit(True)
        p.sort()
        p.gather_push(qm, dt, 1)
        out = torch.zeros((3, 16 ** 3), dtype=torch.float64)
        out = out.pin_memory() if host else out.cuda()
        p.deposit(out)
        p.sync()
        outs.append((_host(xd), _host(ud), out.cpu().numpy()))
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
    import ctypes as C
    L = P.lib()
    pageable = torch.zeros(3 * N, dtype=torch.float64)        # not pinned
    assert not pageable.is_pinned()
    q = P.Part(pg, P.FP64, P.TSC, P.BORIS, capacity=N)
    l0 = q.launches()
    pp = C.c_void_p(pageable.data_ptr())
    ok = _dev(u)
    assert L.part_bind_particles(q.ctx, N, pp, None, C.c_void_p(ok.data_ptr()), None, None,
                                 None, None, None) == 1
    assert "reach" in L.part_last_error(q.ctx).decode()
    assert L.part_set_fields(q.ctx, pp, 6, P.FP64) == 1
    assert q.launches() == l0
    q.set_fields(_dev(f))
    q.bind(N, _dev(x), u=ok)
    q.enable_deposit(True)
    q.sort()
    q.gather_push(qm, dt, 1)
    assert L.part_deposit(q.ctx, pp) == 1
    q.sync()


def test_checkpoint_and_resume_bitwise():
    """The particle state lives in the caller's arrays: saving them after
    sync() and binding them to a fresh context continues the run bit for bit
    (the resumed run's first sort is a full one, the straight run's an
    incremental one; both are the same stable sort)."""
    og, pg, f, x, u, w, ids, N = _boris_case(3, 20, 8, P.TSC, 13)
    qm, dt = 1.0, 0.5 * (2.0 / 20)
    ids = ids.astype(np.int64)

    def run(steps, x0, u0, w0, i0):
        p = P.Part(pg, P.FP64, P.TSC, P.BORIS, capacity=N)
        p.set_fields(_dev(f))
        xd, ud, wd = _dev(x0), _dev(u0), _dev(w0)
        idd = torch.as_tensor(i0).cuda()
        p.bind(N, xd, u=ud, w=wd, ids=idd)
        p.enable_deposit(True)
        out = torch.empty((3, 20 ** 3), dtype=torch.float64, device="cuda")
        for _ in range(steps):
            p.sort()
            p.gather_push(qm, dt, 1)
            p.deposit(out)
        p.sync()
        return _host(xd), _host(ud), _host(wd), _host(idd), _host(out)

    straight = run(6, x, u, w, ids)
    first = run(3, x, u, w, ids)
    resumed = run(3, *first[:4])
    for a, b in zip(straight, resumed):
        assert np.array_equal(a, b)


def test_error_paths():
    og, pg = _grids(3, 16)
    N = 1000
    f = synth.uniform_em_fields(3, 16).reshape(6, -1)
    x, u, w, ids = synth.particles(3, None, N, 3)
    p = P.Part(pg, P.FP64, P.TSC, P.BORIS, capacity=N)
    with pytest.raises(P.PartError) as e:
        p.gather_push(1.0, 0.1, 1)                   # no particles bound
    assert e.value.name == "PART_EINVAL"
    xd, ud = _dev(x), _dev(u)
    p.bind(N, xd, u=ud)
    with pytest.raises(P.PartError):
        p.gather_push(1.0, 0.1, 1)                   # no fields
    p.set_fields(_dev(f))
    p.enable_deposit(True)
    with pytest.raises(P.PartError) as e:
        p.gather_push(1.0, 0.1, 1)                   # deposit without sort
    assert "part_sort" in str(e.value)
    with pytest.raises(P.PartError):
        p.bind(N + 1, xd, u=ud)                      # over capacity
    with pytest.raises(P.PartError):
        p.set_fields(_dev(f[:5]))                    # wrong ncomp
    # a particle moved out of its sorted cell -> PART_EDOMAIN, nothing faults
    p.bind(N, xd, u=ud)
    p.sort()
    p.sync()                                         # sorted state in the bound arrays
    xd[0, 0] = xd[0, 0] + 0.3          # one cell away from its sorted cell
    p.gather_push(1.0, 0.01, 1)
    with pytest.raises(P.PartError) as e:
        p.sync()
    assert e.value.name == "PART_EDOMAIN"
    # non-finite state -> PART_ENONFINITE
    p.enable_deposit(False)
    ud[1, 3] = float("nan")
    p.gather_push(1.0, 0.01, 1)
    with pytest.raises(P.PartError) as e:
        p.sync()
    assert e.value.name == "PART_ENONFINITE"
    p.sync()                                         # status cleared


def _sort_launches(p):
    l0 = p.launches()
    p.sort()
    return p.launches() - l0


@pytest.mark.parametrize("dim,n,ppc", [(3, 20, 8), (2, 40, 16), (3, 16, 4), (3, 8, 3),
                                       (3, 5, 2), (2, 18, 4)])
def test_resort_after_push_bit_exact(dim, n, ppc):
    """After a push that moves every particle by less than a cell, part_sort
    takes the per-brick incremental path; it must give the oracle's stable
    sort of the pushed positions bit for bit (bricks crossed, periodic
    wrap, partial bricks, one or two bricks per axis)."""
    og, pg = _grids(dim, n)
    N = n ** dim * ppc + 5
    x, u, w, ids = synth.particles(dim, None, N, 31 + n, u_th=2.0)   # |v| close to 1
    f = synth.em_fields(dim, n, 7, v_rms=0.05).reshape(6, -1)
    p = P.Part(pg, P.FP64, P.TSC, P.BORIS, capacity=N)
    p.set_fields(_dev(f))
    xd, ud = _dev(x), _dev(u)
    idd = torch.as_tensor(ids.astype(np.int64)).cuda()
    p.bind(N, xd, u=ud, ids=idd)
    full = _sort_launches(p)
    dt = 0.95 * 2.0 / n
    for step in range(3):
        p.gather_push(1.0, dt, 1)
        p.sync()
        xb, ib = _host(xd).copy(), _host(idd).copy()
        inc = _sort_launches(p)
        cs = _host(p.cell_start())
        p.sync()
        assert inc < full                       # the incremental path ran
        keys = O.keys(og, p.brick, xb)
        perm = O.stable_sort(keys)
        assert np.array_equal(_host(idd), ib[perm])
        assert np.array_equal(_host(xd), xb[:, perm])
        assert np.array_equal(cs, O.cell_start(p.nkeys, keys[perm]).astype(np.int64))


def test_resort_falls_back_after_a_long_move():
    """A push with dt >= dx (possible moves of a cell or more) or several fused
    steps make part_sort take the full radix path again."""
    og, pg = _grids(3, 16)
    N = 16 ** 3 * 2
    x, u, w, ids = synth.particles(3, None, N, 12, u_th=2.0)
    f = synth.em_fields(3, 16, 8, v_rms=0.05).reshape(6, -1)
    p = P.Part(pg, P.FP64, P.TSC, P.BORIS, capacity=N)
    p.set_fields(_dev(f))
    xd, ud = _dev(x), _dev(u)
    idd = torch.as_tensor(ids.astype(np.int64)).cuda()
    p.bind(N, xd, u=ud, ids=idd)
    full = _sort_launches(p)
    for dt, nsteps in ((1.5 * 2.0 / 16, 1), (0.6 * 2.0 / 16, 2)):
        p.gather_push(1.0, dt, nsteps)
        p.sync()
        xb, ib = _host(xd).copy(), _host(idd).copy()
        assert _sort_launches(p) == full
        p.sync()
        perm = O.stable_sort(O.keys(og, p.brick, xb))
        assert np.array_equal(_host(idd), ib[perm])


def test_flush_brings_the_sorted_state_home():
    """After a sort and a push the current state may live in the workspace
    copy; part_flush (asynchronous) puts it into the bound arrays, sorted, and
    gives what part_sync gives."""
    og, pg = _grids(3, 16)
    N = 16 ** 3 * 4 + 3
    x, u, w, ids = synth.particles(3, None, N, 21, u_th=0.5)
    f = synth.em_fields(3, 16, 4, v_rms=0.05).reshape(6, -1)
    runs = []
    for use_flush in (True, False):
        p = P.Part(pg, P.FP64, P.TSC, P.BORIS, capacity=N)
        p.set_fields(_dev(f))
        xd, ud = _dev(x), _dev(u)
        idd = torch.as_tensor(ids.astype(np.int64)).cuda()
        p.bind(N, xd, u=ud, ids=idd)
        for _ in range(3):                       # odd number: state ends in the other copy
            p.sort()
            p.gather_push(1.0, 0.5 * 2.0 / 16, 1)
        if use_flush:
            p.flush()
            torch.cuda.synchronize()
        else:
            p.sync()
        runs.append((_host(xd), _host(ud), _host(idd)))
    for a, b in zip(*runs):
        assert np.array_equal(a, b)
    # ids are a permutation of the originals (nothing lost or duplicated)
    assert np.array_equal(np.sort(runs[0][2]), np.arange(N))


def test_pipeline_sort_push_compact_deposit():
    """A run mixing the paths: full sort, pushes with incremental sorts,
    compaction (full sort after it), and a deposit, against the oracle doing
    the same operations on its own copy (stable sort of the keys, Boris step,
    the compaction map)."""
    n = 16
    og, pg = _grids(3, n)
    N = n ** 3 * 4 + 9
    x, u, w, ids = synth.particles(3, None, N, 44, u_th=0.8)
    w = np.random.default_rng(2).uniform(0.5, 2.0, N)
    f = synth.em_fields(3, n, 9, v_rms=0.05).reshape(6, -1)
    p = P.Part(pg, P.FP64, P.TSC, P.BORIS, capacity=N)
    p.set_fields(_dev(f))
    xd, ud, wd = _dev(x), _dev(u), _dev(w)
    idd = torch.as_tensor(ids.astype(np.int64)).cuda()
    p.bind(N, xd, u=ud, w=wd, ids=idd)
    dt = 0.7 * 2.0 / n
    xr, ur, wr, ir = x.copy(), u.copy(), w.copy(), ids.astype(np.int64)

    def oracle_sort():
        nonlocal xr, ur, wr, ir
        perm = O.stable_sort(O.keys(og, p.brick, xr))
        xr, ur, wr, ir = xr[:, perm], ur[:, perm], wr[perm], ir[perm]

    for step in range(4):
        p.sort()
        oracle_sort()
        p.gather_push(1.0, dt, 1)
        xr, ur, _, _ = O.boris_step(og, P.TSC, f, xr, ur, wr, 1.0, dt)
        if step == 1:                            # delete a fifth of the particles
            p.sync()
            d = np.random.default_rng(7).random(xr.shape[1]) < 0.2
            nn = p.compact(torch.as_tensor(d.astype(np.uint8)).cuda())
            k, src = O.compact_map(d)
            assert nn == k
            xr, ur, wr, ir = xr[:, src], ur[:, src], wr[src], ir[src]
    p.enable_deposit(True)
    p.sort()
    oracle_sort()
    p.gather_push(1.0, dt, 1)
    out = torch.empty((3, n ** 3), dtype=torch.float64, device="cuda")
    p.deposit(out)
    p.sync()
    x1, u1, F, xo = O.boris_step(og, P.TSC, f, xr, ur, wr, 1.0, dt, True)
    k = xr.shape[1]
    assert np.array_equal(_host(idd)[:k], ir)
    assert np.max(np.abs(_pdiff(_host(xd).reshape(-1)[:3 * k].reshape(3, k), x1))) <= 1e-11
    assert _rel(_host(ud).reshape(-1)[:3 * k].reshape(3, k), u1, 1e-3) <= 1e-11
    dref = O.deposit(og, P.TSC, xo, F)
    dabs = O.deposit(og, P.TSC, xo, np.abs(F))
    assert np.max(np.abs(_host(out) - dref) / np.maximum(dabs, 1e-300)) <= 1e-11
