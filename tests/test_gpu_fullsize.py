"""Parity at the full benchmark sizes, in the launch configurations the bench
times, on outputs the oracle can compute one by one (sampled particles and
grid cells) and on properties that fix the whole result at any size.

- FP64 Boris + TSC + deposit, 3D 128^3 turbulent, 16,777,216 particles:
  device initialisation against the oracle's (all particles); the sort's
  permutation and cell_start against the oracle's stable sort (all
  particles, bit-exact); 8192 sampled particles after sort + push against
  oracle steps; the deposit at sampled cells (all their contributors run
  through the oracle) and Sum_g F_g = Sum_p F_p over the whole grid.
- Mixed form, 256^3, 134,217,728 particles: the permutation is checked by
  the properties that define a stable sort (the ids form a permutation,
  keys never decrease, equal keys keep index order), which fix it uniquely;
  cell_start against the oracle's; sampled particles and cells against FP64
  oracle steps.
- LP RK2 and SSP-RK3 + spectra, 128^3, 4,194,304 LPs x 128 bins: two steps
  (the second reuses the cached samples) on 4096 sampled LPs.
- LP shock, 160^3, 16,384,000 LPs x 128 bins: one step on LPs at the shock
  and elsewhere; flags bit-exact, spectra 1e-12.
- Compaction of the 16.8M FP64 state: every slot, bit-exact.
- 2D 64^2 uniform B: 100 fused steps on 4096 sampled particles.
- Serving: one 10^7-particle request on a 256^3 snapshot, 20 steps, sampled
  particles against FP64 oracle steps.

Tolerances are those of the small-size tests (FP64: 1e-12 per step; mixed:
f32 arithmetic, 1e-6 cell per step).
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


def _pair(u6):
    """The mixed form's compensated momentum [6][N] as f64 values hi + lo."""
    return u6[:3].astype(np.float64) + u6[3:].astype(np.float64)


def _pdiff(a, b, L=2.0):
    d = a - b
    return d - L * np.round(d / L)


def _dt_turbulent(f6, n, qm=1.0):
    bmax = float(np.sqrt((f6[3:] ** 2).sum(axis=0)).max())
    return min(0.1 / (qm * bmax), 0.5 * (2.0 / n))


def _cell_index(j, n):
    return (j[2] * n + j[1]) * n + j[0]


def _neighbour_cells(j, n, r=2):
    """Linear indices of the cells within r of cell j (periodic, 3D)."""
    out = []
    for dz in range(-r, r + 1):
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                out.append(_cell_index(((j[0] + dx) % n, (j[1] + dy) % n, (j[2] + dz) % n), n))
    return out


def _sample_cells(n, brick, count, seed):
    """Random cells plus the domain corners (periodic seam) and cells on
    brick faces."""
    rng = np.random.default_rng(seed)
    cells = [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(count)]
    cells += [(a, b, c) for a in (0, n - 1) for b in (0, n - 1) for c in (0, n - 1)]
    cells += [(brick[0] - 1, brick[1], 2 * brick[2] - 1), (brick[0], 3, 5)]
    return cells


def _cell_key_table(og, brick, n):
    """Key of every cell, from the oracle's key of the cell centre."""
    j = np.indices((n, n, n)).reshape(3, -1)[::-1]           # x fastest
    xc = -1.0 + (j + 0.5) * (2.0 / n)
    return O.keys(og, brick, xc)


def _assert_stable_sort(ks, ia):
    """ia (each particle's index in the order before the sort, listed in the
    GPU's order after it) is the stable sort of the keys: a permutation,
    keys ks = keys[ia] never decrease, and equal keys keep increasing
    previous index.  These fix the order uniquely."""
    N = ia.shape[0]
    seen = np.zeros(N, dtype=bool)
    seen[ia] = True
    assert seen.all()
    del seen
    step = 1 << 24
    for a in range(0, N - 1, step):
        b = min(a + step + 1, N)
        k, i = ks[a:b], ia[a:b]
        assert np.all(k[1:] >= k[:-1])
        eq = k[1:] == k[:-1]
        assert np.all(i[1:][eq] > i[:-1][eq])


def _contributors(cells, n, key_of_cell, cs, order):
    """Original indices of the particles in the cells around `cells`, from
    the oracle's cell_start `cs` and sorted order `order`."""
    idx = []
    for j in cells:
        for c in _neighbour_cells(j, n):
            k = key_of_cell(c)
            idx.append(order[cs[k]:cs[k + 1]])
    return np.unique(np.concatenate(idx))


def test_fullsize_fp64_boris_128():
    n, ppc, seed, qm = 128, 8, 1236, 1.0
    N = n ** 3 * ppc
    og = O.make_grid(3, (n, n, n))
    f = synth.em_fields(3, n, seed).reshape(6, -1)
    dt = _dt_turbulent(f, n)
    p = P.Part(P.make_grid(3, n), P.FP64, P.TSC, P.BORIS, capacity=N)
    p.set_fields(torch.as_tensor(f).cuda())
    x = torch.empty((3, N), dtype=torch.float64, device="cuda")
    u, w = torch.empty_like(x), torch.empty(N, dtype=torch.float64, device="cuda")
    ids = torch.empty(N, dtype=torch.int64, device="cuda")
    out = torch.empty((3, n ** 3), dtype=torch.float64, device="cuda")
    p.bind(N, x, u=u, w=w, ids=ids)
    p.init_particles(seed, 0.1)
    p.enable_deposit(True)
    p.sync()
    # initialisation: every particle
    x0, u0, w0, i0 = O.init_particles(og, N, seed, 0.1)
    assert np.array_equal(_host(x), x0)
    assert np.max(np.abs(_host(u) - u0) / np.maximum(np.abs(u0), 0.1)) <= 1e-14
    assert np.array_equal(_host(w), w0) and np.array_equal(_host(ids), i0.astype(np.int64))
    # one step as the bench runs it: sort, push through the permutation, deposit
    p.sort()
    cs_gpu = p.cell_start().clone()
    p.gather_push(qm, dt, 1)
    p.deposit(out)
    p.sync()
    keys = O.keys(og, p.brick, x0)
    perm = O.stable_sort(keys).astype(np.int64)
    cs = O.cell_start(p.nkeys, keys[perm]).astype(np.int64)
    assert np.array_equal(_host(ids), perm)
    assert np.array_equal(_host(cs_gpu), cs)
    xg, ug = _host(x), _host(u)
    # sampled particles against oracle steps from their initial state
    s = np.random.default_rng(1).choice(N, 8192, replace=False)
    o = perm[s]
    xr, ur, _, _ = O.boris_step(og, P.TSC, f, x0[:, o], u0[:, o], w0[o], qm, dt, True)
    assert np.max(np.abs(_pdiff(xg[:, s], xr))) <= 1e-12 * 2.0
    assert np.max(np.abs(ug[:, s] - ur) / np.maximum(np.abs(ur), 0.1)) <= 1e-12
    # deposit at sampled cells: all contributors through the oracle
    cells = _sample_cells(n, p.brick, 40, 2)
    ktab = _cell_key_table(og, p.brick, n)
    con = _contributors(cells, n, lambda c: int(ktab[c]), cs, perm)
    _, _, Fc, xoc = O.boris_step(og, P.TSC, f, x0[:, con], u0[:, con], w0[con], qm, dt, True)
    og_ = _host(out)
    for j in cells:
        c = _cell_index(j, n)
        ref = O.deposit_cell(og, P.TSC, xoc, Fc, c)
        dabs = O.deposit_cell(og, P.TSC, xoc, np.abs(Fc), c)
        assert np.all(np.abs(og_[:, c] - ref) <= 1e-12 * np.maximum(dabs, 1e-300)), j
    # momentum: the grid holds what the particles lost, over the whole grid
    Fp = w0[perm] * (ug - u0[:, perm]) / dt
    assert np.all(np.abs(og_.sum(axis=1) - Fp.sum(axis=1)) <= 1e-12 * np.abs(Fp).sum(axis=1))
    del Fp, x0, u0, og_
    # the next step re-sorts incrementally (every particle moved under a cell)
    i1, w1 = _host(ids), _host(w)
    p.sort()
    cs_gpu = p.cell_start().clone()
    p.gather_push(qm, dt, 1)
    p.deposit(out)
    p.sync()
    keys = O.keys(og, p.brick, xg)
    perm = O.stable_sort(keys).astype(np.int64)
    assert np.array_equal(_host(ids), i1[perm])
    assert np.array_equal(_host(cs_gpu), O.cell_start(p.nkeys, keys[perm]).astype(np.int64))
    o = perm[s]
    xr, ur, _, _ = O.boris_step(og, P.TSC, f, xg[:, o], ug[:, o], w1[o], qm, dt, True)
    assert np.max(np.abs(_pdiff(_host(x)[:, s], xr))) <= 1e-12 * 2.0
    assert np.max(np.abs(_host(u)[:, s] - ur) / np.maximum(np.abs(ur), 0.1)) <= 1e-12
    del p, x, u, w, ids, out
    torch.cuda.empty_cache()


def _mixed_to_x(cell, off, n):
    c = cell.astype(np.int64)
    j = np.stack([c % n, (c // n) % n, c // (n * n)])
    return -1.0 + (j + 0.5 + off.astype(np.float64)) * (2.0 / n)


def test_fullsize_mixed_256():
    """134M particles; ids bound so particles can be followed through the
    sort (the kernel is the bench's, with the id plane carried along)."""
    n, ppc, seed, qm = 256, 8, 1237, 1.0
    N = n ** 3 * ppc
    og = O.make_grid(3, (n, n, n))
    f = synth.em_fields(3, n, seed).reshape(6, -1).astype(np.float32)
    dt = _dt_turbulent(f.astype(np.float64), n)
    f64 = f.astype(np.float64)
    p = P.Part(P.make_grid(3, n), P.MIXED, P.TSC, P.BORIS, capacity=N)
    p.set_fields(torch.as_tensor(f).cuda())
    cell = torch.empty(N, dtype=torch.int32, device="cuda")
    off = torch.empty((3, N), dtype=torch.float32, device="cuda")
    u = torch.empty((6, N), dtype=torch.float32, device="cuda")   # compensated pair
    w = torch.empty(N, dtype=torch.float32, device="cuda")
    ids = torch.empty(N, dtype=torch.int64, device="cuda")
    out = torch.empty((3, n ** 3), dtype=torch.float64, device="cuda")
    p.bind(N, cell, off=off, u=u, w=w, ids=ids)
    p.init_particles(seed, 0.1)
    p.enable_deposit(True)
    p.sync()
    cell0_d, off0_d, u0_d, w0_d = cell.clone(), off.clone(), u.clone(), w.clone()
    p.sort()
    cs_gpu = p.cell_start().clone()
    p.gather_push(qm, dt, 1)
    p.deposit(out)
    p.sync()
    # the sort: properties that define the stable sort uniquely
    ktab = _cell_key_table(og, p.brick, n)
    cell0 = _host(cell0_d)
    keys = ktab[cell0]
    del cell0
    ia = _host(ids)
    ks = keys[ia]
    del keys
    _assert_stable_sort(ks, ia)
    cs = O.cell_start(p.nkeys, ks).astype(np.int64)
    del ks
    assert np.array_equal(_host(cs_gpu), cs)

    def init_state(o):
        ot = torch.as_tensor(o).cuda()
        return (_mixed_to_x(_host(cell0_d[ot]), _host(off0_d[:, ot]), n),
                _pair(_host(u0_d[:, ot])), _host(w0_d[ot]).astype(np.float64))

    # sampled particles against FP64 oracle steps from the same state
    s = np.random.default_rng(3).choice(N, 8192, replace=False)
    x0s, u0s, w0s = init_state(ia[s])
    xr, ur, _, _ = O.boris_step(og, P.TSC, f64, x0s, u0s, w0s, qm, dt, True)
    st = torch.as_tensor(s).cuda()
    xg = _mixed_to_x(_host(cell[st]), _host(off[:, st]), n)
    d = _pdiff(xg, xr) / (2.0 / n)
    assert np.max(np.abs(d)) <= 1e-6
    assert np.max(np.abs(_pair(_host(u[:, st])) - ur)) <= 2e-6 * np.max(np.abs(ur))
    # deposit at sampled cells
    cells = _sample_cells(n, p.brick, 24, 4)
    con = _contributors(cells, n, lambda c: int(ktab[c]), cs, ia)
    x0c, u0c, w0c = init_state(con)
    _, _, Fc, xoc = O.boris_step(og, P.TSC, f64, x0c, u0c, w0c, qm, dt, True)
    og_ = _host(out)
    for j in cells:
        c = _cell_index(j, n)
        ref = O.deposit_cell(og, P.TSC, xoc, Fc, c)
        dabs = O.deposit_cell(og, P.TSC, xoc, np.abs(Fc), c)
        assert np.all(np.abs(og_[:, c] - ref) <= 1e-5 * np.maximum(dabs, 1e-300)), j
    # the next step's incremental sort: cells moved by the push
    keys = ktab[_host(cell)]
    p.sort()
    cs_gpu = p.cell_start().clone()
    p.gather_push(qm, dt, 1)
    p.sync()
    i2 = _host(ids)
    pos = np.empty(N, dtype=np.int64)          # slot of each particle after step 1
    pos[ia] = np.arange(N)
    del ia
    prev = pos[i2]                             # ... in the new order: stability is by it
    del pos, i2
    ks = keys[prev]
    del keys
    _assert_stable_sort(ks, prev)
    assert np.array_equal(_host(cs_gpu), O.cell_start(p.nkeys, ks).astype(np.int64))
    del p, cell, off, u, w, ids, out, cell0_d, off0_d, u0_d, w0_d
    torch.cuda.empty_cache()


@pytest.mark.parametrize("order", [2, 3])
def test_fullsize_lp_128(order):
    n, nlp, nb, seed = 128, 1 << 22, 128, 1238
    og = O.make_grid(3, (n, n, n))
    vel, rho, B = synth.fluid_snapshot(3, n, seed)
    vel, rho, B = vel.reshape(3, -1), rho.reshape(1, -1), B.reshape(3, -1)
    p = P.Part(P.make_grid(3, n), P.FP64, P.TSC, P.LP_RK2, capacity=nlp, nbins=nb)
    p.set_fields(torch.as_tensor(np.concatenate([vel, rho, B])).cuda())
    x = torch.empty((3, nlp), dtype=torch.float64, device="cuda")
    chi = torch.empty((nb, nlp), dtype=torch.float64, device="cuda")
    eng = torch.empty_like(chi)
    nold = torch.empty(nlp, dtype=torch.float64, device="cuda")
    p.bind(nlp, x, chi=chi, eng=eng, n_old=nold)
    p.set_lp_order(order)
    p.init_particles(seed, 0.0, 1.0, 1e6, 2.2, 1e-6)
    p.sync()
    x0, _, _, _ = O.init_particles(og, nlp, seed, 0.0)
    assert np.array_equal(_host(x), x0)
    p.sort()
    p.sync()
    dt = 0.5 * 2.0 / n
    c0 = 1.0 / (1e3 * 1.0 * 100 * dt)
    s = torch.as_tensor(np.random.default_rng(5).choice(nlp, 4096, replace=False)).cuda()

    def sampled():
        p.sync()
        return _host(x[:, s]), _host(chi[:, s]), _host(eng[:, s]), _host(nold[s])

    xs, cs_, es, ns = sampled()
    e1, c1 = O.init_spectrum(nb, 1.0, 1e6, 2.2, 1e-6)
    assert np.max(np.abs(es - e1[:, None]) / e1[:, None]) <= 1e-15
    assert np.max(np.abs(cs_ - c1[:, None]) / c1[:, None]) <= 1e-13
    nref = np.array([O.gather(og, P.TSC, rho, xs[:, i])[0] for i in range(xs.shape[1])])
    assert np.max(np.abs(ns - nref) / nref) <= 1e-13
    for _ in range(2):                   # the second step reuses the cached samples
        p.gather_push(0.0, dt, 1)
        p.spec_update(dt, c0, 0.0)
        xg, cg, eg, ng = sampled()
        step = O.lp_rk2_step if order == 2 else O.lp_rk3_step
        xr, nn, b2, gm = step(og, P.TSC, vel, rho, B, xs, dt)
        cr, er, nr = O.spec_update(cs_, es, ns, nn, b2, gm, dt, c0)
        assert np.max(np.abs(_pdiff(xg, xr))) <= 1e-12 * 2.0
        assert np.max(np.abs(eg - er) / er) <= 1e-12
        assert np.max(np.abs(cg - cr) / np.maximum(np.abs(cr), 1e-300)) <= 1e-12
        assert np.max(np.abs(ng - nr) / nr) <= 1e-12
        xs, cs_, es, ns = xg, cg, eg, ng
    del p, x, chi, eng, nold
    torch.cuda.empty_cache()


def test_fullsize_lp_shock_160():
    n, ppc, nb, seed = 160, 4, 128, 1241
    N = n ** 3 * ppc
    og = O.make_grid(3, (n, n, n))
    r = 40.0 / 11.0
    xc = -1.0 + (np.arange(n) + 0.5) * (2.0 / n)
    down = np.broadcast_to(xc > 0.0, (n, n, n)).reshape(-1)
    vel = np.zeros((3, n ** 3))
    vel[0] = np.where(down, 0.1 / r, 0.1)
    rho = np.where(down, 50.0 * r, 50.0)[None]
    B = np.zeros((3, n ** 3))
    B[0] = 1.0
    p = P.Part(P.make_grid(3, n), P.FP64, P.TSC, P.LP_RK2, capacity=N, nbins=nb)
    p.set_fields(torch.as_tensor(np.concatenate([vel, rho, B])).cuda())
    x = torch.empty((3, N), dtype=torch.float64, device="cuda")
    chi = torch.empty((nb, N), dtype=torch.float64, device="cuda")
    eng = torch.empty_like(chi)
    nold = torch.empty(N, dtype=torch.float64, device="cuda")
    st = torch.zeros(N, dtype=torch.uint8, device="cuda")
    p.bind(N, x, chi=chi, eng=eng, n_old=nold)
    p.init_particles(seed, 0.0, 1e2, 1e4, 9.0, 1e-6)
    p.sort()
    p.enable_shocks(1.5, st)
    p.sync()
    dt = 0.5 * (2.0 / n) / 0.1
    r_cell = O.shock_cells(og, vel, rho, 1.5)
    assert np.array_equal(_host(p.shock_cells()), r_cell)
    # LPs just upstream of the shock (most enter it this step) and elsewhere
    near = torch.nonzero((x[0] > -3.0 * 2.0 / n) & (x[0] < 0.0)).flatten()[:3000]
    rest = torch.as_tensor(np.random.default_rng(6).choice(N, 3000, replace=False)).cuda()
    s = torch.cat([near, rest]).unique()
    xs, cs_, es, ns = _host(x[:, s]), _host(chi[:, s]), _host(eng[:, s]), _host(nold[s])
    p.gather_push(0.0, dt, 1)
    p.spec_update(dt, 1e-8, 0.0)
    p.sync()
    xr, nn, b2, gm = O.lp_rk2_step(og, P.TSC, vel, rho, B, xs, dt)
    cr, er, nr = O.spec_update(cs_, es, ns, nn, b2, gm, dt, 1e-8)
    cr, sr = O.lp_shock(og, r_cell, xr, cr, er, np.zeros(xs.shape[1], np.uint8))
    assert 500 < int(sr.sum()) < xs.shape[1]
    assert np.array_equal(_host(st[s]), sr)
    assert np.max(np.abs(_pdiff(_host(x[:, s]), xr))) <= 1e-12 * 2.0
    eg, cg = _host(eng[:, s]), _host(chi[:, s])
    assert np.max(np.abs(eg - er) / er) <= 1e-12
    assert np.max(np.abs(cg - cr) / np.maximum(np.abs(cr), 1e-300)) <= 1e-12
    del p, x, chi, eng, nold, st
    torch.cuda.empty_cache()


@pytest.mark.parametrize("frac", [0.01, 0.1])
def test_fullsize_compact_16m(frac):
    n, ppc, seed = 128, 8, 1240
    N = n ** 3 * ppc
    p = P.Part(P.make_grid(3, n), P.FP64, P.TSC, P.BORIS, capacity=N)
    x = torch.empty((3, N), dtype=torch.float64, device="cuda")
    u, w = torch.empty_like(x), torch.empty(N, dtype=torch.float64, device="cuda")
    ids = torch.empty(N, dtype=torch.int64, device="cuda")
    p.bind(N, x, u=u, w=w, ids=ids)
    p.init_particles(seed, 0.1)
    p.sync()
    before = [_host(t) for t in (x, u, w, ids)]
    d = np.random.default_rng(seed).random(N) < frac
    nn = p.compact(torch.as_tensor(d.astype(np.uint8)).cuda())
    p.sync()
    nk, src = O.compact_map(d)
    assert nn == nk
    xa = _host(x.reshape(-1)[: 3 * nk]).reshape(3, nk)
    ua = _host(u.reshape(-1)[: 3 * nk]).reshape(3, nk)
    assert np.array_equal(xa, before[0][:, src]) and np.array_equal(ua, before[1][:, src])
    assert np.array_equal(_host(w)[:nk], before[2][src])
    assert np.array_equal(_host(ids)[:nk], before[3][src])
    del p, x, u, w, ids
    torch.cuda.empty_cache()


def test_fullsize_2d_uniform_100_steps():
    n, ppc, seed, steps, dt = 64, 16, 1235, 100, 0.1
    N = n * n * ppc
    og = O.make_grid(2, (n, n, n))
    f = synth.uniform_em_fields(2, n, B=(0, 0, 1.0)).reshape(6, -1)
    p = P.Part(P.make_grid(2, n), P.FP64, P.TSC, P.BORIS, capacity=N)
    p.set_fields(torch.as_tensor(f).cuda())
    x = torch.empty((3, N), dtype=torch.float64, device="cuda")
    u = torch.empty_like(x)
    p.bind(N, x, u=u)
    p.init_particles(seed, 0.1)
    p.sort()
    p.sync()
    s = np.random.default_rng(7).choice(N, 4096, replace=False)
    xr, ur = _host(x)[:, s], _host(u)[:, s]
    u_start = ur.copy()
    p.gather_push(1.0, dt, steps)
    p.sync()
    for _ in range(steps):
        xr, ur, _, _ = O.boris_step(og, P.TSC, f, xr, ur, None, 1.0, dt)
    ug = _host(u)[:, s]
    assert np.max(np.abs(_pdiff(_host(x)[:, s], xr))) <= 1e-12 * 2.0 * steps
    assert np.max(np.abs(ug - ur)) <= 1e-12 * steps * np.max(np.abs(ur))
    assert np.max(np.abs(np.linalg.norm(ug, axis=0) / np.linalg.norm(u_start, axis=0) - 1)) \
        < 1e-13
    del p, x, u
    torch.cuda.empty_cache()


def test_fullsize_serving_request_256():
    from paper_2602_23434_b300 import serving as S
    n, N, steps, seed = 256, 10 ** 7, 20, 77
    og = O.make_grid(3, (n, n, n))
    snap = S.make_snapshot(torch, n, 1241, N)
    srv = S.Server(torch, [snap], N * S.STATE_BYTES_PER_PARTICLE + 1, chunk=4096,
                   slice_steps=8)
    rq = srv.submit(0, N, steps, seed=seed)
    srv.run_until_idle()
    cg, og_, ug = rq.result()
    srv.close()
    dt = 0.5 * 2.0 / n
    # the request's initial state: the same initialisation and sort
    p = P.Part(P.make_grid(3, n), P.MIXED, P.TSC, P.BORIS, capacity=N)
    p.set_fields(snap.fields)
    cell = torch.empty(N, dtype=torch.int32, device="cuda")
    off = torch.empty((3, N), dtype=torch.float32, device="cuda")
    u = torch.empty((6, N), dtype=torch.float32, device="cuda")
    p.bind(N, cell, off=off, u=u)
    p.init_particles(seed, 0.1)
    p.sort()
    p.sync()
    s = torch.as_tensor(np.random.default_rng(8).choice(N, 2048, replace=False)).cuda()
    xr = _mixed_to_x(_host(cell[s]), _host(off[:, s]), n)
    ur = _pair(_host(u[:, s]))
    f64 = _host(snap.fields).astype(np.float64)
    for _ in range(steps):
        xr, ur, _, _ = O.boris_step(og, P.TSC, f64, xr, ur, None, 1.0, dt)
    xg = _mixed_to_x(_host(cg[s]), _host(og_[:, s]), n)
    assert np.max(np.abs(_pdiff(xg, xr) / (2.0 / n))) <= 1e-6 * steps
    assert np.max(np.abs(_pair(_host(ug[:, s])) - ur)) <= 1e-6 * steps * np.max(np.abs(ur))
    del p, cell, off, u, snap, cg, og_, ug
    torch.cuda.empty_cache()
