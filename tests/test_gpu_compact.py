"""Hole/filler compaction of Sec. 3.2 on the GPU against the oracle's map,
bit-exact: every bound array of every mode (FP64 Boris, mixed Boris, LP)
must hold, in slot j < n_new, exactly the old particle src[j] that the
oracle's five-step procedure names, with row stride n_new afterwards.
A sort after compaction must then give the oracle's stable sort of the
survivors (the compacted set is an ordinary particle set again).
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


def _rows(t, rows, n):
    """First rows*n elements of a flat plane buffer as [rows][n]."""
    return _host(t.reshape(-1)[: rows * n]).reshape(rows, n)


def _masks(N, seed):
    rng = np.random.default_rng(seed)
    out = {"none": np.zeros(N, bool), "all": np.ones(N, bool)}
    for frac in (0.01, 0.5, 0.9):
        out[f"rand{frac}"] = rng.random(N) < frac
    tail = np.zeros(N, bool)
    tail[N - N // 7:] = True                  # only the tail dies: nothing moves
    head = np.zeros(N, bool)
    head[: N // 5] = True                     # only the head dies: the tail fills it
    out["tail"], out["head"] = tail, head
    return out


@pytest.mark.parametrize("N", [1, 33, 20 ** 3 * 4 + 13])
@pytest.mark.parametrize("which", ["none", "all", "rand0.01", "rand0.5", "rand0.9",
                                   "tail", "head"])
def test_compact_fp64_boris(N, which):
    n = 20
    x, u, w, ids = synth.particles(3, None, N, 31)
    w = np.random.default_rng(3).uniform(0.5, 2.0, N)
    d = _masks(N, 7 + N)[which]
    p = P.Part(P.make_grid(3, n), P.FP64, P.TSC, P.BORIS, capacity=N)
    xd, ud, wd = (torch.as_tensor(a).cuda() for a in (x, u, w))
    idd = torch.as_tensor(ids.astype(np.int64)).cuda()
    p.bind(N, xd, u=ud, w=wd, ids=idd)
    nn = p.compact(torch.as_tensor(d.astype(np.uint8)).cuda())
    p.sync()
    nk, src = O.compact_map(d)
    assert nn == nk
    assert np.array_equal(_rows(xd, 3, nk), x[:, src])
    assert np.array_equal(_rows(ud, 3, nk), u[:, src])
    assert np.array_equal(_rows(wd, 1, nk)[0], w[src])
    assert np.array_equal(_host(idd)[:nk], ids[src].astype(np.int64))


def test_compact_after_sort_then_sort_again():
    """Compaction flushes a pending sort first; the survivors then sort like
    any particle set."""
    n, N = 20, 20 ** 3 * 6 + 5
    og = O.make_grid(3, (n, n, n))
    x, u, w, ids = synth.particles(3, None, N, 41)
    p = P.Part(P.make_grid(3, n), P.FP64, P.TSC, P.BORIS, capacity=N)
    xd, ud = torch.as_tensor(x).cuda(), torch.as_tensor(u).cuda()
    idd = torch.as_tensor(ids.astype(np.int64)).cuda()
    p.bind(N, xd, u=ud, ids=idd)
    p.sort()
    keys = O.keys(og, p.brick, x)
    perm = O.stable_sort(keys)
    xs, us, is_ = x[:, perm], u[:, perm], ids[perm]
    d = np.random.default_rng(5).random(N) < 0.3
    nn = p.compact(torch.as_tensor(d.astype(np.uint8)).cuda())
    nk, src = O.compact_map(d)
    assert nn == nk
    xc, uc, ic = xs[:, src], us[:, src], is_[src]
    p.sort()
    cs = _host(p.cell_start())
    p.sync()
    k2 = O.keys(og, p.brick, xc)
    perm2 = O.stable_sort(k2)
    assert np.array_equal(_rows(xd, 3, nk), xc[:, perm2])
    assert np.array_equal(_rows(ud, 3, nk), uc[:, perm2])
    assert np.array_equal(_host(idd)[:nk], ic[perm2].astype(np.int64))
    assert np.array_equal(cs, O.cell_start(p.nkeys, k2[perm2]).astype(np.int64))


@pytest.mark.parametrize("which", ["rand0.5", "head", "all"])
def test_compact_mixed_boris(which):
    n, N = 16, 16 ** 3 * 5 + 3
    rng = np.random.default_rng(8)
    cell = rng.integers(0, n ** 3, N).astype(np.int32)
    off = rng.uniform(-0.5, 0.5, (3, N)).astype(np.float32)
    # the momentum is a compensated pair [6][N]: f32 value and residual
    u = rng.normal(0, 0.3, (6, N)).astype(np.float32)
    u[3:] *= 1e-8
    w = rng.uniform(0.5, 2.0, N).astype(np.float32)
    ids = np.arange(N, dtype=np.int64) * 3 + 1
    d = _masks(N, 9)[which]
    p = P.Part(P.make_grid(3, n), P.MIXED, P.CIC, P.BORIS, capacity=N)
    cd, od, ud, wd, idd = (torch.as_tensor(a).cuda() for a in (cell, off, u, w, ids))
    p.bind(N, cd, off=od, u=ud, w=wd, ids=idd)
    nn = p.compact(torch.as_tensor(d.astype(np.uint8)).cuda())
    p.sync()
    nk, src = O.compact_map(d)
    assert nn == nk
    assert np.array_equal(_host(cd)[:nk], cell[src])
    assert np.array_equal(_rows(od, 3, nk), off[:, src])
    assert np.array_equal(_rows(ud, 6, nk), u[:, src])
    assert np.array_equal(_host(wd)[:nk], w[src])
    assert np.array_equal(_host(idd)[:nk], ids[src])


@pytest.mark.parametrize("which", ["rand0.01", "rand0.9", "tail"])
def test_compact_lp(which):
    n, N, nb = 16, 16 ** 3 * 3 + 9, 12
    rng = np.random.default_rng(10)
    x = rng.uniform(-1.0, 1.0, (3, N))
    chi = rng.uniform(0.0, 1.0, (nb, N))
    eng = np.sort(rng.uniform(1.0, 10.0, (nb, N)), axis=0)
    n_old = rng.uniform(0.5, 2.0, N)
    ids = np.arange(N, dtype=np.int64)
    d = _masks(N, 11)[which]
    p = P.Part(P.make_grid(3, n), P.FP64, P.TSC, P.LP_RK2, capacity=N, nbins=nb)
    xd, cd, ed, nd, idd = (torch.as_tensor(a).cuda() for a in (x, chi, eng, n_old, ids))
    p.bind(N, xd, ids=idd, chi=cd, eng=ed, n_old=nd)
    nn = p.compact(torch.as_tensor(d.astype(np.uint8)).cuda())
    p.sync()
    nk, src = O.compact_map(d)
    assert nn == nk
    assert np.array_equal(_rows(xd, 3, nk), x[:, src])
    assert np.array_equal(_rows(cd, nb, nk), chi[:, src])
    assert np.array_equal(_rows(ed, nb, nk), eng[:, src])
    assert np.array_equal(_host(nd)[:nk], n_old[src])
    assert np.array_equal(_host(idd)[:nk], ids[src])


def test_compact_empty_and_errors():
    p = P.Part(P.make_grid(3, 8), P.FP64, P.TSC, P.BORIS, capacity=4)
    xd = torch.zeros((3, 4), dtype=torch.float64, device="cuda")
    ud = torch.zeros((3, 4), dtype=torch.float64, device="cuda")
    p.bind(0, xd, u=ud)
    assert p.compact(None) == 0
    p.bind(4, xd, u=ud)
    with pytest.raises(P.PartError) as e:
        p.compact(None)
    assert e.value.name == "PART_EINVAL"


def _flat(t, rows, n):
    """First rows*n elements of a flat buffer as [rows][n] (row stride n)."""
    return _host(t.reshape(-1)[: rows * n]).reshape(rows, n)


@pytest.mark.parametrize("mode", ["fp64", "mixed", "lp"])
def test_inject_then_sort_then_compact(mode):
    """Run-time injection (Sec. 3.2): buffers allocated once at the capacity;
    the set grows by k = 0, a ragged k and then exactly to the capacity; every
    plane equals the concatenation of the old and the new particles at the new
    row stride; one more particle is refused.  The grown set then sorts like
    any particle set (the oracle's stable sort) and compacts bit-exactly.  LP
    shock flags of the new particles are cleared, the old ones kept."""
    n, C, n0, k2 = 16, 16 ** 3 * 3 + 7, 4000, 1237
    og = O.make_grid(3, (n, n, n))
    rng = np.random.default_rng(17)
    x_all, u_all, _, ids_all = synth.particles(3, None, C, 19)
    ids_all = ids_all.astype(np.int64) * 5 + 3
    w_all = rng.uniform(0.5, 2.0, C)
    nb = 6
    chi_all = rng.uniform(0.0, 1.0, (nb, C))
    eng_all = np.sort(rng.uniform(1.0, 10.0, (nb, C)), axis=0)
    nold_all = rng.uniform(0.5, 2.0, C)
    if mode == "mixed":
        dx = 2.0 / n
        j = np.minimum(np.floor((x_all + 1.0) / dx), n - 1).astype(np.int64)
        off_all = ((x_all + 1.0) / dx - j - 0.5).astype(np.float32)
        cell_all = ((j[2] * n + j[1]) * n + j[0]).astype(np.int32)
        planes = {"x": (cell_all, 1, torch.int32), "off": (off_all, 3, torch.float32),
                  "u": (np.concatenate([u_all.astype(np.float32),
                                        (u_all - u_all.astype(np.float32)).astype(np.float32)]),
                        6, torch.float32),
                  "w": (w_all.astype(np.float32), 1, torch.float32),
                  "ids": (ids_all, 1, torch.int64)}
        p = P.Part(P.make_grid(3, n), P.MIXED, P.TSC, P.BORIS, capacity=C)
    elif mode == "fp64":
        planes = {"x": (x_all, 3, torch.float64), "u": (u_all, 3, torch.float64),
                  "w": (w_all, 1, torch.float64), "ids": (ids_all, 1, torch.int64)}
        p = P.Part(P.make_grid(3, n), P.FP64, P.TSC, P.BORIS, capacity=C)
    else:
        planes = {"x": (x_all, 3, torch.float64), "chi": (chi_all, nb, torch.float64),
                  "eng": (eng_all, nb, torch.float64), "n_old": (nold_all, 1, torch.float64),
                  "ids": (ids_all, 1, torch.int64)}
        p = P.Part(P.make_grid(3, n), P.FP64, P.TSC, P.LP_RK2, capacity=C, nbins=nb)

    def rows_of(a, rows):
        return a.reshape(rows, -1)

    # buffers of capacity rows x C; the first n0 particles at row stride n0
    buf = {}
    for k, (a, rows, dt) in planes.items():
        b = torch.zeros(rows * C, dtype=dt, device="cuda")
        b[: rows * n0] = torch.as_tensor(np.ascontiguousarray(rows_of(a, rows)[:, :n0])).reshape(-1)
        buf[k] = b
    p.bind(n0, buf["x"], off=buf.get("off"), u=buf.get("u"), w=buf.get("w"), ids=buf["ids"],
           chi=buf.get("chi"), eng=buf.get("eng"), n_old=buf.get("n_old"))
    st = None
    if mode == "lp":
        vel, rho, B = synth.fluid_snapshot(3, n, 5, v_rms=0.05)
        p.set_fields(torch.as_tensor(np.concatenate([vel, rho, B]).reshape(7, -1)).cuda())
        st = torch.ones(C, dtype=torch.uint8, device="cuda")
        p.enable_shocks(1.2, st)

    def src(lo, hi):
        return {k: torch.as_tensor(np.ascontiguousarray(rows_of(a, rows)[:, lo:hi])).cuda()
                for k, (a, rows, dt) in planes.items()}

    cur = n0
    for k in (0, k2, C - n0 - k2):
        s = src(cur, cur + k)
        p.inject(k, s["x"], off=s.get("off"), u=s.get("u"), w=s.get("w"), ids=s["ids"],
                 chi=s.get("chi"), eng=s.get("eng"), n_old=s.get("n_old"))
        cur += k
        p.sync()
        for name, (a, rows, dt) in planes.items():
            assert np.array_equal(_flat(buf[name], rows, cur), rows_of(a, rows)[:, :cur]), name
        if st is not None:
            sh = _host(st)[:cur]
            assert np.all(sh[:n0] == 1) and np.all(sh[n0:] == 0)
    assert cur == C
    s = src(0, 1)
    with pytest.raises(P.PartError) as e:
        p.inject(1, s["x"], off=s.get("off"), u=s.get("u"), w=s.get("w"), ids=s["ids"],
                 chi=s.get("chi"), eng=s.get("eng"), n_old=s.get("n_old"))
    assert e.value.name == "PART_EINVAL"
    # sort: the oracle's stable sort of the whole grown set
    p.sort()
    p.sync()
    if mode == "mixed":
        tab = np.array([O.cell_key(og, p.brick, (c % n, (c // n) % n, c // (n * n)))
                        for c in range(n ** 3)], dtype=np.uint32)
        keys = tab[cell_all]
    else:
        keys = O.keys(og, p.brick, x_all)
    perm = O.stable_sort(keys)
    for name, (a, rows, dt) in planes.items():
        assert np.array_equal(_flat(buf[name], rows, C), rows_of(a, rows)[:, perm]), name
    # compaction of the grown, sorted set
    d = rng.random(C) < 0.3
    nn = p.compact(torch.as_tensor(d.astype(np.uint8)).cuda())
    nk, srcmap = O.compact_map(d)
    assert nn == nk
    p.sync()
    for name, (a, rows, dt) in planes.items():
        assert np.array_equal(_flat(buf[name], rows, nk), rows_of(a, rows)[:, perm][:, srcmap]), \
            name
