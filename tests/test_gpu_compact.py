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
    u = rng.normal(0, 0.3, (3, N)).astype(np.float32)
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
    assert np.array_equal(_rows(ud, 3, nk), u[:, src])
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
