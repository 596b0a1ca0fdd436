"""Domain decomposition with particle exchange (Sec. 3.3, "Multi-core
communication") through the CUDA library, as two processes on one GPU that
talk over gloo (the kernels of the two ranks never wait on one another: every
message goes through the host between launches).

Each rank's context covers its half of a 16^3 periodic grid plus halo cells;
after each step the particles that entered a halo cell are packed by
part_exchange_pack, sent, removed by part_compact and appended by
part_exchange_unpack on the neighbour; the deposit's halo planes are packed
and added by part_box_pack / part_box_add.  After four steps the union of the
ranks' particles is compared with one oracle run on the whole grid:
  FP64 Boris: ids exact, state within 1e-12 per step, the last deposit within
    1e-12 of the sum of |contributions| per cell;
  mixed form: ids exact, positions within 1e-6 cell and momenta within 2e-6
    of max|u| per step (the mixed form's one-step tolerances);
  LP (Heun RK2 + spectral update): ids exact, positions and spectra within
    1e-12 per step.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from oracle import oracle as O  # noqa: E402
from paper_2602_23434_b300 import synth  # noqa: E402

NG, PPC, STEPS, SEED, NB = 16, 3, 4, 91, 16


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem(mode):
    N = NG ** 3 * PPC
    x, u, _, ids = synth.particles(3, None, N, SEED, u_th=0.3)
    w = np.random.default_rng(SEED).uniform(0.5, 2.0, N)
    dt = 0.5 * 2.0 / NG
    if mode == "lp":
        vel, rho, B = synth.fluid_snapshot(3, NG, SEED, v_rms=0.2)
        f = np.concatenate([vel, rho, B])
    else:
        f = synth.em_fields(3, NG, SEED, v_rms=0.05)
    return f, x, u, w, ids.astype(np.int64), dt


def _lp_init(x, f):
    g = O.make_grid(3, (NG,) * 3)
    e0, c0 = O.init_spectrum(NB, 1.0, 1e4, 2.2, 1e-6)
    n = x.shape[1]
    chi = np.repeat(c0[:, None], n, axis=1)
    eng = np.repeat(e0[:, None], n, axis=1)
    _, n_old, _, _ = O.lp_rk2_step(g, O.TSC, f[:3], f[3:4], f[4:], x, 0.0)
    return chi, eng, n_old


C0 = 0.5


def _rank(rank, world, port, mode, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put(_rank_body(rank, mode))
    except Exception:                     # report to the parent, do not hang it
        import traceback
        q.put((rank, "error", traceback.format_exc()))
    finally:
        dist.destroy_process_group()


def _rank_body(rank, mode):
    from paper_2602_23434_b300 import _lib as P
    from paper_2602_23434_b300 import multirank as M
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    # the LP push samples up to a cell outside the interior: two halo cells
    dec = M.Decomp(3, (NG,) * 3, (2, 1, 1), rank, halo=2 if mode == "lp" else 1)
    f, x, u, w, ids, dt = _problem(mode)
    N = ids.shape[0]
    mine = np.ones(N, bool)
    for a in range(3):
        s = (x[a] - dec.xmin_local[a]) * (1.0 / dec.dx[a])
        mine &= (s >= dec.interior[a][0]) & (s < dec.interior[a][1])
    n = int(mine.sum())
    cap = N                                   # room for every particle
    fl = dec.local_fields(f)
    ncomp = fl.shape[0]
    G = int(np.prod(dec.n_local))

    def plane(a, rows, dtype):
        b = torch.zeros(rows * cap, dtype=dtype, device=dev)
        b[: rows * n] = torch.as_tensor(np.ascontiguousarray(a).reshape(-1)).to(dev)
        return b

    idd = plane(ids[mine], 1, torch.int64)
    if mode == "fp64":
        p = P.Part(dec.grid(), P.FP64, P.TSC, P.BORIS, capacity=cap)
        p.set_fields(torch.as_tensor(fl.reshape(ncomp, -1)).to(dev))
        xd = plane(x[:, mine], 3, torch.float64)
        ud = plane(u[:, mine], 3, torch.float64)
        wd = plane(w[mine], 1, torch.float64)
        p.bind(n, xd, u=ud, w=wd, ids=idd)
        p.enable_deposit(True)
    elif mode == "mixed":
        p = P.Part(dec.grid(), P.MIXED, P.TSC, P.BORIS, capacity=cap)
        p.set_fields(torch.as_tensor(fl.reshape(ncomp, -1).astype(np.float32)).to(dev))
        xm = x[:, mine]
        j = np.zeros((3, n), np.int64)
        off = np.zeros((3, n), np.float32)
        for a in range(3):
            s = (xm[a] - dec.xmin_local[a]) * (1.0 / dec.dx[a])
            j[a] = np.floor(s)
            off[a] = (s - j[a] - 0.5).astype(np.float32)
        nl = dec.n_local
        cell = ((j[2] * nl[1] + j[1]) * nl[0] + j[0]).astype(np.int32)
        uf = u[:, mine].astype(np.float32)
        cd = plane(cell, 1, torch.int32)
        od = plane(off, 3, torch.float32)
        ud = plane(np.concatenate([uf, np.zeros_like(uf)]), 6, torch.float32)
        wd = plane(w[mine].astype(np.float32), 1, torch.float32)
        p.bind(n, cd, off=od, u=ud, w=wd, ids=idd)
        p.enable_deposit(True)
    else:
        p = P.Part(dec.grid(), P.FP64, P.TSC, P.LP_RK2, capacity=cap, nbins=NB)
        p.set_fields(torch.as_tensor(fl.reshape(ncomp, -1)).to(dev))
        chi, eng, n_old = _lp_init(x, f)
        xd = plane(x[:, mine], 3, torch.float64)
        chd = plane(chi[:, mine], NB, torch.float64)
        end = plane(eng[:, mine], NB, torch.float64)
        nod = plane(n_old[mine], 1, torch.float64)
        p.bind(n, xd, chi=chd, eng=end, n_old=nod, ids=idd)
    ops = M.LibOps(p, n)
    comm = M.Comm(dist)
    out = torch.zeros(3 * G, dtype=torch.float64, device=dev)
    for _ in range(STEPS):
        if mode == "lp":
            p.gather_push(0.0, dt, 1)
            p.spec_update(dt, C0, 0.0)
        else:
            p.sort()
            p.gather_push(1.0, dt, 1)
            p.deposit(out)
        M.exchange_particles(dec, ops, comm)
        if mode != "lp":
            M.accumulate_deposit(dec, ops, comm, out)
    p.sync()
    n = ops.n

    def rows(b, r):
        return b[: r * n].view(r, n).cpu().numpy()

    res = {"ids": rows(idd, 1)[0], "lo_g": dec.lo_g, "nl": dec.nl}
    if mode == "fp64":
        res.update(x=rows(xd, 3), u=rows(ud, 3))
    elif mode == "mixed":
        c = rows(cd, 1)[0].astype(np.int64)
        nl = dec.n_local
        jj = np.stack([c % nl[0], (c // nl[0]) % nl[1], c // (nl[0] * nl[1])])
        o = rows(od, 3).astype(np.float64)
        res.update(x=np.stack([dec.xmin_local[a] + (jj[a] + 0.5 + o[a]) * dec.dx[a]
                               for a in range(3)]),
                   u=rows(ud, 6)[:3].astype(np.float64) + rows(ud, 6)[3:].astype(np.float64))
    else:
        res.update(x=rows(xd, 3), chi=rows(chd, NB), eng=rows(end, NB))
    if mode != "lp":
        lo = dec.interior
        res["dep"] = out.view(3, *dec.n_local[::-1])[:, lo[2][0]:lo[2][1], lo[1][0]:lo[1][1],
                                                    lo[0][0]:lo[0][1]].cpu().numpy()
    return rank, res


def _reference(mode):
    f, x, u, w, ids, dt = _problem(mode)
    g = O.make_grid(3, (NG,) * 3)
    if mode == "mixed":
        # start from the positions the mixed form can hold (f32 offsets of the
        # global grid's cells: the local grids' cells are shifted by whole
        # cells, so their offsets are the same)
        s = (x + 1.0) * (NG / 2.0)
        j = np.floor(s)
        x = -1.0 + (j + 0.5 + (s - j - 0.5).astype(np.float32).astype(np.float64)) * (2.0 / NG)
        u = u.astype(np.float32).astype(np.float64)
        w = w.astype(np.float32).astype(np.float64)
        f = f.astype(np.float32).astype(np.float64)
    out = {"ids": ids}
    if mode == "lp":
        chi, eng, n_old = _lp_init(x, f)
        for _ in range(STEPS):
            x, nn, b2, gm = O.lp_rk2_step(g, O.TSC, f[:3], f[3:4], f[4:], x, dt)
            chi, eng, n_old = O.spec_update(chi, eng, n_old, nn, b2, gm, dt, C0)
        out.update(x=x, chi=chi, eng=eng)
        return out
    f6 = f.reshape(6, -1)
    for _ in range(STEPS):
        x, u, F, xo = O.boris_step(g, O.TSC, f6, x, u, w, 1.0, dt, True)
    out.update(x=x, u=u, dep=O.deposit(g, O.TSC, xo, F), dabs=O.deposit(g, O.TSC, xo, np.abs(F)))
    return out


@pytest.mark.parametrize("mode", ["fp64", "mixed", "lp"])
def test_two_ranks_one_gpu_match_one_domain(mode):
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, mode, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
    for g in got:
        assert not isinstance(g[1], str), g[2]
    res = [g[1] for g in sorted(got, key=lambda t: t[0])]
    ref = _reference(mode)
    ids = np.concatenate([r["ids"] for r in res])
    assert np.array_equal(np.sort(ids), np.sort(ref["ids"]))       # each id on one rank
    o, ro = np.argsort(ids), np.argsort(ref["ids"])
    x = np.concatenate([r["x"] for r in res], axis=1)[:, o]
    d = x - ref["x"][:, ro]
    d -= 2.0 * np.round(d / 2.0)
    if mode == "mixed":
        assert np.max(np.abs(d)) / (2.0 / NG) <= 1e-6 * STEPS
        u = np.concatenate([r["u"] for r in res], axis=1)[:, o]
        assert np.max(np.abs(u - ref["u"][:, ro])) <= 2e-6 * STEPS * np.max(np.abs(ref["u"]))
    else:
        assert np.max(np.abs(d)) <= 1e-12 * STEPS
    if mode == "fp64":
        u = np.concatenate([r["u"] for r in res], axis=1)[:, o]
        assert np.max(np.abs(u - ref["u"][:, ro])) <= 1e-12 * STEPS * np.max(np.abs(ref["u"]))
    if mode == "lp":
        for k in ("chi", "eng"):
            v = np.concatenate([r[k] for r in res], axis=1)[:, o]
            rv = ref[k][:, ro]
            assert np.max(np.abs(v - rv) / np.maximum(np.abs(rv), 1e-300)) <= 1e-12 * STEPS
        return
    dep = np.full((3, NG, NG, NG), np.nan)
    for r in res:
        lo, nl = r["lo_g"], r["nl"]
        dep[:, lo[2]:lo[2] + nl[2], lo[1]:lo[1] + nl[1], lo[0]:lo[0] + nl[0]] = r["dep"]
    dep = dep.reshape(3, -1)
    assert not np.any(np.isnan(dep))
    tol = 1e-12 if mode == "fp64" else 1e-5
    assert np.max(np.abs(dep - ref["dep"]) / np.maximum(ref["dabs"], 1e-300)) <= tol


def _replicated_rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2602_23434_b300 import _lib as P
        from paper_2602_23434_b300 import multirank as M
        torch.cuda.set_device(0)
        dev = torch.device("cuda", 0)
        f, x, u, w, ids, dt = _problem("fp64")
        sel = ids % world == rank                 # particles partitioned over the ranks
        n = int(sel.sum())
        p = P.Part(P.make_grid(3, NG), P.FP64, P.TSC, P.BORIS, capacity=n)
        p.set_fields(torch.as_tensor(f.reshape(6, -1)).to(dev))
        xd = torch.as_tensor(np.ascontiguousarray(x[:, sel])).to(dev)
        ud = torch.as_tensor(np.ascontiguousarray(u[:, sel])).to(dev)
        wd = torch.as_tensor(np.ascontiguousarray(w[sel])).to(dev)
        p.bind(n, xd, u=ud, w=wd)
        p.enable_deposit(True)
        p.sort()
        p.gather_push(1.0, dt, 1)
        out = torch.empty(3 * NG ** 3, dtype=torch.float64, device=dev)
        p.deposit(out)
        p.sync()
        tot = M.combine_replicated(M.LibOps(p, n), dist, out)
        torch.cuda.synchronize()
        q.put((rank, tot.cpu().numpy()))
    except Exception:
        import traceback
        q.put((rank, "error", traceback.format_exc()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_one_gpu_replicated_deposit_sum():
    """Fields replicated, particles split by id over two ranks: the ranks'
    deposits summed in rank order by part_sum_ordered equal the one-rank
    oracle deposit within 1e-12 of sum |contrib|, the same bits on both."""
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_replicated_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
    for g in got:
        assert not isinstance(g[1], str), g[2]
    res = dict(got)
    assert np.array_equal(res[0], res[1])
    f, x, u, w, ids, dt = _problem("fp64")
    g = O.make_grid(3, (NG,) * 3)
    _, _, F, xo = O.boris_step(g, O.TSC, f.reshape(6, -1), x, u, w, 1.0, dt, True)
    dref = O.deposit(g, O.TSC, xo, F).reshape(-1)
    dabs = O.deposit(g, O.TSC, xo, np.abs(F)).reshape(-1)
    assert np.max(np.abs(res[0] - dref) / np.maximum(dabs, 1e-300)) <= 1e-12


@pytest.mark.parametrize("mode", ["fp64", "mixed", "lp"])
def test_exchange_pack_unpack_every_plane_bit_exact(mode):
    """part_exchange_pack on rank 0 of a 2 x 1 x 1 split, part_exchange_unpack
    into rank 1's context (one process): every bound plane of every leaving
    particle arrives bit for bit, in index order, moved into the receiver's
    frame (FP64/LP: x + L across the seam; mixed: the cell re-based), LP shock
    flags included; the flags mark exactly the particles in halo cells."""
    from paper_2602_23434_b300 import _lib as P
    from paper_2602_23434_b300 import multirank as M
    dev = torch.device("cuda", 0)
    d0, d1 = (M.Decomp(3, (NG,) * 3, (2, 1, 1), r) for r in (0, 1))
    rng = np.random.default_rng(5)
    n, cap, nb = 3001, 8000, 6
    nl = d0.n_local
    # positions over rank 0's whole local grid: interior and both halo layers
    s = rng.uniform(0.0, 1.0, (3, n)) * np.array(nl)[:, None]
    s[:, :7] = [[0.0], [3.5], [4.5]]                 # exactly on the lower face
    x = np.array(d0.xmin_local)[:, None] + s * np.array(d0.dx)[:, None]
    ids = np.arange(n, dtype=np.int64) * 7 + 3
    mk = {"fp64": (P.FP64, P.BORIS, 0), "mixed": (P.MIXED, P.BORIS, 0), "lp": (P.FP64, P.LP_RK2, nb)}
    prec, mode_c, nbins = mk[mode]
    ctx = [P.Part(d.grid(), prec, P.TSC, mode_c, capacity=cap, nbins=nbins) for d in (d0, d1)]

    def buf(a, rows, dt):
        b = torch.zeros(rows * cap, dtype=dt, device=dev)
        b[: a.size] = torch.as_tensor(np.ascontiguousarray(a).reshape(-1)).to(dev)
        return b

    planes = {"ids": (ids, 1, torch.int64)}
    if mode == "fp64":
        planes.update(x=(x, 3, torch.float64), u=(rng.normal(0, 1, (3, n)), 3, torch.float64),
                      w=(rng.uniform(0.5, 2, n), 1, torch.float64))
    elif mode == "mixed":
        j = np.minimum(np.floor(s), np.array(nl)[:, None] - 1).astype(np.int64)
        cell = ((j[2] * nl[1] + j[1]) * nl[0] + j[0]).astype(np.int32)
        planes.update(x=(cell, 1, torch.int32),
                      off=((s - j - 0.5).astype(np.float32), 3, torch.float32),
                      u=(rng.normal(0, 1, (6, n)).astype(np.float32), 6, torch.float32),
                      w=(rng.uniform(0.5, 2, n).astype(np.float32), 1, torch.float32))
    else:
        planes.update(x=(x, 3, torch.float64), chi=(rng.uniform(0, 1, (nb, n)), nb, torch.float64),
                      eng=(np.sort(rng.uniform(1, 10, (nb, n)), axis=0), nb, torch.float64),
                      n_old=(rng.uniform(0.5, 2, n), 1, torch.float64))
    b0 = {k: buf(a, r, dt) for k, (a, r, dt) in planes.items()}
    ctx[0].bind(n, b0["x"], off=b0.get("off"), u=b0.get("u"), w=b0.get("w"), ids=b0["ids"],
                chi=b0.get("chi"), eng=b0.get("eng"), n_old=b0.get("n_old"))
    m = 11                                           # rank 1 already holds a few particles
    b1 = {k: buf(np.asarray(a)[..., :m] if np.asarray(a).ndim > 1 else np.asarray(a)[:m], r, dt)
          for k, (a, r, dt) in planes.items()}
    ctx[1].bind(m, b1["x"], off=b1.get("off"), u=b1.get("u"), w=b1.get("w"), ids=b1["ids"],
                chi=b1.get("chi"), eng=b1.get("eng"), n_old=b1.get("n_old"))
    shk0 = shk1 = None
    if mode == "lp":
        f7 = np.ones((7, int(np.prod(nl))))
        for c in ctx:
            c.set_fields(torch.as_tensor(f7).to(dev))
        shk0 = torch.as_tensor(rng.integers(0, 2, cap).astype(np.uint8)).to(dev)
        shk1 = torch.zeros(cap, dtype=torch.uint8, device=dev)
        ctx[0].enable_shocks(1.5, shk0)
        ctx[1].enable_shocks(1.5, shk1)
    sh0 = shk0.cpu().numpy()[:n].copy() if shk0 is not None else None
    to_l, to_r = d0.shifts(0)
    lo, hi = d0.interior[0]
    leaving = torch.zeros(n, dtype=torch.uint8, device=dev)
    big = torch.empty(ctx[0].exchange_bytes(n) + 8, dtype=torch.uint8, device=dev)
    big2 = torch.empty_like(big)
    kl, kr, ok = ctx[0].exchange_pack(0, lo, hi, to_l, to_r, big, big2, leaving)
    assert ok
    torch.cuda.synchronize()
    # the library's own rounding of s = (x - xmin) / dx (the cell index in mixed form)
    sx = s[0] if mode == "mixed" else (x[0] - d0.xmin_local[0]) * (1.0 / d0.dx[0])
    left, right = sx < lo, sx >= hi
    assert (kl, kr) == (int(left.sum()), int(right.sum())) and kl > 0 and kr > 0
    assert np.array_equal(leaving.cpu().numpy(), (left | right).astype(np.uint8))
    # the right-moving ones into rank 1 (its left neighbour is rank 0)
    ctx[1].exchange_unpack(kr, big2[: ctx[1].exchange_bytes(kr)])
    ctx[1].sync()
    sel = np.nonzero(right)[0]
    tot = m + kr
    for k, (a, rows, dt) in planes.items():
        got = b1[k][: rows * tot].view(rows, tot).cpu().numpy()[:, m:]
        want = np.asarray(a).reshape(rows, -1)[:, sel].copy()
        if k == "x" and mode != "mixed":
            want[0] = want[0] + to_r[0]
        if k == "x" and mode == "mixed":
            c = want[0].astype(np.int64)
            jx, jy, jz = c % nl[0], (c // nl[0]) % nl[1], c // (nl[0] * nl[1])
            n1 = d1.n_local
            want[0] = ((jz * n1[1] + jy) * n1[0] + jx + to_r[1]).astype(np.int32)
        assert np.array_equal(got, want), k
    if mode == "lp":
        assert np.array_equal(shk1.cpu().numpy()[m:tot], sh0[sel])
