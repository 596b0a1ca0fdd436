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
