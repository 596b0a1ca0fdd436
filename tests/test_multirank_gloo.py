"""Several ranks on CPU processes (gloo): the host protocol of the domain
decomposition (Sec. 3.3, "Multi-core communication") and the rank-ordered
sum of replicated deposits, driven by a test double of the device calls.

The double does on the host what the library does on the device: the push
and deposit are the oracle's (on each rank's local grid: its box plus halo
cells, open along split axes), the pack classifies with the library's
rounding of s = (x - xmin) / dx, the compaction is the oracle's hole/filler
map.  Everything else -- neighbours, the periodic seam, the order of the
axes, counts before buffers, the deposit halo planes -- is the product's
``multirank`` module.

Checked against one oracle run on the whole periodic grid after four steps:
every id on exactly one rank, inside that rank's box; positions and momenta
within 1e-12 per step (the local grids round the cell offsets differently
from the whole grid, by an ulp); the deposit of the last step, assembled from
the ranks' interiors, within 1e-12 of the sum of |contributions| per cell.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import oracle as O
from paper_2602_23434_b300 import multirank as M
from paper_2602_23434_b300 import synth

N_GLOBAL, PPC, STEPS, SEED = 16, 3, 4, 77


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class NpOps:
    """Host test double of multirank.LibOps (FP64 Boris particles)."""

    def __init__(self, dec, x, u, w, ids):
        self.dec = dec
        self.g = O.make_grid(dec.dim, dec.n_local, xmin=dec.xmin_local, dx=dec.dx,
                             open_axes=[1 if s else 0 for s in dec.split])
        self.x, self.u, self.w, self.ids = x, u, w, ids
        self.n = ids.shape[0]
        self.torch = torch

    # the step the library would run: gather + Boris + drift, deposit at x^n
    def step(self, f_local, qm, dt):
        x1, u1, F, xo = O.boris_step(self.g, O.TSC, f_local, self.x, self.u, self.w, qm, dt,
                                     True)
        dep = O.deposit(self.g, O.TSC, xo, F)
        self.x, self.u = x1, u1
        return dep

    def _rec(self, sel):
        return np.concatenate([self.ids[sel].astype(np.float64)[None], self.x[:, sel],
                               self.u[:, sel], self.w[sel][None]]).reshape(-1)

    def pack(self, a, lo, hi, to_left, to_right):
        s = (self.x[a] - self.dec.xmin_local[a]) * (1.0 / self.dec.dx[a])
        left, right = s < lo, s >= hi
        bl, br = self._rec(left).reshape(8, -1), self._rec(right).reshape(8, -1)
        bl[1 + a] = bl[1 + a] + to_left[0]
        br[1 + a] = br[1 + a] + to_right[0]
        lv = (left | right).astype(np.uint8)
        return (int(left.sum()), int(right.sum()), torch.as_tensor(bl.reshape(-1).copy()),
                torch.as_tensor(br.reshape(-1).copy()), lv)

    def recv_buffer(self, k):
        return torch.empty(8 * k, dtype=torch.float64)

    def count_tensor(self, k):
        return torch.tensor([int(k)], dtype=torch.int64)

    def compact(self, leaving):
        nk, src = O.compact_map(leaving)
        self.x, self.u, self.w, self.ids = (self.x[:, src], self.u[:, src], self.w[src],
                                            self.ids[src])
        self.n = nk

    def unpack(self, k, buf):
        if not k:
            return
        r = buf.numpy().reshape(8, k)
        self.ids = np.concatenate([self.ids, r[0].astype(np.int64)])
        self.x = np.concatenate([self.x, r[1:4]], axis=1)
        self.u = np.concatenate([self.u, r[4:7]], axis=1)
        self.w = np.concatenate([self.w, r[7]])
        self.n += k

    @staticmethod
    def _view(arr, dims):
        return arr.reshape(3, dims[2], dims[1], dims[0])

    def box_pack(self, arr, ncomp, dims, lo, ext):
        v = self._view(arr, dims)
        return torch.as_tensor(v[:, lo[2]:lo[2] + ext[2], lo[1]:lo[1] + ext[1],
                                 lo[0]:lo[0] + ext[0]].reshape(-1).copy())

    def box_add(self, arr, ncomp, dims, lo, ext, src):
        v = self._view(arr, dims)
        v[:, lo[2]:lo[2] + ext[2], lo[1]:lo[1] + ext[1], lo[0]:lo[0] + ext[0]] += \
            src.numpy().reshape(3, ext[2], ext[1], ext[0])

    def empty_f64(self, k):
        return torch.empty(k, dtype=torch.float64)

    def sum_ordered(self, parts):
        p = parts.numpy()
        out = p[0].copy()
        for r in range(1, p.shape[0]):
            out = out + p[r]
        return torch.as_tensor(out)

    def sync(self):
        pass


def _problem():
    f = synth.em_fields(3, N_GLOBAL, SEED, v_rms=0.05)
    N = N_GLOBAL ** 3 * PPC
    x, u, w, ids = synth.particles(3, None, N, SEED, u_th=0.3)
    w = np.random.default_rng(SEED).uniform(0.5, 2.0, N)
    dt = 0.5 * 2.0 / N_GLOBAL
    return f, x, u, w, ids.astype(np.int64), dt


def _reference():
    f, x, u, w, ids, dt = _problem()
    g = O.make_grid(3, (N_GLOBAL,) * 3)
    f6 = f.reshape(6, -1)
    dep = None
    for _ in range(STEPS):
        x, u, F, xo = O.boris_step(g, O.TSC, f6, x, u, w, 1.0, dt, True)
        dep = O.deposit(g, O.TSC, xo, F)
        dabs = O.deposit(g, O.TSC, xo, np.abs(F))
    return x, u, ids, dep, dabs


def _decomposed(rank, world, pdims, port, q, halo=1):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put(_decomposed_body(rank, pdims, halo))
    except Exception:                           # report to the parent, do not hang it
        import traceback
        q.put((rank, "error", traceback.format_exc()))
    finally:
        dist.destroy_process_group()


def _decomposed_body(rank, pdims, halo):
    dec = M.Decomp(3, (N_GLOBAL,) * 3, pdims, rank, halo=halo)
    f, x, u, w, ids, dt = _problem()
    fl = dec.local_fields(f).reshape(6, -1)
    # the particles of this rank's interior, by the local grid's rounding
    mine = np.ones(ids.shape[0], bool)
    for a in range(3):
        s = (x[a] - dec.xmin_local[a]) * (1.0 / dec.dx[a])
        mine &= (s >= dec.interior[a][0]) & (s < dec.interior[a][1])
    ops = NpOps(dec, x[:, mine], u[:, mine], w[mine], ids[mine])
    comm = M.Comm(dist)
    for _ in range(STEPS):
        dep = ops.step(fl, 1.0, dt)
        M.exchange_particles(dec, ops, comm)
        M.accumulate_deposit(dec, ops, comm, dep)
    lo, nl = dec.interior, dec.nl
    inner = dep.reshape(3, *dec.n_local[::-1])[:, lo[2][0]:lo[2][1], lo[1][0]:lo[1][1],
                                               lo[0][0]:lo[0][1]]
    # each particle inside this rank's box
    for a in range(3):
        s = (ops.x[a] - dec.xmin_local[a]) * (1.0 / dec.dx[a])
        assert np.all((s >= lo[a][0]) & (s < lo[a][1])), "a particle outside its box"
    return (rank, ops.ids, ops.x, ops.u, dec.lo_g, nl, inner.copy())


def _run(pdims, halo=1):
    world = int(np.prod(pdims))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_decomposed, args=(r, world, pdims, port, q, halo))
             for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
    for o in out:
        assert not isinstance(o[1], str), o[2]
    for p in procs:
        assert p.exitcode == 0
    return out


@pytest.mark.parametrize("pdims,halo", [((2, 1, 1), 1), ((4, 1, 1), 1), ((2, 2, 1), 1),
                                        ((2, 2, 2), 1), ((2, 2, 1), 2)])
def test_decomposed_run_matches_one_domain(pdims, halo):
    out = _run(pdims, halo)
    xr, ur, idr, dref, dabs = _reference()
    ids = np.concatenate([o[1] for o in out])
    assert np.array_equal(np.sort(ids), np.sort(idr))            # each id once
    x = np.concatenate([o[2] for o in out], axis=1)
    u = np.concatenate([o[3] for o in out], axis=1)
    order = np.argsort(ids)
    ref = np.argsort(idr)
    dxp = x[:, order] - xr[:, ref]
    dxp -= 2.0 * np.round(dxp / 2.0)
    assert np.max(np.abs(dxp)) <= 1e-12 * STEPS
    assert np.max(np.abs(u[:, order] - ur[:, ref])) <= 1e-12 * STEPS * np.max(np.abs(ur))
    # the last deposit, assembled from the interiors
    n = N_GLOBAL
    dep = np.full((3, n, n, n), np.nan)
    for _, _, _, _, lo_g, nl, inner in out:
        dep[:, lo_g[2]:lo_g[2] + nl[2], lo_g[1]:lo_g[1] + nl[1],
            lo_g[0]:lo_g[0] + nl[0]] = inner
    dep = dep.reshape(3, -1)
    assert not np.any(np.isnan(dep))
    assert np.max(np.abs(dep - dref) / np.maximum(dabs, 1e-300)) <= 1e-12


def _replicated(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        f, x, u, w, ids, dt = _problem()
        g = O.make_grid(3, (N_GLOBAL,) * 3)
        sel = ids % world == rank                     # particles partitioned over ranks
        _, _, F, xo = O.boris_step(g, O.TSC, f.reshape(6, -1), x[:, sel], u[:, sel], w[sel],
                                   1.0, dt, True)
        mine = O.deposit(g, O.TSC, xo, F).reshape(-1)
        ops = NpOps.__new__(NpOps)
        ops.torch = torch
        tot = M.combine_replicated(ops, dist, torch.as_tensor(mine))
        q.put((rank, tot.numpy().copy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_replicated_deposit_sum(world):
    """Particles split over ranks, fields replicated: the rank-ordered sum of
    the ranks' deposits equals the one-rank deposit within 1e-12 of
    sum |contrib| per cell, with the same bits on every rank."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_replicated, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=240) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    f, x, u, w, ids, dt = _problem()
    g = O.make_grid(3, (N_GLOBAL,) * 3)
    _, _, F, xo = O.boris_step(g, O.TSC, f.reshape(6, -1), x, u, w, 1.0, dt, True)
    dref = O.deposit(g, O.TSC, xo, F).reshape(-1)
    dabs = O.deposit(g, O.TSC, xo, np.abs(F)).reshape(-1)
    for r in range(1, world):
        assert np.array_equal(out[r], out[0])
    assert np.max(np.abs(out[0] - dref) / np.maximum(dabs, 1e-300)) <= 1e-12


def test_decomp_geometry():
    """Boxes tile the grid, halos and shifts are consistent between neighbours."""
    n, pd = (17, 12, 9), (3, 2, 1)
    decs = [M.Decomp(3, n, pd, r) for r in range(6)]
    for a in range(3):
        cover = sorted((d.lo_g[a], d.lo_g[a] + d.nl[a]) for d in decs)
        assert cover[0][0] == 0 and cover[-1][1] == n[a]
    for d in decs:
        for a in range(2):
            left, right = d.neighbors(a)
            tl, tr = d.shifts(a)
            dl, dr = decs[left], decs[right]
            assert tl[2] == dl.n_local[a] and tr[2] == dr.n_local[a]
            # the left halo cell is the left neighbour's last interior cell
            assert d.local_index(a)[0] == dl.local_index(a)[dl.interior[a][1] - 1]
            assert d.local_index(a)[-1] == dr.local_index(a)[dr.interior[a][0]]
            # the mixed form's re-based cell index lands on those cells
            assert 0 + tl[1] == dl.interior[a][1] - 1
            assert (d.n_local[a] - 1) + tr[1] == dr.interior[a][0]
        assert not d.split[2] and d.h[2] == 0
