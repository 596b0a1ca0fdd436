"""Several ranks: domain decomposition with particle exchange (Sec. 3.3,
"Multi-core communication") and the cross-rank sum of the deposit.

Two ways to split the particle step over ranks, both driven through libpart:

* ``Decomp`` + ``exchange_particles`` + ``accumulate_deposit``: the grid is
  cut into boxes over a Cartesian process grid.  Each rank's context covers
  its box plus, along every split axis, one halo cell per side holding the
  neighbour's fields (those axes are open in the local grid).  After a push,
  the particles in a halo cell are exchanged with the neighbours, one axis
  after the other (the paper's three directions, its eight steps per
  direction); the deposit's halo planes are sent to their owners and added
  there, so every rank ends with the complete deposit of its interior.
* ``combine_replicated``: particles partitioned over ranks, fields
  replicated; every rank deposits onto the whole grid and the grids are summed
  in rank order (a reduce-scatter by all-to-all, the library's ordered sum,
  then an all-gather), so every rank holds the same bits.

The data path runs in the library's kernels (part_exchange_pack / _unpack,
part_compact, part_box_pack / _add, part_sum_ordered); this module sequences
them and the torch.distributed messages.  Device work goes through an ``ops``
object -- ``LibOps`` here -- so the host protocol can also be driven by a
test double on processes without a GPU.
"""
from __future__ import annotations

import math

from . import _lib as P


# ----------------------------------------------------------------------------- geometry
class Decomp:
    """Cartesian split of an n[0] x n[1] x n[2] periodic grid on
    [xmin, xmin + L) over pdims[0] x pdims[1] x pdims[2] ranks (rank =
    (cz * py + cy) * px + cx).  Axis a of rank r holds the global cells
    [lo_g[a], lo_g[a] + nl[a]) with lo_g = c n / p (integer division), plus
    h[a] = `halo` cells per side when the axis is split.

    halo = 1 suffices for the Boris push: it gathers at x^n, inside the
    interior, so its stencil reaches one cell out, and so does its deposit.
    The LP push needs halo = 2: its Heun step samples the velocity at x* and
    the fluid at x^{n+1}, up to a cell outside the interior, and the stencil
    there reaches one cell further."""

    def __init__(self, dim: int, n, pdims, rank: int, xmin=(-1.0, -1.0, -1.0),
                 L=(2.0, 2.0, 2.0), halo: int = 1):
        n = list(n) + [1] * (3 - len(n))
        pdims = list(pdims) + [1] * (3 - len(pdims))
        if dim == 2:
            n[2], pdims[2] = 1, 1
        self.dim, self.n, self.pdims = dim, n, pdims
        self.world = pdims[0] * pdims[1] * pdims[2]
        if not 0 <= rank < self.world:
            raise ValueError("rank outside the process grid")
        if halo < 1:
            raise ValueError("halo must be >= 1")
        self.rank = rank
        self.halo = halo
        self.coords = self.coords_of(rank)
        self.xmin, self.L = [float(v) for v in xmin], [float(v) for v in L]
        self.dx = [self.L[a] / n[a] for a in range(3)]
        self.split, self.h, self.lo_g, self.nl = [], [], [], []
        for a in range(3):
            p = pdims[a]
            if p > 1 and (a >= dim or n[a] < max(2, halo) * p):
                raise ValueError(f"axis {a}: cannot split {n[a]} cells over {p} ranks")
            lo = self.coords[a] * n[a] // p
            hi = (self.coords[a] + 1) * n[a] // p
            self.split.append(p > 1)
            self.h.append(halo if p > 1 else 0)
            self.lo_g.append(lo)
            self.nl.append(hi - lo)
        self.n_local = [self.nl[a] + 2 * self.h[a] for a in range(3)]
        self.xmin_local = [self.xmin[a] + (self.lo_g[a] - self.h[a]) * self.dx[a]
                           for a in range(3)]
        self.interior = [(self.h[a], self.h[a] + self.nl[a]) for a in range(3)]

    def coords_of(self, rank: int):
        px, py, _ = self.pdims
        return [rank % px, (rank // px) % py, rank // (px * py)]

    def rank_of(self, coords) -> int:
        px, py, pz = self.pdims
        c = [coords[0] % px, coords[1] % py, coords[2] % pz]
        return (c[2] * py + c[1]) * px + c[0]

    def neighbors(self, a: int):
        """(left, right) ranks along axis a (periodic)."""
        cl, cr = list(self.coords), list(self.coords)
        cl[a] -= 1
        cr[a] += 1
        return self.rank_of(cl), self.rank_of(cr)

    def nl_of(self, a: int, c: int) -> int:
        p = self.pdims[a]
        c %= p
        return (c + 1) * self.n[a] // p - c * self.n[a] // p

    def grid(self):
        """The rank's part_grid: its box plus halo cells, open along split axes,
        with the whole domain's dx."""
        return P.make_grid(self.dim, self.n_local, xmin=self.xmin_local,
                           L=[self.n_local[a] * self.dx[a] for a in range(3)],
                           open_axes=[1 if s else 0 for s in self.split], dx=self.dx)

    def shifts(self, a: int):
        """(to_left, to_right) as part_xshift tuples (dx, dj, n_axis) along a:
        FP64/LP positions move by one period across the domain's seam; mixed
        cell indices are re-based into the receiver's box (halo cell h - 1
        is the left neighbour's last interior cell h + nl_left - 1, halo cell
        h + nl the right neighbour's first interior cell h)."""
        p, c, h = self.pdims[a], self.coords[a], self.h[a]
        nl_left, nl_right = self.nl_of(a, c - 1), self.nl_of(a, c + 1)
        to_left = (self.L[a] if c == 0 else 0.0, nl_left, nl_left + 2 * h)
        to_right = (-self.L[a] if c == p - 1 else 0.0, -self.nl[a], nl_right + 2 * h)
        return to_left, to_right

    def local_index(self, a: int):
        """Global cell indices of the local grid's cells along axis a."""
        return [(self.lo_g[a] - self.h[a] + i) % self.n[a] for i in range(self.n_local[a])]

    def local_fields(self, fields):
        """Fields [ncomp][nz][ny][nx] of the whole grid (numpy or torch) -> the
        rank's box with halos, contiguous, same type."""
        f = fields
        for a, dimaxis in ((0, 3), (1, 2), (2, 1)):
            idx = self.local_index(a)
            if hasattr(f, "index_select"):
                import torch
                f = f.index_select(dimaxis, torch.as_tensor(idx, device=f.device))
            else:
                import numpy as np
                f = np.take(f, idx, axis=dimaxis)
        return f.contiguous() if hasattr(f, "contiguous") else f.copy()

    def halo_boxes(self, a: int):
        """Boxes (lo, ext) of one deposit exchange along axis a: the h left and
        h right halo planes to send, and where the received planes are added
        (the first and the last h interior planes).  Along axes exchanged
        before a the boxes span the interior only (their halos have gone to
        their owners); along the others, the whole local extent."""
        lo, ext = [0, 0, 0], list(self.n_local)
        for b in range(3):
            if b < a and self.split[b]:
                lo[b], ext[b] = self.h[b], self.nl[b]
        h = self.h[a]
        ext[a] = h
        send_l, send_r, add_l, add_r = (list(lo) for _ in range(4))
        send_l[a] = 0
        send_r[a] = h + self.nl[a]
        add_l[a] = h                                  # from the left: its right halo
        add_r[a] = self.nl[a]                         # from the right: its left halo
        return send_l, send_r, add_l, add_r, ext


# ----------------------------------------------------------------------------- messages
class Comm:
    """Neighbour messages over torch.distributed.  Buffers are 1-D tensors;
    with the gloo backend, device tensors travel through host copies."""

    def __init__(self, dist, group=None):
        self.dist, self.group = dist, group
        self.gloo = dist.get_backend(group) == "gloo"

    def _host(self, t):
        return t.cpu() if (self.gloo and t.is_cuda) else t

    def sendrecv(self, a: int, left: int, right: int, send_left, send_right, recv_from_right,
                 recv_from_left):
        """Send send_left to the left neighbour and send_right to the right one;
        receive the left-moving message from the right neighbour and the
        right-moving one from the left neighbour (tags keep the two apart
        when both neighbours are one rank)."""
        d = self.dist
        sl, sr = self._host(send_left), self._host(send_right)
        rr, rl = self._host(recv_from_right), self._host(recv_from_left)
        tl, tr = 2 * a, 2 * a + 1
        if self.gloo:
            reqs = [d.isend(sl, left, group=self.group, tag=tl),
                    d.isend(sr, right, group=self.group, tag=tr),
                    d.irecv(rr, right, group=self.group, tag=tl),
                    d.irecv(rl, left, group=self.group, tag=tr)]
            for q in reqs:
                q.wait()
        else:
            ops = [d.P2POp(d.isend, sl, left, self.group, tl),
                   d.P2POp(d.isend, sr, right, self.group, tr),
                   d.P2POp(d.irecv, rr, right, self.group, tl),
                   d.P2POp(d.irecv, rl, left, self.group, tr)]
            for q in d.batch_isend_irecv(ops):
                q.wait()
        if rr is not recv_from_right:
            recv_from_right.copy_(rr)
        if rl is not recv_from_left:
            recv_from_left.copy_(rl)


# ----------------------------------------------------------------------------- device ops
class LibOps:
    """The device side of the protocol on one library context."""

    def __init__(self, part, n: int):
        self.part, self.torch = part, part.torch
        self.n = n                      # particles bound now
        self.dev = part.device
        self._send = [None, None]

    def _buf(self, i: int, nbytes: int):
        b = self._send[i]
        if b is None or b.numel() < nbytes:
            b = self.torch.empty(max(8, int(nbytes * 1.25)), dtype=self.torch.uint8,
                                 device=self.dev)
            self._send[i] = b
        return b

    def bytes_for(self, k: int) -> int:
        return max(8, self.part.exchange_bytes(k))

    def pack(self, a: int, lo: int, hi: int, to_left, to_right):
        t = self.torch
        leaving = t.empty(max(self.n, 1), dtype=t.uint8, device=self.dev)
        bl, br = self._buf(0, 8), self._buf(1, 8)
        kl, kr, ok = self.part.exchange_pack(a, lo, hi, to_left, to_right, bl, br, leaving)
        if not ok:
            bl, br = self._buf(0, self.bytes_for(kl)), self._buf(1, self.bytes_for(kr))
            kl, kr, ok = self.part.exchange_pack(a, lo, hi, to_left, to_right, bl, br, leaving)
            assert ok
        return kl, kr, bl[: self.bytes_for(kl)], br[: self.bytes_for(kr)], leaving

    def recv_buffer(self, k: int):
        return self.torch.empty(self.bytes_for(k), dtype=self.torch.uint8, device=self.dev)

    def count_tensor(self, k: int):
        return self.torch.tensor([int(k)], dtype=self.torch.int64, device=self.dev)

    def compact(self, leaving):
        self.n = self.part.compact(leaving)

    def unpack(self, k: int, buf):
        if k:
            self.part.exchange_unpack(k, buf)
            self.n += k

    def box_pack(self, arr, ncomp, dims, lo, ext):
        out = self.torch.empty(ncomp * ext[0] * ext[1] * ext[2], dtype=self.torch.float64,
                               device=self.dev)
        P.box_pack(arr, ncomp, dims, lo, ext, out, self.part.stream.cuda_stream)
        return out

    def box_add(self, arr, ncomp, dims, lo, ext, src):
        P.box_add(arr, ncomp, dims, lo, ext, src, self.part.stream.cuda_stream)

    def empty_f64(self, k: int):
        return self.torch.empty(k, dtype=self.torch.float64, device=self.dev)

    def sum_ordered(self, parts):
        out = self.torch.empty(parts.shape[1], dtype=self.torch.float64, device=self.dev)
        P.sum_ordered(out, parts.contiguous(), self.part.stream.cuda_stream)
        return out

    def sync(self):
        self.part.stream.synchronize()


# ----------------------------------------------------------------------------- protocol
def exchange_particles(dec: Decomp, ops, comm: Comm) -> int:
    """Move every particle that a push took into a halo cell to the rank that
    owns it: per split axis, the paper's eight steps (flag and count, post the
    receives, size the buffers, pack, send, resize, wait, fill the holes and
    compact).  Returns the rank's particle count afterwards."""
    for a in range(dec.dim):
        if not dec.split[a]:
            continue
        left, right = dec.neighbors(a)
        to_left, to_right = dec.shifts(a)
        lo, hi = dec.interior[a]
        kl, kr, bl, br, leaving = ops.pack(a, lo, hi, to_left, to_right)
        # counts first, so each side can size its receive buffers
        c_from_r, c_from_l = ops.count_tensor(0), ops.count_tensor(0)
        comm.sendrecv(a, left, right, ops.count_tensor(kl), ops.count_tensor(kr), c_from_r,
                      c_from_l)
        kfr, kfl = int(c_from_r.item()), int(c_from_l.item())
        rr, rl = ops.recv_buffer(kfr), ops.recv_buffer(kfl)
        ops.sync()                       # packed buffers complete before they are sent
        comm.sendrecv(a, left, right, bl, br, rr, rl)
        ops.compact(leaving)
        ops.unpack(kfl, rl)              # from the left first, then from the right
        ops.unpack(kfr, rr)
    return ops.n


def accumulate_deposit(dec: Decomp, ops, comm: Comm, grid3) -> None:
    """grid3: the rank's deposit [3][nz][ny][nx] over its local grid (halos
    included), flat or shaped, contiguous.  Adds the neighbours' halo planes
    into the interior, axis after axis (corner contributions travel on), so
    the interior holds the whole deposit of its cells."""
    dims = dec.n_local
    for a in range(dec.dim):
        if not dec.split[a]:
            continue
        left, right = dec.neighbors(a)
        send_l, send_r, add_l, add_r, ext = dec.halo_boxes(a)
        pl = ops.box_pack(grid3, 3, dims, send_l, ext)
        pr = ops.box_pack(grid3, 3, dims, send_r, ext)
        nbox = 3 * ext[0] * ext[1] * ext[2]
        rr, rl = ops.empty_f64(nbox), ops.empty_f64(nbox)
        ops.sync()
        comm.sendrecv(a, left, right, pl, pr, rr, rl)
        ops.box_add(grid3, 3, dims, add_l, ext, rl)   # from the left first
        ops.box_add(grid3, 3, dims, add_r, ext, rr)


def combine_replicated(ops, dist, grid_flat, group=None):
    """Rank-ordered sum of every rank's whole-grid deposit (1-D float64
    tensor of `count` values): slice s of all ranks' grids goes to rank s
    (all-to-all), which adds them in rank order (part_sum_ordered); the summed
    slices are then gathered by every rank.  Returns the summed grid, the
    same bits on every rank."""
    torch = ops.torch
    world = dist.get_world_size(group)
    if world == 1:
        return grid_flat
    count = grid_flat.numel()
    s = math.ceil(count / world)
    gloo = dist.get_backend(group) == "gloo"
    send = torch.zeros(world * s, dtype=torch.float64, device=grid_flat.device)
    send[:count] = grid_flat
    if gloo and send.is_cuda:
        hs = send.cpu()
        hr = torch.empty_like(hs)
        dist.all_to_all_single(hr, hs, group=group)
        recv = hr.to(send.device)
    else:
        recv = torch.empty_like(send)
        dist.all_to_all_single(recv, send, group=group)
    mine = ops.sum_ordered(recv.view(world, s))
    ops.sync()
    if gloo and mine.is_cuda:
        parts = [torch.empty(s, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(parts, mine.cpu(), group=group)
        out = torch.cat(parts).to(grid_flat.device)
    else:
        parts = [torch.empty_like(mine) for _ in range(world)]
        dist.all_gather(parts, mine, group=group)
        out = torch.cat(parts)
    return out[:count]
