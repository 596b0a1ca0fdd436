"""ctypes binding of libpart.so (include/part.h), argument marshalling only.

Every computation runs in the CUDA library; this module turns torch tensors
into device pointers, allocates the caller-owned workspace with torch, and
raises PartError on any non-OK status.  If libpart.so is missing or cannot be
loaded the import fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libpart.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "part.h")

FP64, MIXED = 0, 1
CIC, TSC = 1, 2
BORIS, LP_RK2 = 0, 1

STATUS = {0: "PART_OK", 1: "PART_EINVAL", 2: "PART_ENOMEM", 3: "PART_ECUDA",
          4: "PART_ETIMEOUT", 5: "PART_ENONFINITE", 6: "PART_EUNSUPPORTED",
          7: "PART_EDOMAIN"}


class PartError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.name = STATUS.get(code, str(code))


class Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("xmin", C.c_double * 3),
                ("dx", C.c_double * 3), ("periodic", C.c_int * 3)]


def make_grid(dim: int, n, xmin=(-1.0, -1.0, -1.0), L=(2.0, 2.0, 2.0),
              open_axes=(0, 0, 0), dx=None) -> Grid:
    """Grid of n cells per axis on [xmin, xmin + L); dim 2 -> n[2] = 1;
    periodic, except the axes with open_axes[a] = 1 (outflow).  dx, if
    given, sets the cell widths directly (a subdomain's grid keeps the whole
    domain's dx bit for bit)."""
    if isinstance(n, int):
        n = (n, n, n if dim == 3 else 1)
    n = list(n) + [1] * (3 - len(n))
    if dim == 2:
        n[2] = 1
    g = Grid()
    g.dim = dim
    for a in range(3):
        g.n[a] = int(n[a])
        g.xmin[a] = float(xmin[a])
        if dx is not None:
            g.dx[a] = float(dx[a])
        else:
            g.dx[a] = float(L[a]) / n[a] if (a < dim) else float(L[a])
        g.periodic[a] = 0 if open_axes[a] else 1
    return g


class WorkItem(C.Structure):
    """part_work_item of include/part.h (72 bytes)."""
    _fields_ = [("cell", C.c_void_p), ("off", C.c_void_p), ("u", C.c_void_p),
                ("stride", C.c_int64), ("first", C.c_int64), ("count", C.c_int32),
                ("nsteps", C.c_int32), ("snapshot", C.c_int32), ("reserved", C.c_int32),
                ("q_over_m", C.c_double), ("dt", C.c_double)]


class XShift(C.Structure):
    """part_xshift: a packed particle's move into the receiver's frame."""
    _fields_ = [("dx", C.c_double), ("dj", C.c_int32), ("n_axis", C.c_int32)]


if C.sizeof(WorkItem) != 72:
    raise ImportError("part_work_item layout mismatch with include/part.h (72 bytes)")

_lib = None


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_2602_23434_b300/build.py "
                          "(there is no CPU fallback)")
    L = C.CDLL(LIB_PATH)
    P = C.c_void_p
    G = C.POINTER(Grid)
    st = C.c_int
    sigs = {
        "part_brick_dims": (st, [G, C.POINTER(C.c_int), C.POINTER(C.c_int64)]),
        "part_workspace_size": (st, [G, C.c_int, C.c_int, C.c_int64, C.c_int,
                                     C.POINTER(C.c_size_t)]),
        "part_init": (st, [C.POINTER(P), G, C.c_int, C.c_int, C.c_int, C.c_int64, C.c_int, P,
                           C.c_size_t, P]),
        "part_destroy": (st, [P]),
        "part_set_fields": (st, [P, P, C.c_int, C.c_int]),
        "part_bind_particles": (st, [P, C.c_int64, P, P, P, P, P, P, P, P]),
        "part_sort": (st, [P]),
        "part_cell_start": (st, [P, C.POINTER(P), C.POINTER(C.c_int64)]),
        "part_compact": (st, [P, P, C.POINTER(C.c_int64)]),
        "part_enable_shocks": (st, [P, C.c_double, P]),
        "part_set_lp_order": (st, [P, C.c_int]),
        "part_set_lp_arith": (st, [P, C.c_int]),
        "part_set_spec_lazy": (st, [P, C.c_int]),
        "part_flush": (st, [P]),
        "part_set_outflow": (st, [P, P]),
        "part_shock_cells": (st, [P, C.POINTER(P), C.POINTER(C.c_int64)]),
        "part_set_shock_slope": (st, [P, C.c_int]),
        "part_shock_slopes": (st, [P, C.POINTER(P), C.POINTER(C.c_int64)]),
        "part_enable_deposit": (st, [P, C.c_int]),
        "part_gather_push": (st, [P, C.c_double, C.c_double, C.c_int]),
        "part_deposit": (st, [P, P]),
        "spec_update": (st, [P, C.c_double, C.c_double, C.c_double]),
        "part_init_particles": (st, [P, C.c_uint64, C.c_double, C.c_double, C.c_double,
                                     C.c_double, C.c_double]),
        "part_sync": (st, [P]),
        "part_last_error": (C.c_char_p, [P]),
        "part_launch_count": (C.c_int64, [P]),
        "part_selftest_wait": (st, [P, C.c_int64, C.c_int]),
        "part_inject": (st, [P, C.c_int64, P, P, P, P, P, P, P, P]),
        "part_sort_fp64_noalloc": (st, [G, C.c_int64, P, P, P, P, P, P]),
        "part_probe_fp64_fma": (st, [P, P, C.c_int, C.c_int, C.c_int,
                                     C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "part_exchange_bytes": (st, [P, C.c_int64, C.POINTER(C.c_size_t)]),
        "part_exchange_pack": (st, [P, C.c_int, C.c_int, C.c_int, C.POINTER(XShift),
                                    C.POINTER(XShift), P, C.c_size_t, P, C.c_size_t, P,
                                    C.POINTER(C.c_int64)]),
        "part_exchange_unpack": (st, [P, C.c_int64, P, C.c_size_t]),
        "part_box_pack": (st, [P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                               C.POINTER(C.c_int), P, P]),
        "part_box_add": (st, [P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                              C.POINTER(C.c_int), P, P]),
        "part_sum_ordered": (st, [P, P, C.c_int64, C.c_int, P]),
        "part_server_sizes": (st, [C.c_int, C.c_int, C.POINTER(C.c_size_t),
                                   C.POINTER(C.c_size_t)]),
        "part_server_init": (st, [C.POINTER(P), C.POINTER(P), C.c_int, C.c_int, P, C.c_size_t,
                                  P, C.c_size_t, P, C.c_int, C.c_int]),
        "part_server_items": (C.POINTER(WorkItem), [P]),
        "part_server_run": (st, [P, C.c_int]),
        "part_server_sync": (st, [P]),
        "part_server_destroy": (st, [P]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def header_functions(path: str = HEADER) -> list[str]:
    """Names of the functions include/part.h declares."""
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(",
                                 txt, flags=re.M)) - {"if", "while"})


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


class Part:
    """One library context: workspace, stream, bound particles and fields."""

    def __init__(self, grid: Grid, prec: int = FP64, shape: int = TSC, mode: int = BORIS,
                 capacity: int = 0, nbins: int = 0, stream=None, device=None):
        import torch
        self.torch = torch
        self.L = lib()
        self.grid = grid
        self.prec, self.shape, self.mode = prec, shape, mode
        self.capacity, self.nbins = capacity, nbins
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = C.c_size_t()
        self._check(self.L.part_workspace_size(C.byref(grid), prec, mode, capacity, nbins,
                                               C.byref(nbytes)), None)
        self.ws_bytes = nbytes.value
        # torch's caching allocator returns 512-byte aligned blocks
        self.ws = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=self.device)
        self.ctx = C.c_void_p()
        self._check(self.L.part_init(C.byref(self.ctx), C.byref(grid), prec, shape, mode,
                                     capacity, nbins, C.c_void_p(self.ws.data_ptr()),
                                     self.ws_bytes, C.c_void_p(self.stream.cuda_stream)), None)
        self._keep = ()
        b = (C.c_int * 3)()
        nk = C.c_int64()
        self._check(self.L.part_brick_dims(C.byref(grid), b, C.byref(nk)))
        self.brick = tuple(b)
        self.nkeys = nk.value

    def _check(self, code: int, ctx="self"):
        if code != 0:
            c = self.ctx if ctx == "self" else None
            msg = self.L.part_last_error(c)
            raise PartError(code, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            self.L.part_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ calls
    def set_fields(self, fields):
        """Device tensor, or pinned host tensor (read once over the host link)."""
        if not ((fields.is_cuda or fields.is_pinned()) and fields.is_contiguous()):
            raise ValueError("fields must be a contiguous device or pinned host tensor")
        prec = FP64 if fields.dtype == self.torch.float64 else MIXED
        self._check(self.L.part_set_fields(self.ctx, _ptr(fields), fields.shape[0], prec))
        self._fields = fields

    def bind(self, n, x, off=None, u=None, w=None, ids=None, chi=None, eng=None, n_old=None):
        self._check(self.L.part_bind_particles(self.ctx, n, _ptr(x), _ptr(off), _ptr(u),
                                               _ptr(w), _ptr(ids), _ptr(chi), _ptr(eng),
                                               _ptr(n_old)))
        self._keep = (x, off, u, w, ids, chi, eng, n_old)

    def sort(self):
        self._check(self.L.part_sort(self.ctx))

    def cell_start(self):
        """View of cell_start[nkeys + 1] inside the workspace (int64 copy)."""
        p = C.c_void_p()
        nk = C.c_int64()
        self._check(self.L.part_cell_start(self.ctx, C.byref(p), C.byref(nk)))
        off = p.value - self.ws.data_ptr()
        raw = self.ws[off: off + 4 * (nk.value + 1)]
        return raw.view(self.torch.int32).to(self.torch.int64) & 0xFFFFFFFF

    def compact(self, deleted) -> int:
        """Sec. 3.2 compaction by a device uint8 mask; returns the new count (the
        bound arrays now have row stride n_new)."""
        nn = C.c_int64()
        self._check(self.L.part_compact(self.ctx, _ptr(deleted), C.byref(nn)))
        return nn.value

    def inject(self, k, x, off=None, u=None, w=None, ids=None, chi=None, eng=None,
               n_old=None):
        """Append k particles (device arrays, bound layout, row stride k); the
        bound arrays must hold rows x (n + k) elements."""
        self._check(self.L.part_inject(self.ctx, int(k), _ptr(x), _ptr(off), _ptr(u), _ptr(w),
                                       _ptr(ids), _ptr(chi), _ptr(eng), _ptr(n_old)))
        self._keep_inj = (x, off, u, w, ids, chi, eng, n_old)

    def set_outflow(self, mask):
        """Device uint8[n] written by every push: 1 where the particle left the
        domain through an open face (None: not written)."""
        self._check(self.L.part_set_outflow(self.ctx, _ptr(mask)))
        self._keep_out = mask

    def flush(self):
        """Current particle state into the bound arrays (asynchronous)."""
        self._check(self.L.part_flush(self.ctx))

    def set_lp_order(self, order: int):
        """LP time marching: 2 (Heun) or 3 (SSP-RK3)."""
        self._check(self.L.part_set_lp_order(self.ctx, order))

    def set_lp_arith(self, paired: bool):
        """LP push arithmetic: FP64 (False, the default) or paired f32 (True)."""
        self._check(self.L.part_set_lp_arith(self.ctx, 1 if paired else 0))

    def set_spec_lazy(self, lazy: bool):
        """spec_update composes per-LP maps (True) or updates every bin (False,
        the default); the bins are brought up to date at sync/flush."""
        self._check(self.L.part_set_spec_lazy(self.ctx, 1 if lazy else 0))

    def enable_shocks(self, r_min: float, state):
        """Diffusive shock acceleration of the LP spectra (Eq. convolution_spectra);
        state: device uint8[n] per-LP flags (None disables)."""
        self._check(self.L.part_enable_shocks(self.ctx, r_min, _ptr(state)))
        self._keep_shock = state

    def shock_cells(self):
        """View of the per-cell compression ratios r[G] (0: no shock)."""
        p = C.c_void_p()
        nc = C.c_int64()
        self._check(self.L.part_shock_cells(self.ctx, C.byref(p), C.byref(nc)))
        off = p.value - self.ws.data_ptr()
        return self.ws[off: off + 8 * nc.value].view(self.torch.float64)

    def set_shock_slope(self, relativistic: bool):
        """Eq. slope with (True) or without (False, the default) q_R."""
        self._check(self.L.part_set_shock_slope(self.ctx, 1 if relativistic else 0))

    def shock_slopes(self):
        """View of the per-cell index q[G] of Eq. slope (0: no shock)."""
        p = C.c_void_p()
        nc = C.c_int64()
        self._check(self.L.part_shock_slopes(self.ctx, C.byref(p), C.byref(nc)))
        off = p.value - self.ws.data_ptr()
        return self.ws[off: off + 8 * nc.value].view(self.torch.float64)

    def enable_deposit(self, on=True):
        self._check(self.L.part_enable_deposit(self.ctx, 1 if on else 0))

    def gather_push(self, qm: float, dt: float, nsteps: int = 1):
        self._check(self.L.part_gather_push(self.ctx, qm, dt, nsteps))

    def deposit(self, out):
        """Device tensor, or pinned host tensor (written over the host link)."""
        if not ((out.is_cuda or out.is_pinned()) and out.dtype == self.torch.float64
                and out.is_contiguous()):
            raise ValueError("out must be a contiguous float64 device or pinned host tensor")
        self._check(self.L.part_deposit(self.ctx, _ptr(out)))

    def spec_update(self, dt: float, c0: float, u_rad: float = 0.0):
        self._check(self.L.spec_update(self.ctx, dt, c0, u_rad))

    def init_particles(self, seed: int, u_th: float = 0.0, eps_min: float = 1.0,
                       eps_max: float = 1e6, p_index: float = 2.2, N0: float = 1e-6):
        self._check(self.L.part_init_particles(self.ctx, seed, u_th, eps_min, eps_max,
                                               p_index, N0))

    def sync(self):
        self._check(self.L.part_sync(self.ctx))

    def exchange_bytes(self, k: int) -> int:
        """Bytes of a packed exchange buffer for k particles (part_exchange_bytes)."""
        b = C.c_size_t()
        self._check(self.L.part_exchange_bytes(self.ctx, int(k), C.byref(b)))
        return b.value

    def exchange_pack(self, axis: int, lo: int, hi: int, to_left, to_right, send_left,
                      send_right, leaving):
        """part_exchange_pack; to_left / to_right are (dx, dj, n_axis).  Returns
        (count_left, count_right, packed): packed is False when a buffer was too
        small (nothing packed; resize to exchange_bytes(count) and call again)."""
        cnt = (C.c_int64 * 2)()
        sl, sr = XShift(*to_left), XShift(*to_right)
        nl = send_left.numel() if send_left is not None else 0
        nr = send_right.numel() if send_right is not None else 0
        code = self.L.part_exchange_pack(self.ctx, int(axis), int(lo), int(hi), C.byref(sl),
                                         C.byref(sr), _ptr(send_left), nl, _ptr(send_right), nr,
                                         _ptr(leaving), cnt)
        if code == 2:   # PART_ENOMEM: counts set, buffers too small
            return int(cnt[0]), int(cnt[1]), False
        self._check(code)
        return int(cnt[0]), int(cnt[1]), True

    def exchange_unpack(self, k: int, recv):
        """part_exchange_unpack: append k particles from a packed buffer."""
        self._check(self.L.part_exchange_unpack(self.ctx, int(k), _ptr(recv),
                                                recv.numel() if recv is not None else 0))

    def launches(self) -> int:
        return int(self.L.part_launch_count(self.ctx))

    def selftest_wait(self, limit_ns: int, arrive: bool):
        """One bounded mbarrier wait on the device (see part_selftest_wait)."""
        self._check(self.L.part_selftest_wait(self.ctx, int(limit_ns), 1 if arrive else 0))


def probe_fp64_fma(stream_ptr: int, sink, ctas_per_sm: int = 4, iters: int = 8192,
                   reps: int = 5) -> tuple[float, float]:
    """Measured FP64 FMA rate of the current device (part_probe_fp64_fma):
    (TFLOP/s, best launch ms).  sink: a device tensor of at least one
    float64; stream_ptr: a cudaStream_t as an integer (0 = default)."""
    L = lib()
    tf, ms = C.c_double(0.0), C.c_double(0.0)
    code = L.part_probe_fp64_fma(C.c_void_p(stream_ptr or None), C.c_void_p(sink.data_ptr()),
                                 int(ctas_per_sm), int(iters), int(reps), C.byref(tf),
                                 C.byref(ms))
    if code != 0:
        raise PartError(code, L.part_last_error(None).decode())
    return tf.value, ms.value


def _raise(code: int):
    if code != 0:
        msg = lib().part_last_error(None)
        raise PartError(code, msg.decode() if msg else "")


def _i3(v):
    return (C.c_int * 3)(*[int(a) for a in v])


def box_pack(src, ncomp: int, dims, lo, ext, dst, stream_ptr: int = 0):
    """part_box_pack: dst (packed [ncomp][ext z][ext y][ext x]) <- the box of
    src ([ncomp][dims z][dims y][dims x]); device float64 tensors."""
    _raise(lib().part_box_pack(_ptr(src), int(ncomp), _i3(dims), _i3(lo), _i3(ext), _ptr(dst),
                               C.c_void_p(stream_ptr or None)))


def box_add(dst, ncomp: int, dims, lo, ext, src, stream_ptr: int = 0):
    """part_box_add: the box of dst += src (packed)."""
    _raise(lib().part_box_add(_ptr(dst), int(ncomp), _i3(dims), _i3(lo), _i3(ext), _ptr(src),
                              C.c_void_p(stream_ptr or None)))


def sum_ordered(out, parts, stream_ptr: int = 0):
    """part_sum_ordered: out[i] = parts[0][i] + parts[1][i] + ... in row order;
    parts a contiguous device float64 tensor [nparts][count]."""
    _raise(lib().part_sum_ordered(_ptr(out), _ptr(parts), int(parts.shape[1]),
                                  int(parts.shape[0]), C.c_void_p(stream_ptr or None)))
