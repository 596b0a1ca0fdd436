"""ctypes front end of the FP64 CPU oracle (``part_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  Nothing here touches the CUDA library,
and the CUDA library never calls this module.

Every function takes and returns numpy float64 / uint32 arrays in the layouts
of ``part_oracle.h``: positions and velocities ``[3][n]``, fields
``[comp][z][y][x]`` cell-centred, spectra bin-major ``[nb][n]``.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "part_oracle.c")
_HDR = os.path.join(_HERE, "part_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

CIC, TSC = 1, 2


def compile_source(src: str, out: str) -> str:
    """gcc -O2, no FP contraction, OpenMP: the one way the oracle is built."""
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call([
        "gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
        "-Wl,-Bsymbolic", "-I", _HERE, "-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` if it is missing or older than its sources."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB) for s in (_SRC, _HDR))
    if force or stale:
        compile_source(_SRC, _LIB)
    return _LIB


class Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3),
                ("xmin", C.c_double * 3), ("dx", C.c_double * 3), ("open", C.c_int * 3)]


def make_grid(dim: int, n, xmin=(-1.0, -1.0, -1.0), dx=None, open_axes=(0, 0, 0)) -> Grid:
    """Grid on [xmin, xmin + n dx); default domain [-1, 1]^dim (Sec. 4.1);
    open_axes[a] = 1 makes axis a open (outflow) instead of periodic."""
    n = list(n) + [1] * (3 - len(n))
    if dim == 2:
        n[2] = 1
    if dx is None:
        # an inactive z axis (dim 2) spans the same [-1, 1) as the others
        dx = [2.0 / n[0], 2.0 / n[1], 2.0 / n[2] if dim == 3 else 2.0]
    g = Grid()
    g.dim = dim
    for a in range(3):
        g.n[a] = int(n[a])
        g.xmin[a] = float(xmin[a])
        g.dx[a] = float(dx[a])
        g.open[a] = int(open_axes[a])
    return g


_lib = None
_D = C.POINTER(C.c_double)
_U32 = C.POINTER(C.c_uint32)
_U64 = C.POINTER(C.c_uint64)
_I = C.POINTER(C.c_int)


def lib():
    global _lib
    if _lib is None:
        _lib = load(build())
    return _lib


@contextlib.contextmanager
def using(path: str):
    """Run the wrappers against another build of part_oracle.c (the tests plant
    single mistakes in copies of it to show that the pins catch them)."""
    global _lib
    saved = _lib
    _lib = load(path)
    try:
        yield
    finally:
        _lib = saved


def load(path: str):
    """Open a build of part_oracle.c and declare its C signatures."""
    L = C.CDLL(path)
    G = C.POINTER(Grid)
    sig = {
        "or_shape": (C.c_double, [C.c_int, C.c_double]),
        "or_cell_coord": (None, [G, _D, _I, _D]),
        "or_wrap": (C.c_double, [G, C.c_int, C.c_double]),
        "or_gather": (None, [G, C.c_int, _D, C.c_int, _D, _D]),
        "or_boris_kick": (None, [_D, _D, _D, C.c_double, C.c_double]),
        "or_boris_step": (None, [G, C.c_int, _D, C.c_int64, _D, _D, _D, C.c_double,
                                 C.c_double, _D, _D]),
        "or_deposit": (None, [G, C.c_int, C.c_int64, _D, _D, _D]),
        "or_deposit_cell": (None, [G, C.c_int, C.c_int64, _D, _D, C.c_int64, _D]),
        "or_cell_key": (C.c_uint32, [G, _I, _I]),
        "or_key_count": (C.c_int64, [G, _I]),
        "or_keys": (None, [G, _I, C.c_int64, _D, _U32]),
        "or_stable_sort": (None, [C.c_int64, _U32, _U32]),
        "or_cell_start": (None, [C.c_int64, C.c_int64, _U32, _U32]),
        "or_lp_rk2_step": (None, [G, C.c_int, _D, _D, _D, C.c_int64, _D, C.c_double,
                                  _D, _D, _D]),
        "or_lp_rk3_step": (None, [G, C.c_int, _D, _D, _D, C.c_int64, _D, C.c_double,
                                  _D, _D, _D]),
        "or_spec_update": (None, [C.c_int, C.c_int64, _D, _D, _D, _D, _D, _D,
                                  C.c_double, C.c_double, C.c_double]),
        "or_init_spectrum": (None, [C.c_int, C.c_double, C.c_double, C.c_double,
                                    C.c_double, _D, _D]),
        "or_philox4x32_10": (None, [_U32, _U32, _U32]),
        "or_init_particles": (None, [G, C.c_int64, C.c_uint64, C.c_double, _D, _D, _D,
                                     _U64]),
        "or_compact_map": (C.c_int64, [C.c_int64, C.POINTER(C.c_uint8),
                                       C.POINTER(C.c_int64)]),
        "or_set_threads": (None, [C.c_int]),
        "or_outside": (C.c_int, [G, _D]),
        "or_max_threads": (C.c_int, []),
        "or_rh_compression": (C.c_double, [C.c_double, C.c_double]),
        "or_dsa_index": (C.c_double, [C.c_double]),
        "or_shock_cells": (None, [G, _D, _D, C.c_double, _D]),
        "or_shock_convolve": (None, [C.c_int, _D, _D, C.c_double, C.c_double, _D]),
        "or_kw_index": (C.c_double, [C.c_double, C.c_double]),
        "or_shock_frame_speeds": (C.c_int, [C.c_double, C.c_double, C.c_double, C.c_double,
                                            C.c_double, C.c_double, _D, _D]),
        "or_shock_slopes": (None, [G, _D, _D, _D, C.c_int, _D]),
        "or_lp_shock": (None, [G, _D, _D, C.c_int, C.c_int64, _D, _D, _D,
                               C.POINTER(C.c_uint8)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def _d(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _u32(a):
    assert a.dtype == np.uint32 and a.flags.c_contiguous
    return a.ctypes.data_as(_U32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def shape_fn(shape: int, xi: float) -> float:
    return lib().or_shape(shape, float(xi))


def cell_coord(g: Grid, x):
    x = _f64(x).reshape(3)
    j = (C.c_int * 3)()
    d = np.zeros(3)
    lib().or_cell_coord(C.byref(g), _d(x), j, _d(d))
    return np.array(list(j)), d


def wrap(g: Grid, axis: int, x: float) -> float:
    return lib().or_wrap(C.byref(g), axis, float(x))


def gather(g: Grid, shape: int, fields, x):
    fields = _f64(fields)
    ncomp = fields.shape[0]
    out = np.zeros(ncomp)
    lib().or_gather(C.byref(g), shape, _d(fields), ncomp, _d(_f64(x).reshape(3)), _d(out))
    return out


def boris_kick(u, E, B, qm: float, dt: float):
    u = _f64(u).copy()
    lib().or_boris_kick(_d(u), _d(_f64(E)), _d(_f64(B)), qm, dt)
    return u


def boris_step(g: Grid, shape: int, fields6, x, u, w, qm: float, dt: float,
               want_force: bool = False):
    """One Boris step in place on copies; returns (x, u, F or None, x_old)."""
    x = _f64(x).copy()
    u = _f64(u).copy()
    n = x.shape[1]
    F = np.zeros((3, n)) if want_force else None
    xo = np.zeros((3, n))
    wp = _d(_f64(w)) if w is not None else None
    lib().or_boris_step(C.byref(g), shape, _d(_f64(fields6)), n, _d(x), _d(u), wp, qm, dt,
                        _d(F) if F is not None else None, _d(xo))
    return x, u, F, xo


def deposit(g: Grid, shape: int, x, F):
    x = _f64(x)
    F = _f64(F)
    G = g.n[0] * g.n[1] * g.n[2]
    out = np.zeros((3, G))
    lib().or_deposit(C.byref(g), shape, x.shape[1], _d(x), _d(F), _d(out))
    return out


def deposit_cell(g: Grid, shape: int, x, F, cell: int):
    x = _f64(x)
    F = _f64(F)
    out = np.zeros(3)
    lib().or_deposit_cell(C.byref(g), shape, x.shape[1], _d(x), _d(F), int(cell), _d(out))
    return out


def _brick(b):
    arr = (C.c_int * 3)(*[int(v) for v in b])
    return arr


def cell_key(g: Grid, brick, j) -> int:
    return int(lib().or_cell_key(C.byref(g), _brick(brick), _brick(j)))


def key_count(g: Grid, brick) -> int:
    return int(lib().or_key_count(C.byref(g), _brick(brick)))


def keys(g: Grid, brick, x):
    x = _f64(x)
    out = np.zeros(x.shape[1], dtype=np.uint32)
    lib().or_keys(C.byref(g), _brick(brick), x.shape[1], _d(x), _u32(out))
    return out


def stable_sort(k):
    k = np.ascontiguousarray(k, dtype=np.uint32)
    perm = np.zeros(k.shape[0], dtype=np.uint32)
    lib().or_stable_sort(k.shape[0], _u32(k), _u32(perm))
    return perm


def cell_start(nkeys: int, sorted_keys):
    sk = np.ascontiguousarray(sorted_keys, dtype=np.uint32)
    cs = np.zeros(nkeys + 1, dtype=np.uint32)
    lib().or_cell_start(nkeys, sk.shape[0], _u32(sk), _u32(cs))
    return cs


def lp_rk2_step(g: Grid, shape: int, vel, rho, bfield, x, dt: float):
    """One Heun step on a copy of x; returns (x, n_new, b2m, gam)."""
    x = _f64(x).copy()
    n = x.shape[1]
    n_new, b2m, gam = np.zeros(n), np.zeros(n), np.zeros(n)
    lib().or_lp_rk2_step(C.byref(g), shape, _d(_f64(vel)), _d(_f64(rho)), _d(_f64(bfield)),
                         n, _d(x), dt, _d(n_new), _d(b2m), _d(gam))
    return x, n_new, b2m, gam


def lp_rk3_step(g: Grid, shape: int, vel, rho, bfield, x, dt: float):
    """One SSP-RK3 step on a copy of x; returns (x, n_new, b2m, gam)."""
    x = _f64(x).copy()
    n = x.shape[1]
    n_new, b2m, gam = np.zeros(n), np.zeros(n), np.zeros(n)
    lib().or_lp_rk3_step(C.byref(g), shape, _d(_f64(vel)), _d(_f64(rho)), _d(_f64(bfield)),
                         n, _d(x), dt, _d(n_new), _d(b2m), _d(gam))
    return x, n_new, b2m, gam


def spec_update(chi, eng, n_old, n_new, b2m, gam, dt: float, c0: float, u_rad: float = 0.0):
    """Spectral update on copies; returns (chi, eng, n_old)."""
    chi = _f64(chi).copy()
    eng = _f64(eng).copy()
    n_old = _f64(n_old).copy()
    nb, n = chi.shape
    lib().or_spec_update(nb, n, _d(chi), _d(eng), _d(n_old), _d(_f64(n_new)), _d(_f64(b2m)),
                         _d(_f64(gam)), dt, c0, u_rad)
    return chi, eng, n_old


def init_spectrum(nb: int, emin: float, emax: float, p: float, N0: float):
    eng, chi = np.zeros(nb), np.zeros(nb)
    lib().or_init_spectrum(nb, emin, emax, p, N0, _d(eng), _d(chi))
    return eng, chi


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_u32(c), _u32(k), _u32(out))
    return out


def init_particles(g: Grid, n: int, seed: int, u_th: float):
    x, u, w = np.zeros((3, n)), np.zeros((3, n)), np.zeros(n)
    ids = np.zeros(n, dtype=np.uint64)
    lib().or_init_particles(C.byref(g), n, seed, u_th, _d(x), _d(u), _d(w),
                            ids.ctypes.data_as(_U64))
    return x, u, w, ids


def compact_map(deleted):
    """Sec. 3.2 compaction: (n_keep, src) with src[j] the old index in slot j."""
    d = np.ascontiguousarray(deleted, dtype=np.uint8)
    src = np.zeros(max(d.shape[0], 1), dtype=np.int64)
    nk = lib().or_compact_map(d.shape[0], d.ctypes.data_as(C.POINTER(C.c_uint8)),
                              src.ctypes.data_as(C.POINTER(C.c_int64)))
    return int(nk), src[:nk]


def rh_compression(gamma: float, mach: float) -> float:
    return lib().or_rh_compression(gamma, mach)


def dsa_index(r: float) -> float:
    return lib().or_dsa_index(r)


def shock_cells(g: Grid, vel, rho, r_min: float):
    """Per-cell compression ratio of detected shocks (0 = none), shape [G]."""
    rho = _f64(rho).reshape(-1)
    out = np.zeros(rho.shape[0])
    lib().or_shock_cells(C.byref(g), _d(_f64(vel).reshape(3, -1)), _d(rho), r_min, _d(out))
    return out


def kw_index(beta_u: float, beta_d: float) -> float:
    """Eq. slope for a relativistic shock from its shock-frame flow speeds."""
    return lib().or_kw_index(beta_u, beta_d)


def shock_frame_speeds(v_u, s2_u, rho_u, v_d, s2_d, rho_d):
    """(beta_u, beta_d) in the shock frame, or None where there is none."""
    bu, bd = C.c_double(), C.c_double()
    ok = lib().or_shock_frame_speeds(v_u, s2_u, rho_u, v_d, s2_d, rho_d,
                                     C.byref(bu), C.byref(bd))
    return (bu.value, bd.value) if ok else None


def shock_slopes(g: Grid, vel, rho, r_cell, relativistic: bool):
    """Per-cell q of Eq. slope for the shock cells r_cell > 0, shape [G]."""
    rho = _f64(rho).reshape(-1)
    out = np.zeros(rho.shape[0])
    lib().or_shock_slopes(C.byref(g), _d(_f64(vel).reshape(3, -1)), _d(rho),
                          _d(_f64(r_cell)), int(bool(relativistic)), _d(out))
    return out


def shock_convolve(eng, chi, q: float, cn: float):
    """Eq. convolution_spectra on one spectrum; returns chi_out."""
    eng, chi = _f64(eng), _f64(chi)
    out = np.zeros(chi.shape[0])
    lib().or_shock_convolve(chi.shape[0], _d(eng), _d(chi), q, cn, _d(out))
    return out


def lp_shock(g: Grid, r_cell, x, chi, eng, state, q_cell=None):
    """Shock update on copies; returns (chi, state).  q_cell: per-cell index
    of Eq. slope (None: 3r/(r-1))."""
    chi = _f64(chi).copy()
    st = np.ascontiguousarray(state, dtype=np.uint8).copy()
    nb, n = chi.shape
    qc = None if q_cell is None else _f64(q_cell)
    lib().or_lp_shock(C.byref(g), _d(_f64(r_cell)), None if qc is None else _d(qc), nb, n,
                      _d(_f64(x)), _d(chi), _d(_f64(eng)),
                      st.ctypes.data_as(C.POINTER(C.c_uint8)))
    return chi, st


def set_threads(n: int) -> None:
    """OpenMP threads of the oracle's parallel loops (timing only)."""
    lib().or_set_threads(int(n))


def max_threads() -> int:
    return int(lib().or_max_threads())


def outside(g: Grid, x):
    """Per particle: 1 if it lies outside the domain along an open axis."""
    x = _f64(x)
    return np.array([lib().or_outside(C.byref(g), _d(np.ascontiguousarray(x[:, i])))
                     for i in range(x.shape[1])], dtype=np.uint8)
