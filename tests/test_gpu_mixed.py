"""Mixed form (int32 cell + f32 offset, f32 push and fields, the momentum as
a compensated f32 pair, deposit sums beyond f32) against the FP64 oracle,
through the C ABI.

Tolerances follow from f32 arithmetic (unit roundoff 6e-8): one step agrees
with the FP64 oracle to 1e-6 cell in position and 2e-6 of max|u| in
momentum; the deposit to 1e-5 of the sum of |contributions| per cell (each
contribution is an f32 product); the sort is bit-exact; the deposit is
bitwise reproducible.  Over 1000 steps in uniform fields, for every one of
4096 particles: gyrophase drift <= 1e-5 rad and energy drift
|gamma/gamma_FP64 - 1| <= 1e-6, the stated error budget of the mixed form.
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


def _to_mixed(x, n, dim):
    """Positions [3][N] on [-1, 1)^dim -> (linear cell, f32 offset in cell units)."""
    dx = 2.0 / n
    j = np.zeros((3, x.shape[1]), dtype=np.int64)
    off = np.zeros((3, x.shape[1]), dtype=np.float32)
    for a in range(dim):
        s = (x[a] + 1.0) / dx
        j[a] = np.minimum(np.floor(s), n - 1)
        off[a] = (s - j[a] - 0.5).astype(np.float32)
    nz = n if dim == 3 else 1
    cell = (j[2] * n + j[1]) * n + j[0]
    assert np.all(cell < n * n * nz)
    return cell.astype(np.int32), off


def _from_mixed(cell, off, n, dim):
    """(cell, offset) -> f64 positions (exact conversion of the f32 offset)."""
    c = cell.astype(np.int64)
    j = np.stack([c % n, (c // n) % n, c // (n * n)])
    x = np.zeros((3, c.shape[0]))
    for a in range(3):
        if a < dim:
            x[a] = -1.0 + (j[a] + 0.5 + off[a].astype(np.float64)) * (2.0 / n)
    return x


def _cell_units_diff(xg, xr, n):
    d = (xg - xr) / (2.0 / n)
    return d - n * np.round(d / n)


def _u6(u):
    """Momentum [3][N] -> the mixed form's compensated pair [6][N]: f32 value,
    residual 0 (the oracle starts from the f32 value exactly)."""
    uf = np.ascontiguousarray(u, dtype=np.float32)
    return np.concatenate([uf, np.zeros_like(uf)])


def _u64(u6):
    """Compensated pair [6][N] -> its value in f64 (hi + lo, exact)."""
    return u6[:3].astype(np.float64) + u6[3:].astype(np.float64)


def _state(dim, n, ppc, seed, u_th=0.3):
    N = n ** dim * ppc + 11
    x, u, w, ids = synth.particles(dim, None, N, seed, u_th=u_th)
    cell, off = _to_mixed(x, n, dim)
    uf = _u6(u)
    wf = np.random.default_rng(seed).uniform(0.5, 2.0, N).astype(np.float32)
    return N, cell, off, uf, wf, ids


def _key_table(og, brick, n, dim):
    nz = n if dim == 3 else 1
    tab = np.zeros(n * n * nz, dtype=np.uint32)
    for c in range(tab.size):
        tab[c] = O.cell_key(og, brick, (c % n, (c // n) % n, c // (n * n)))
    return tab


@pytest.mark.parametrize("dim,n,ppc", [(3, 20, 8), (2, 40, 16)])
def test_mixed_sort_bit_exact(dim, n, ppc):
    og = O.make_grid(dim, (n, n, n))
    N, cell, off, uf, wf, ids = _state(dim, n, ppc, 5)
    p = P.Part(P.make_grid(dim, n), P.MIXED, P.TSC, P.BORIS, capacity=N)
    cd = torch.as_tensor(cell).cuda()
    od, ud = torch.as_tensor(off).cuda(), torch.as_tensor(uf).cuda()
    idd = torch.as_tensor(ids.astype(np.int64)).cuda()
    p.bind(N, cd, off=od, u=ud, ids=idd)
    p.sort()
    cs = _host(p.cell_start())
    p.sync()
    keys = _key_table(og, p.brick, n, dim)[cell]
    perm = O.stable_sort(keys)
    assert np.array_equal(_host(idd), ids[perm].astype(np.int64))
    assert np.array_equal(_host(cd), cell[perm])
    assert np.array_equal(_host(od), off[:, perm])
    assert np.array_equal(cs, O.cell_start(p.nkeys, keys[perm]).astype(np.int64))


def _check_step_and_deposit(dim, n, shape, f, cell, off, uf, wf):
    """One sorted mixed step with deposit against the FP64 oracle from the
    identical state, then the same step again from that state: bitwise equal."""
    N = cell.shape[0]
    og = O.make_grid(dim, (n, n, n))
    qm, dt = 1.0, 0.5 * (2.0 / n)
    p = P.Part(P.make_grid(dim, n), P.MIXED, shape, P.BORIS, capacity=N)
    p.set_fields(torch.as_tensor(f.astype(np.float32)).cuda())
    cd = torch.as_tensor(cell).cuda()
    od, ud = torch.as_tensor(off).cuda(), torch.as_tensor(uf).cuda()
    wd = torch.as_tensor(wf).cuda()
    p.bind(N, cd, off=od, u=ud, w=wd)
    p.enable_deposit(True)
    p.sort()
    p.sync()
    c0, o0, u0, w0 = _host(cd), _host(od), _host(ud), _host(wd)
    p.gather_push(qm, dt, 1)
    out = torch.empty((3, f.shape[1]), dtype=torch.float64, device="cuda")
    p.deposit(out)
    p.sync()
    x0 = _from_mixed(c0, o0, n, dim)
    xr, ur, F, xo = O.boris_step(og, shape, f, x0, _u64(u0),
                                 w0.astype(np.float64), qm, dt, True)
    xg = _from_mixed(_host(cd), _host(od), n, dim)
    assert np.max(np.abs(_cell_units_diff(xg, xr, n))) <= 1e-6
    assert np.max(np.abs(_u64(_host(ud)) - ur)) <= 2e-6 * np.max(np.abs(ur))
    assert np.all(np.abs(_host(od)) <= 0.5)
    dref = O.deposit(og, shape, xo, F)
    dabs = O.deposit(og, shape, xo, np.abs(F))
    err = np.max(np.abs(_host(out) - dref) / np.maximum(dabs, 1e-300))
    assert err <= 1e-5, err
    # bitwise reproducible
    cd2, od2, ud2 = (torch.as_tensor(c0).cuda(), torch.as_tensor(o0).cuda(),
                     torch.as_tensor(u0).cuda())
    p.bind(N, cd2, off=od2, u=ud2, w=torch.as_tensor(w0).cuda())
    p.sort()
    p.gather_push(qm, dt, 1)
    out2 = torch.empty_like(out)
    p.deposit(out2)
    p.sync()
    assert torch.equal(out, out2) and torch.equal(cd, cd2) and torch.equal(od, od2)


@pytest.mark.parametrize("dim,n,ppc", [(3, 20, 8), (2, 40, 16)])
@pytest.mark.parametrize("shape", [P.TSC, P.CIC])
def test_mixed_step_and_deposit_vs_fp64(dim, n, ppc, shape):
    f = synth.em_fields(dim, n, 23, v_rms=0.05).reshape(6, -1)
    N, cell, off, uf, wf, ids = _state(dim, n, ppc, 7)
    _check_step_and_deposit(dim, n, shape, f, cell, off, uf, wf)


@pytest.mark.parametrize("case", ["dense", "clustered"])
def test_mixed_deposit_full_and_empty_planes(case):
    """The 3D kernel with deposit takes a brick plane (8 x 8 cells) in chunks
    of up to 640 particles and skips empty planes: planes of about 1536
    particles (24 per cell, three chunks each, partial bricks on a 12^3
    grid), and a clustered set (one cell holding 900 particles, a quarter of
    the particles in one brick corner, the other bricks' planes mostly
    empty), both against the FP64 oracle."""
    dim = 3
    if case == "dense":
        n = 12
        N, cell, off, uf, wf, ids = _state(dim, n, 24, 31)
    else:
        n = 16
        rng = np.random.default_rng(32)
        N = 4000
        x, u, _, _ = synth.particles(dim, None, N, 33, u_th=0.3)
        dx = 2.0 / n
        # 900 particles in cell (5, 6, 7); 1000 in the 2^3 cells at the corner of brick 0
        x[:, :900] = (-1.0 + (np.array([5, 6, 7])[:, None] + rng.random((3, 900))) * dx)
        x[:, 900:1900] = -1.0 + rng.random((3, 1000)) * 2 * dx
        # the rest in the upper half in z only: the lower bricks' upper planes stay empty
        x[2, 1900:] = rng.random(N - 1900) * 0.999
        cell, off = _to_mixed(x, n, dim)
        uf = _u6(u)
        wf = rng.uniform(0.5, 2.0, N).astype(np.float32)
    f = synth.em_fields(dim, n, 29, v_rms=0.05).reshape(6, -1)
    _check_step_and_deposit(dim, n, P.TSC, f, cell, off, uf, wf)


def _angle(u):
    return np.arctan2(u[1], u[0])


@pytest.mark.parametrize("E", [(0.0, 0.0, 0.0), (0.0, 0.01, 0.0)])
def test_mixed_drift_1000_steps(E):
    """Uniform B = z (and crossed E): 1000 fused mixed steps vs 1000 FP64
    oracle steps from the identical initial state."""
    dim, n = 2, 64
    og = O.make_grid(dim, (n, n, n))
    f = synth.uniform_em_fields(dim, n, B=(0.0, 0.0, 1.0), E=E).reshape(6, -1)
    N = 4096
    x, u, _, _ = synth.particles(dim, None, N, 99, u_th=0.1)
    cell, off = _to_mixed(x, n, dim)
    uf = _u6(u)
    qm, dt, steps = 1.0, 0.1, 1000
    p = P.Part(P.make_grid(dim, n), P.MIXED, P.TSC, P.BORIS, capacity=N)
    p.set_fields(torch.as_tensor(f.astype(np.float32)).cuda())
    cd = torch.as_tensor(cell).cuda()
    od, ud = torch.as_tensor(off).cuda(), torch.as_tensor(uf).cuda()
    p.bind(N, cd, off=od, u=ud)
    p.gather_push(qm, dt, steps)
    p.sync()
    xr, ur = _from_mixed(cell, off, n, dim), _u64(uf)
    for _ in range(steps):
        xr, ur, _, _ = O.boris_step(og, P.TSC, f, xr, ur, None, qm, dt)
    ug = _u64(_host(ud))
    # gyrophase = angle of u_perp about the drift momentum gamma_d E x B / B^2
    vd = np.cross(np.array(E), np.array([0.0, 0.0, 1.0]))
    ud_ = vd / np.sqrt(1 - vd @ vd)
    dphi = _angle(ug - ud_[:, None]) - _angle(ur - ud_[:, None])
    dphi = np.abs((dphi + np.pi) % (2 * np.pi) - np.pi)
    rperp = np.linalg.norm((ur - ud_[:, None])[:2], axis=0)
    gam_g = np.sqrt(1 + np.sum(ug * ug, axis=0))
    gam_r = np.sqrt(1 + np.sum(ur * ur, axis=0))
    egy = np.abs(gam_g / gam_r - 1)
    print(f"E={E}: gyrophase drift percentiles 50/99/max {np.percentile(dphi, 50):.2e} "
          f"{np.percentile(dphi, 99):.2e} {dphi.max():.2e} rad (smallest gyration radius "
          f"{rperp.min():.2e}, its drift {dphi[np.argmin(rperp)]:.2e}); max energy drift "
          f"{egy.max():.2e}")
    # The stated budget, for every particle, the tightest gyrations included:
    # the momentum is carried as a compensated pair, so the per-step rounding
    # of the stored f32 value no longer random-walks the phase.
    assert dphi.max() <= 1e-5
    assert egy.max() <= 1e-6


@pytest.mark.parametrize("dim,n,ppc", [(3, 20, 8), (2, 40, 16), (3, 24, 2)])
def test_mixed_resort_after_push_bit_exact(dim, n, ppc):
    """The incremental sort on the mixed form (cells moved by the push)."""
    og = O.make_grid(dim, (n, n, n))
    N, cell, off, uf, wf, ids = _state(dim, n, ppc, 9, u_th=2.0)
    f = synth.em_fields(dim, n, 3, v_rms=0.05).reshape(6, -1)
    p = P.Part(P.make_grid(dim, n), P.MIXED, P.TSC, P.BORIS, capacity=N)
    p.set_fields(torch.as_tensor(f.astype(np.float32)).cuda())
    cd = torch.as_tensor(cell).cuda()
    od, ud = torch.as_tensor(off).cuda(), torch.as_tensor(uf).cuda()
    idd = torch.as_tensor(ids.astype(np.int64)).cuda()
    p.bind(N, cd, off=od, u=ud, ids=idd)
    p.sort()
    tab = _key_table(og, p.brick, n, dim)
    for _ in range(3):
        p.gather_push(1.0, 0.95 * 2.0 / n, 1)
        p.sync()
        cb, ib, ob = _host(cd).copy(), _host(idd).copy(), _host(od).copy()
        p.sort()
        cs = _host(p.cell_start())
        p.sync()
        keys = tab[cb]
        perm = O.stable_sort(keys)
        assert np.array_equal(_host(idd), ib[perm])
        assert np.array_equal(_host(cd), cb[perm])
        assert np.array_equal(_host(od), ob[:, perm])
        assert np.array_equal(cs, O.cell_start(p.nkeys, keys[perm]).astype(np.int64))
