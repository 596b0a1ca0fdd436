"""Shock acceleration of LP spectra (Eq. convolution_spectra, Eq. slope) on
the GPU against the oracle, through the C ABI.

Tolerances: shock cells and the per-LP shock flags are bit-exact (one
division and comparisons in FP64 on both sides); spectra 1e-12 relative per
step (the GPU evaluates the same integral as a running sum of separable
terms, the oracle as a direct double loop: both are a few ulp per term of
positive sums), 1e-10 after 100 steps.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2602_23434_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2602_23434_b300 import _lib as P  # noqa: E402

import test_oracle_pins as pins  # noqa: E402  (the boosted relativistic shock state)

R_E2 = 40.0 / 11.0        # Rankine-Hugoniot r of the shock test (M^2 = 30, gamma 5/3)


def _host(t):
    return t.detach().cpu().numpy()


def _rel(gpu, ref, floor=1e-300):
    return np.max(np.abs(gpu - ref) / np.maximum(np.abs(ref), floor)) if gpu.size else 0.0


def _rh_fields(n, r=R_E2, rho_u=50.0, v_u=0.1):
    """Stationary shock at x = 0 on [-1,1]^2: x < 0 upstream, x > 0 downstream
    (r rho_u, v_u / r); B = (1, 0, 0).  Returns vel[3,G], rho[1,G], B[3,G]."""
    xc = -1.0 + (np.arange(n) + 0.5) * (2.0 / n)
    down = np.broadcast_to(xc[None, :] > 0.0, (n, n)).reshape(-1)
    rho = np.where(down, r * rho_u, rho_u)[None]
    vel = np.zeros((3, n * n))
    vel[0] = np.where(down, v_u / r, v_u)
    B = np.zeros((3, n * n))
    B[0] = 1.0
    return vel, rho, B


class LPRun:
    """GPU LP context with shocks plus the oracle's copy of the same state."""

    def __init__(self, dim, n, vel, rho, B, x, nb, r_min, eps=(1e2, 1e4), p=9.0, rel=False):
        self.og = O.make_grid(dim, (n, n, n))
        self.vel, self.rho, self.B = vel, rho, B
        N = x.shape[1]
        self.p = P.Part(P.make_grid(dim, n), P.FP64, P.TSC, P.LP_RK2, capacity=N, nbins=nb)
        self.p.set_fields(torch.as_tensor(np.concatenate([vel, rho, B])).cuda())
        e1, c1 = O.init_spectrum(nb, eps[0], eps[1], p, 1e-6)
        self.eng = np.repeat(e1[:, None], N, axis=1)
        self.chi = np.repeat(c1[:, None], N, axis=1)
        self.nold = np.array([O.gather(self.og, P.TSC, rho, x[:, i])[0] for i in range(N)])
        self.x, self.st = x.copy(), np.zeros(N, np.uint8)
        self.xd = torch.as_tensor(x).cuda()
        self.chid = torch.as_tensor(self.chi).cuda()
        self.engd = torch.as_tensor(self.eng).cuda()
        self.noldd = torch.as_tensor(self.nold).cuda()
        self.std = torch.zeros(N, dtype=torch.uint8, device="cuda")
        self.p.bind(N, self.xd, chi=self.chid, eng=self.engd, n_old=self.noldd)
        if rel:
            self.p.set_shock_slope(True)
        self.p.enable_shocks(r_min, self.std)
        self.r_cell = O.shock_cells(self.og, vel, rho, r_min)
        self.q_cell = O.shock_slopes(self.og, vel, rho, self.r_cell, rel) if rel else None

    def step(self, dt, c0, gpu=True, cpu=True):
        if gpu:
            self.p.gather_push(0.0, dt, 1)
            self.p.spec_update(dt, c0, 0.0)
        if cpu:
            self.x, nn, b2, gm = O.lp_rk2_step(self.og, P.TSC, self.vel, self.rho, self.B,
                                               self.x, dt)
            self.chi, self.eng, self.nold = O.spec_update(self.chi, self.eng, self.nold, nn,
                                                          b2, gm, dt, c0)
            self.chi, self.st = O.lp_shock(self.og, self.r_cell, self.x, self.chi, self.eng,
                                           self.st, q_cell=self.q_cell)

    def compare(self, tol):
        self.p.sync()
        assert np.array_equal(_host(self.std), self.st)
        assert np.max(np.abs(_host(self.xd) - self.x)) <= 1e-12
        assert _rel(_host(self.engd), self.eng) <= tol
        assert _rel(_host(self.chid), self.chi) <= tol
        assert _rel(_host(self.noldd), self.nold) <= tol


def test_shock_cells_bit_exact():
    n = 40
    vel, rho, B = _rh_fields(n)
    run = LPRun(2, n, vel, rho, B, np.zeros((3, 1)), 8, 1.5)
    got = _host(run.p.shock_cells())
    assert np.array_equal(got, run.r_cell)
    assert np.count_nonzero(got) == 2 * n
    # 3D turbulent snapshot (lognormal density): many marginal cells
    n3 = 24
    v3, r3, b3 = synth.fluid_snapshot(3, n3, 51, v_rms=0.05)
    v3, r3, b3 = v3.reshape(3, -1), r3.reshape(1, -1), b3.reshape(3, -1)
    run3 = LPRun(3, n3, v3, r3, b3, np.zeros((3, 1)), 8, 1.2)
    got3 = _host(run3.p.shock_cells())
    assert np.array_equal(got3, run3.r_cell)
    assert 0 < np.count_nonzero(got3) < got3.size


def test_shock_step_matches_oracle_2d():
    """LPs scattered around the shock: one step, some of them enter the
    shock cells; flags, positions and spectra against the oracle."""
    n, N, nb = 40, 3001, 128
    vel, rho, B = _rh_fields(n)
    rng = np.random.default_rng(4)
    x = np.zeros((3, N))
    x[0] = rng.uniform(-0.12, 0.02, N)
    x[1] = rng.uniform(-1.0, 1.0, N)
    run = LPRun(2, n, vel, rho, B, x, nb, 1.5)
    dt = 0.5 * (2.0 / n) / 0.1
    run.step(dt, 1e-6)
    assert 100 < int(run.st.sum()) < N
    run.compare(1e-12)
    run.step(dt, 1e-6)        # a second step: flagged LPs are not convolved again
    run.compare(1e-12)


def test_shock_test_100_lps_through_the_shock():
    """Sec. 4.1.2 on the GPU: 100 LPs from upstream through the shock in 100
    steps, against the oracle step by step, and the post-shock slope
    q - 2 = 2.138 within the paper's 0.5%."""
    n, N, nb = 128, 100, 128
    vel, rho, B = _rh_fields(n)
    rng = np.random.default_rng(3)
    x = np.zeros((3, N))
    x[0] = rng.uniform(-0.6, -0.2, N)
    x[1] = rng.uniform(-1.0, 1.0, N)
    run = LPRun(2, n, vel, rho, B, x, nb, 1.5)
    dt = 0.5 * (2.0 / n) / 0.1
    for _ in range(100):
        run.step(dt, 1e-8)
    run.compare(1e-10)
    q = O.dsa_index(R_E2)
    eng, chi = _host(run.engd), _host(run.chid)
    for i in range(N):
        up = eng[:, i] >= eng[-1, i] / 10.0
        slope = -np.polyfit(np.log(eng[up, i]), np.log(chi[up, i]), 1)[0]
        assert abs(slope - (q - 2.0)) / (q - 2.0) <= 0.005


def test_shock_3d_turbulent_with_sort_and_compaction():
    """3D turbulent snapshot, many LPs: flags and spectra follow the LPs
    through part_sort and part_compact."""
    n, nb = 20, 32
    v3, r3, b3 = synth.fluid_snapshot(3, n, 61, v_rms=0.05)
    v3, r3, b3 = v3.reshape(3, -1), r3.reshape(1, -1), b3.reshape(3, -1)
    N = n ** 3 * 2 + 7
    rng = np.random.default_rng(5)
    x = rng.uniform(-1.0, 1.0, (3, N))
    run = LPRun(3, n, v3, r3, b3, x, nb, 1.2, eps=(1.0, 1e6), p=2.2)
    dt = 0.5 * (2.0 / n) / 0.05
    run.step(dt, 2e-3)
    run.compare(1e-12)
    assert run.st.sum() > 0
    # sort: the GPU permutes its arrays; the oracle follows with the same order
    run.p.sort()
    run.p.sync()
    keys = O.keys(run.og, run.p.brick, run.x)
    perm = O.stable_sort(keys)
    run.x, run.chi, run.eng = run.x[:, perm], run.chi[:, perm], run.eng[:, perm]
    run.nold, run.st = run.nold[perm], run.st[perm]
    run.compare(1e-12)
    for _ in range(3):
        run.step(dt, 2e-3)
    run.compare(1e-11)
    # compaction by a random mask
    d = rng.random(N) < 0.2
    nk = run.p.compact(torch.as_tensor(d.astype(np.uint8)).cuda())
    k, src = O.compact_map(d)
    assert nk == k
    run.p.sync()
    got_st = _host(run.std)[:nk]
    assert np.array_equal(got_st, run.st[src])
    chi_g = _host(run.chid).reshape(-1)[: nb * nk].reshape(nb, nk)
    assert _rel(chi_g, run.chi[:, src]) <= 1e-11


def _rel_fields(n, beta_b, mirror=False):
    """A relativistic shock (shock-frame normal speeds 0.9 and 0.35, with
    tangential motion) seen from a frame where it moves at beta_b, front at
    x = 0 on [-1,1]^2; B = (1, 0, 0).  vel[3,G], rho[1,G], B[3,G]."""
    vel, rho = pins._rel_snapshot(n, beta_b, mirror)
    B = np.zeros((3, n * n))
    B[0] = 1.0
    return vel.reshape(3, -1), rho.reshape(1, -1), B


def test_relativistic_slopes_match_oracle():
    """Eq. slope with q_R per shock cell: the moving relativistic shock in
    both flow directions, 1e-13 relative (a few FP64 roundings of the same
    steps), and a 3D turbulent snapshot with speeds up to about c (valid and
    missing shock frames, weak jumps with q up to ~1e5), 1e-13 q relative.
    Without the correction q = 3r/(r-1) bit-exact, and the setting switches
    both ways on enabled shocks."""
    n = 40
    q_true = O.kw_index(0.9, 0.35)
    for beta_b, mirror in ((0.3, False), (0.3, True), (-0.5, False), (0.0, True)):
        vel, rho, B = _rel_fields(n, beta_b, mirror)
        run = LPRun(2, n, vel, rho, B, np.zeros((3, 1)), 8, 1.5, rel=True)
        assert np.array_equal(_host(run.p.shock_cells()), run.r_cell)
        got = _host(run.p.shock_slopes())
        assert np.array_equal(got > 0, run.r_cell > 0) and np.count_nonzero(got) == 2 * n
        assert _rel(got[got > 0], run.q_cell[got > 0]) <= 1e-13
        assert abs(got[got > 0] / q_true - 1.0).max() <= 1e-12
        run.p.set_shock_slope(False)
        q0 = O.shock_slopes(run.og, vel, rho, run.r_cell, False)
        assert np.array_equal(_host(run.p.shock_slopes()), q0)
        run.p.set_shock_slope(True)
        assert _rel(_host(run.p.shock_slopes()), run.q_cell) <= 1e-13
    n3 = 24
    v3, r3, b3 = synth.fluid_snapshot(3, n3, 52, v_rms=0.45)
    v3, r3, b3 = v3.reshape(3, -1), r3.reshape(1, -1), b3.reshape(3, -1)
    run3 = LPRun(3, n3, v3, r3, b3, np.zeros((3, 1)), 8, 1.2, rel=True)
    assert np.array_equal(_host(run3.p.shock_cells()), run3.r_cell)
    got3 = _host(run3.p.shock_slopes())
    sh = run3.r_cell > 0
    assert np.array_equal(got3 > 0, sh) and sh.sum() > 20
    # q divides by b_u - b_d, so its rounding grows with q: against extended
    # precision the oracle itself is within 2.5e-14 q relative on this snapshot
    qr = run3.q_cell[sh]
    assert np.max(np.abs(got3[sh] - qr) / (qr * np.maximum(1.0, qr))) <= 1e-13
    q0 = 3.0 * run3.r_cell[sh] / (run3.r_cell[sh] - 1.0)
    assert np.count_nonzero(run3.q_cell[sh] != q0) > 0      # the correction applied


def test_relativistic_shock_step_matches_oracle():
    """LPs crossing the moving relativistic shock (speeds ~0.6-0.95 c):
    flags, positions and spectra after each of three steps against the
    oracle with its per-cell q."""
    n, N, nb = 40, 2001, 64
    vel, rho, B = _rel_fields(n, 0.3)
    rng = np.random.default_rng(8)
    x = np.zeros((3, N))
    x[0] = rng.uniform(-0.15, 0.02, N)
    x[1] = rng.uniform(-1.0, 1.0, N)
    run = LPRun(2, n, vel, rho, B, x, nb, 1.5, rel=True)
    dt = 0.5 * (2.0 / n) / 0.95
    for _ in range(3):
        run.step(dt, 1e-6)
        run.compare(1e-12)
    assert 100 < int(run.st.sum()) < N


def test_shock_error_paths():
    pg = P.make_grid(2, 16)
    pb = P.Part(pg, P.FP64, P.TSC, P.BORIS, capacity=8)
    st = torch.zeros(8, dtype=torch.uint8, device="cuda")
    with pytest.raises(P.PartError):
        pb.enable_shocks(1.5, st)                             # Boris mode
    p = P.Part(pg, P.FP64, P.TSC, P.LP_RK2, capacity=8, nbins=4)
    x = torch.zeros((3, 8), dtype=torch.float64, device="cuda")
    chi = torch.ones((4, 8), dtype=torch.float64, device="cuda")
    nold = torch.ones(8, dtype=torch.float64, device="cuda")
    p.bind(8, x, chi=chi, eng=chi.clone(), n_old=nold)
    with pytest.raises(P.PartError):
        p.enable_shocks(1.5, st)                              # no fields yet
    vel, rho, B = _rh_fields(16)
    p.set_fields(torch.as_tensor(np.concatenate([vel, rho, B])).cuda())
    for bad in (1.0, 0.5, float("nan")):
        with pytest.raises(P.PartError):
            p.enable_shocks(bad, st)
    for bad in (-1, 2):
        with pytest.raises(P.PartError):
            p._check(p.L.part_set_shock_slope(p.ctx, bad))
    with pytest.raises(P.PartError):
        pb.set_shock_slope(True)                              # Boris mode
    p.enable_shocks(1.5, st)
    p.enable_shocks(1.5, None)                                # off again
    with pytest.raises(P.PartError):
        p.shock_slopes()
    with pytest.raises(P.PartError):
        p.shock_cells()
