"""Third-order LP time marching (SSP-RK3) on the GPU against the oracle and
against closed forms, through the C ABI: one step within 1e-12 (as RK2),
the time order of both schemes on a solid rotation (a circle after one
period), and the paper's simple-advection test (Sec. 4.1.1) run on the GPU.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2602_23434_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2602_23434_b300 import _lib as P  # noqa: E402


def _host(t):
    return t.detach().cpu().numpy()


class LP:
    def __init__(self, dim, n, f7, x, nb=1, shape=P.TSC, order=3):
        N = x.shape[1]
        self.p = P.Part(P.make_grid(dim, n), P.FP64, shape, P.LP_RK2, capacity=N, nbins=nb)
        self.p.set_fields(torch.as_tensor(np.ascontiguousarray(f7)).cuda())
        self.p.set_lp_order(order)
        self.x = torch.as_tensor(np.ascontiguousarray(x)).cuda()
        self.chi = torch.ones((nb, N), dtype=torch.float64, device="cuda")
        self.eng = torch.ones((nb, N), dtype=torch.float64, device="cuda")
        self.nold = torch.ones(N, dtype=torch.float64, device="cuda")
        self.p.bind(N, self.x, chi=self.chi, eng=self.eng, n_old=self.nold)


@pytest.mark.parametrize("dim,n,shape", [(3, 20, P.TSC), (2, 40, P.TSC), (3, 12, P.CIC)])
def test_rk3_step_matches_oracle(dim, n, shape):
    og = O.make_grid(dim, (n, n, n))
    vel, rho, B = synth.fluid_snapshot(dim, n, 43, v_rms=0.05)
    f7 = np.concatenate([vel, rho, B]).reshape(7, -1)
    N = n ** dim * 2 + 3
    rng = np.random.default_rng(6)
    x = np.zeros((3, N))
    x[:dim] = rng.uniform(-1.0, 1.0, (dim, N))
    e1, c1 = O.init_spectrum(64, 1.0, 1e6, 2.2, 1e-6)
    lp = LP(dim, n, f7, x, nb=64, shape=shape)
    lp.eng.copy_(torch.as_tensor(np.repeat(e1[:, None], N, 1)))
    lp.chi.copy_(torch.as_tensor(np.repeat(c1[:, None], N, 1)))
    no = np.array([O.gather(og, shape, rho.reshape(1, -1), x[:, i])[0] for i in range(N)])
    lp.nold.copy_(torch.as_tensor(no))
    dt, c0 = 0.5 * 2.0 / n, 2e-3
    lp.p.gather_push(0.0, dt, 1)
    lp.p.spec_update(dt, c0, 0.1)
    lp.p.sync()
    xr, nn, b2, gm = O.lp_rk3_step(og, shape, vel.reshape(3, -1), rho.reshape(1, -1),
                                   B.reshape(3, -1), x, dt)
    d = _host(lp.x) - xr
    assert np.max(np.abs(d - 2.0 * np.round(d / 2.0))) <= 2e-12
    ch, en, nor = O.spec_update(np.repeat(c1[:, None], N, 1), np.repeat(e1[:, None], N, 1),
                                no, nn, b2, gm, dt, c0, 0.1)
    assert np.max(np.abs(_host(lp.chi) - ch) / np.abs(ch)) <= 1e-12
    assert np.max(np.abs(_host(lp.eng) - en) / np.abs(en)) <= 1e-12
    assert np.max(np.abs(_host(lp.nold) - nor) / np.abs(nor)) <= 1e-12


def _rotation_fields(n):
    xc = -1 + (np.arange(n) + 0.5) * 2 / n
    X, Y = np.meshgrid(xc, xc)
    f7 = np.zeros((7, n * n))
    f7[0], f7[1], f7[3] = -Y.reshape(-1), X.reshape(-1), 1.0
    return f7


def test_time_order_on_solid_rotation_gpu():
    """v = (-y, x) (interpolated exactly by TSC away from the seam); one LP
    per dt at radius 0.5 for one period: error ratios 4 (Heun) and 8 (RK3)."""
    n = 64
    f7 = _rotation_fields(n)
    for order in (2, 3):
        errs = []
        for ns in (50, 100, 200, 400):
            lp = LP(2, n, f7, np.array([[0.5], [0.0], [0.0]]), order=order)
            for _ in range(ns):
                lp.p.gather_push(0.0, 2 * math.pi / ns, 1)
            lp.p.sync()
            x = _host(lp.x)
            errs.append(math.hypot(x[0, 0] - 0.5, x[1, 0]))
        for a, b in zip(errs, errs[1:]):
            assert abs(math.log2(a / b) - order) < 0.02, (order, errs)


def _e1_exact(t):
    s3 = math.sqrt(3)
    v = 2 / math.pi * math.atan(0.5 * (s3 * math.tan(math.pi * (s3 + 9 * t) / (6 * s3)) - 1))
    return (v + 1) % 2 - 1


def test_simple_advection_on_the_gpu():
    """Sec. 4.1.1 on the GPU with both schemes: the LP position at t = 10
    agrees with the oracle's to 1e-11 and converges as n^-2 (TSC-limited).
    The LP push also samples gamma_g = (1 - v^2)^-1/2 (c = 1), so the test's
    speeds 2 + sin(pi x') are run at a tenth, over ten times the time, with
    ten times the step: the same path and the same steps."""
    for order, step in ((2, O.lp_rk2_step), (3, O.lp_rk3_step)):
        errs = []
        for n in (32, 64, 128):
            yc = -1 + (np.arange(n) + 0.5) * 2 / n
            f7 = np.zeros((7, n, n))
            f7[1] = np.repeat((0.1 * (2 + np.sin(np.pi * yc)))[:, None], n, axis=1)
            f7[3] = 1.0
            f7 = f7.reshape(7, -1)
            nsteps = int(round(10.0 / (0.3 * (2 / n) / 3)))
            dt = 100.0 / nsteps
            lp = LP(2, n, f7, np.zeros((3, 1)), order=order)
            for _ in range(nsteps):
                lp.p.gather_push(0.0, dt, 1)
            lp.p.sync()
            y = _host(lp.x)[1, 0]
            g = O.make_grid(2, (n, n))
            x = np.zeros((3, 1))
            for _ in range(nsteps):
                x, _, _, _ = step(g, O.TSC, f7[:3], f7[3:4], f7[4:], x, dt)
            assert abs(y - x[1, 0]) <= 1e-11
            errs.append(abs((y - _e1_exact(10.0) + 1) % 2 - 1))
        for a, b in zip(errs, errs[1:]):
            assert 1.9 < math.log2(a / b) < 2.1, (order, errs)


def test_lp_order_errors():
    pg = P.make_grid(2, 16)
    pb = P.Part(pg, P.FP64, P.TSC, P.BORIS, capacity=4)
    with pytest.raises(P.PartError):
        pb.set_lp_order(3)
    p = P.Part(pg, P.FP64, P.TSC, P.LP_RK2, capacity=4, nbins=2)
    for bad in (1, 4, 0):
        with pytest.raises(P.PartError):
            p.set_lp_order(bad)
    p.set_lp_order(3)
    p.set_lp_order(2)


def test_rk3_with_shocks_matches_oracle():
    """SSP-RK3 advection with the shock update on the stationary shock."""
    n, N, nb = 40, 2001, 64
    r = 40.0 / 11.0
    og = O.make_grid(2, (n, n, n))
    xc = -1.0 + (np.arange(n) + 0.5) * (2.0 / n)
    down = np.broadcast_to(xc[None, :] > 0.0, (n, n)).reshape(-1)
    f7 = np.zeros((7, n * n))
    f7[0] = np.where(down, 0.1 / r, 0.1)
    f7[3] = np.where(down, 50.0 * r, 50.0)
    f7[4] = 1.0
    rng = np.random.default_rng(12)
    x = np.zeros((3, N))
    x[0] = rng.uniform(-0.12, 0.02, N)
    x[1] = rng.uniform(-1.0, 1.0, N)
    lp = LP(2, n, f7, x, nb=nb, order=3)
    e1, c1 = O.init_spectrum(nb, 1e2, 1e4, 9.0, 1e-6)
    eng, chi = np.repeat(e1[:, None], N, 1), np.repeat(c1[:, None], N, 1)
    no = np.array([O.gather(og, P.TSC, f7[3:4], x[:, i])[0] for i in range(N)])
    lp.eng.copy_(torch.as_tensor(eng))
    lp.chi.copy_(torch.as_tensor(chi))
    lp.nold.copy_(torch.as_tensor(no))
    st = torch.zeros(N, dtype=torch.uint8, device="cuda")
    lp.p.enable_shocks(1.5, st)
    rc = O.shock_cells(og, f7[:3], f7[3:4], 1.5)
    sr = np.zeros(N, np.uint8)
    dt = 0.5 * (2.0 / n) / 0.1
    for _ in range(2):
        lp.p.gather_push(0.0, dt, 1)
        lp.p.spec_update(dt, 1e-6, 0.0)
        x, nn, b2, gm = O.lp_rk3_step(og, P.TSC, f7[:3], f7[3:4], f7[4:], x, dt)
        chi, eng, no = O.spec_update(chi, eng, no, nn, b2, gm, dt, 1e-6)
        chi, sr = O.lp_shock(og, rc, x, chi, eng, sr)
    lp.p.sync()
    assert int(sr.sum()) > 100
    assert np.array_equal(_host(st), sr)
    assert np.max(np.abs(_host(lp.x) - x)) <= 1e-12
    assert np.max(np.abs(_host(lp.chi) - chi) / np.maximum(np.abs(chi), 1e-300)) <= 1e-12
