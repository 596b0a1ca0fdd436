"""The deferred form of the LP spectra (part_set_spec_lazy) against the FP64
oracle, through the C ABI, and the hand-back of the spectra at a rebind.

In the deferred form spec_update composes each LP's per-step affine maps
(y = 1/eps <- A y + C, psi = chi eps^2 <- psi / A) and the bins are brought
up to date when the spectra are handed back.  The composition rounds
differently from the steps one by one, so the bars are those of the eager
update: spectra 1e-12 relative per step against the oracle, and close to the
eager GPU run.  Covered: both push arithmetics, RK2 and RK3, hand-back every
step or once at the end, shocks (the shocked LPs' bins brought up to date
first), sort, compaction, injection, switching the form, rebinding.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2602_23434_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2602_23434_b300 import _lib as P  # noqa: E402


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def _host(t):
    return t.detach().cpu().numpy()


def _pdiff(a, b, L=2.0):
    d = a - b
    return d - L * np.round(d / L)


def _rel(gpu, ref):
    return np.max(np.abs(gpu - ref) / np.maximum(np.abs(ref), 1e-300)) if gpu.size else 0.0


def _fluid(dim, n, seed):
    vel, rho, B = synth.fluid_snapshot(dim, n, seed, v_rms=0.05)
    return np.concatenate([vel, rho, B]).reshape(7, -1)


def _rh(n, r=40.0 / 11.0):
    xc = -1.0 + (np.arange(n) + 0.5) * (2.0 / n)
    down = np.broadcast_to(xc[None, :] > 0.0, (n, n)).reshape(-1)
    f7 = np.zeros((7, n * n))
    f7[0] = np.where(down, 0.1 / r, 0.1)
    f7[3] = np.where(down, 50.0 * r, 50.0)
    f7[4] = 1.0
    return f7


class Run:
    """An LP context (rows packed at the bound count inside capacity-sized
    buffers) and the oracle's copy of its state."""

    def __init__(self, dim, n, f7, x, nb, order=2, paired=False, lazy=True, capacity=None,
                 spec=(1.0, 1e6, 2.2)):
        self.og = O.make_grid(dim, (n, n, n))
        self.f7, self.order, self.nb = f7, order, nb
        N = x.shape[1]
        cap = capacity or N
        self.p = P.Part(P.make_grid(dim, n), P.FP64, P.TSC, P.LP_RK2, capacity=cap, nbins=nb)
        self.p.set_fields(_dev(f7))
        self.p.set_lp_order(order)
        self.p.set_lp_arith(paired)
        self.p.set_spec_lazy(lazy)
        e1, c1 = O.init_spectrum(nb, *spec, 1e-6)
        self.x = x.copy()
        self.eng = np.repeat(e1[:, None], N, 1)
        self.chi = np.repeat(c1[:, None], N, 1) * np.linspace(0.5, 2.0, N)[None, :]
        self.nold = np.array([O.gather(self.og, P.TSC, f7[3:4], x[:, i])[0] for i in range(N)])

        def packed(a, rows):
            t = torch.zeros(rows * cap, dtype=torch.float64, device="cuda")
            t[: a.size].copy_(_dev(a.reshape(-1)))
            return t.reshape(rows, cap) if rows > 1 else t
        self.xd, self.chid = packed(self.x, 3), packed(self.chi, nb)
        self.engd, self.noldd = packed(self.eng, nb), packed(self.nold, 1)
        self.p.bind(N, self.xd, chi=self.chid, eng=self.engd, n_old=self.noldd)

    def plain(self):
        N = self.x.shape[1]
        v = lambda t, r: _host(t).reshape(-1)[: r * N].reshape(r, N)  # noqa: E731
        return v(self.xd, 3), v(self.chid, self.nb), v(self.engd, self.nb), _host(self.noldd)[:N]

    def step(self, dt, c0, u_rad=0.05):
        self.p.gather_push(0.0, dt, 1)
        self.p.spec_update(dt, c0, u_rad)
        f = O.lp_rk2_step if self.order == 2 else O.lp_rk3_step
        self.x, nn, b2, gm = f(self.og, P.TSC, self.f7[:3], self.f7[3:4], self.f7[4:], self.x,
                               dt)
        self.chi, self.eng, self.nold = O.spec_update(self.chi, self.eng, self.nold, nn, b2, gm,
                                                      dt, c0, u_rad)

    def compare(self, k):
        self.p.sync()
        xg, cg, eg, ng = self.plain()
        assert np.max(np.abs(_pdiff(xg, self.x))) <= 2e-12 * k
        assert _rel(eg, self.eng) <= 1e-12 * k
        assert _rel(cg, self.chi) <= 1e-12 * k
        assert _rel(ng, self.nold) <= 1e-12 * k


@pytest.mark.parametrize("paired", [False, True])
@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("every_step", [False, True])
def test_lazy_steps_match_oracle(paired, order, every_step):
    """Six steps, the spectra handed back after every step or only at the end
    (one composed map of six steps per LP)."""
    dim, n = 3, 16
    N = n ** 3 + 7
    x = np.random.default_rng(31).uniform(-1.0, 1.0, (3, N))
    run = Run(dim, n, _fluid(dim, n, 41), x, 64, order, paired)
    dt, c0 = 0.5 * 2.0 / n, 3e-3
    for k in range(6):
        run.step(dt, c0)
        if every_step:
            run.compare(k + 1)
    run.compare(6)


def test_lazy_agrees_with_the_eager_update():
    """The same twelve steps in both forms: positions bit-identical (the push
    does not depend on the form), spectra within 1e-13 relative."""
    dim, n, nb = 3, 16, 64
    N = n ** 3
    x = np.random.default_rng(33).uniform(-1.0, 1.0, (3, N))
    out = []
    for lazy in (False, True):
        run = Run(dim, n, _fluid(dim, n, 43), x, nb, lazy=lazy)
        for _ in range(12):
            run.p.gather_push(0.0, 0.5 * 2.0 / n, 1)
            run.p.spec_update(0.5 * 2.0 / n, 3e-3, 0.05)
        run.p.sync()
        out.append(run.plain())
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][3], out[1][3])
    assert _rel(out[1][1], out[0][1]) <= 1e-13
    assert _rel(out[1][2], out[0][2]) <= 1e-13


@pytest.mark.parametrize("rel", [False, True])
def test_lazy_with_shocks(rel):
    """LPs crossing the Rankine-Hugoniot shock in the deferred form: a shocked
    LP's bins are brought up to date before its convolution; flags bit-exact,
    spectra 1e-12 per step, handed back only at the end."""
    n, N, nb = 40, 3001, 64
    f7 = _rh(n)
    rng = np.random.default_rng(4)
    x = np.zeros((3, N))
    x[0] = rng.uniform(-0.12, 0.02, N)
    x[1] = rng.uniform(-1.0, 1.0, N)
    run = Run(2, n, f7, x, nb, spec=(1e2, 1e4, 9.0))
    st = torch.zeros(N, dtype=torch.uint8, device="cuda")
    run.p.set_shock_slope(rel)
    run.p.enable_shocks(1.5, st)
    rc = O.shock_cells(run.og, f7[:3], f7[3:4], 1.5)
    qc = O.shock_slopes(run.og, f7[:3], f7[3:4], rc, rel)
    sto = np.zeros(N, np.uint8)
    dt = 0.5 * (2.0 / n) / 0.1
    for k in range(4):
        run.step(dt, 1e-6, 0.0)
        run.chi, sto = O.lp_shock(run.og, rc, run.x, run.chi, run.eng, sto, q_cell=qc)
    run.compare(4)
    assert np.array_equal(_host(st), sto) and int(sto.sum()) > 100


def test_lazy_through_sort_compaction_injection_and_switching():
    """The deferred form across the calls that hand the spectra back: a sort
    (the oracle follows the same permutation), a compaction, an injection,
    and switching the form off and on between steps."""
    dim, n, nb = 3, 12, 32
    N0, K = 2500, 300
    rng = np.random.default_rng(35)
    x0 = rng.uniform(-1.0, 1.0, (3, N0 + K))
    run = Run(dim, n, _fluid(dim, n, 45), x0[:, :N0], nb, capacity=N0 + K)
    dt, c0 = 0.5 * 2.0 / n, 3e-3
    for _ in range(3):
        run.step(dt, c0)
    run.p.sort()                                  # hands the spectra back, then permutes
    run.p.sync()
    perm = O.stable_sort(O.keys(run.og, run.p.brick, run.x))
    run.x, run.chi, run.eng, run.nold = (run.x[:, perm], run.chi[:, perm], run.eng[:, perm],
                                         run.nold[perm])
    run.compare(3)
    for _ in range(2):
        run.step(dt, c0)
    d = rng.random(run.x.shape[1]) < 0.2
    k = run.p.compact(_dev(d.astype(np.uint8)))
    kk, src = O.compact_map(d)
    assert k == kk
    run.x, run.chi, run.eng, run.nold = run.x[:, src], run.chi[:, src], run.eng[:, src], \
        run.nold[src]
    run.compare(5)
    run.p.set_spec_lazy(False)
    run.step(dt, c0)
    run.p.set_spec_lazy(True)
    run.step(dt, c0)
    xn = x0[:, N0:]
    e1, c1 = O.init_spectrum(nb, 1.0, 1e6, 2.2, 1e-6)
    cn, en = np.repeat(c1[:, None], K, 1), np.repeat(e1[:, None], K, 1)
    nn0 = np.array([O.gather(run.og, P.TSC, run.f7[3:4], xn[:, i])[0] for i in range(K)])
    run.p.inject(K, x=_dev(xn), chi=_dev(cn), eng=_dev(en), n_old=_dev(nn0))
    run.x = np.concatenate([run.x, xn], 1)
    run.chi, run.eng = np.concatenate([run.chi, cn], 1), np.concatenate([run.eng, en], 1)
    run.nold = np.concatenate([run.nold, nn0])
    for _ in range(2):
        run.step(dt, c0)
    run.compare(9)


@pytest.mark.parametrize("lazy", [False, True])
def test_rebind_hands_the_previous_spectra_back(lazy):
    """Binding other arrays leaves the previous ones holding (chi, eps) as of
    the last update, in either form, and the new ones start from theirs."""
    dim, n, nb = 3, 12, 32
    N = 2000
    rng = np.random.default_rng(37)
    f7 = _fluid(dim, n, 47)
    a = Run(dim, n, f7, rng.uniform(-1.0, 1.0, (3, N)), nb, lazy=lazy)
    dt, c0 = 0.5 * 2.0 / n, 3e-3
    for _ in range(2):
        a.step(dt, c0)
    xb = rng.uniform(-1.0, 1.0, (3, N))
    e1, c1 = O.init_spectrum(nb, 1.0, 1e6, 2.2, 1e-6)
    cb, eb = np.repeat(c1[:, None], N, 1), np.repeat(e1[:, None], N, 1)
    nb_ = np.array([O.gather(a.og, P.TSC, f7[3:4], xb[:, i])[0] for i in range(N)])
    xbd, cbd, ebd, nbd = _dev(xb), _dev(cb), _dev(eb), _dev(nb_)
    a.p.bind(N, xbd, chi=cbd, eng=ebd, n_old=nbd)
    a.p.sync()
    xg, cg, eg, ng = a.plain()                    # the first arrays, handed back
    assert np.max(np.abs(_pdiff(xg, a.x))) <= 4e-12
    assert _rel(eg, a.eng) <= 2e-12 and _rel(cg, a.chi) <= 2e-12
    a.p.gather_push(0.0, dt, 1)
    a.p.spec_update(dt, c0, 0.05)
    a.p.sync()
    xr, nn, b2, gm = O.lp_rk2_step(a.og, P.TSC, f7[:3], f7[3:4], f7[4:], xb, dt)
    cr, er, nr = O.spec_update(cb, eb, nb_, nn, b2, gm, dt, c0, 0.05)
    assert _rel(_host(ebd), er) <= 1e-12 and _rel(_host(cbd), cr) <= 1e-12


def test_lazy_errors():
    pg = P.make_grid(3, 8)
    pb = P.Part(pg, P.FP64, P.TSC, P.BORIS, capacity=4)
    with pytest.raises(P.PartError):
        pb.set_spec_lazy(True)                     # Boris mode
    p = P.Part(pg, P.FP64, P.TSC, P.LP_RK2, capacity=4, nbins=2)
    for bad in (-1, 2):
        with pytest.raises(P.PartError):
            p._check(p.L.part_set_spec_lazy(p.ctx, bad))
    p.set_spec_lazy(True)
    p.set_spec_lazy(False)
