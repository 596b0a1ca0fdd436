"""The LP step in paired-f32 arithmetic (part_set_lp_arith(1)) against the FP64
oracle, through the C ABI.

The paired step carries every value as two floats (~48 bits): positions come
out within ~1e-15 of the FP64 step and the samples within ~1e-13 relative, so
the bars of the FP64 kernel hold unchanged: positions 1e-12 per step (2e-12
for RK3), spectra 1e-12 relative per step, shock flags and outflow masks
bit-exact.  Covered: RK2 and RK3, TSC and CIC, 2D and 3D, the cached v, B
across steps, flushes and injection in between, shocks (non-relativistic and
relativistic slopes), an open axis with compaction, switching the arithmetic
in the middle of a run, and the argument checks.
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
    """Largest relative difference; bins that are zero in the oracle (the
    lowest bin after a shock) must be zero on the GPU too."""
    return np.max(np.abs(gpu - ref) / np.maximum(np.abs(ref), 1e-300)) if gpu.size else 0.0


class Run:
    """A paired-arithmetic LP context and the oracle's copy of its state."""

    def __init__(self, dim, n, f7, x, nb, shape=P.TSC, order=2, seed_spec=(1.0, 1e6, 2.2),
                 open_axes=(0, 0, 0), capacity=None):
        self.og = O.make_grid(dim, (n, n, n), open_axes=open_axes)
        self.f7, self.shape, self.order, self.nb = f7, shape, order, nb
        N = x.shape[1]
        cap = capacity or N
        self.p = P.Part(P.make_grid(dim, n, open_axes=open_axes), P.FP64, shape, P.LP_RK2,
                        capacity=cap, nbins=nb)
        self.p.set_fields(_dev(f7))
        self.p.set_lp_order(order)
        self.p.set_lp_arith(True)
        e1, c1 = O.init_spectrum(nb, *seed_spec, 1e-6)
        self.x = x.copy()
        self.eng = np.repeat(e1[:, None], N, 1)
        self.chi = np.repeat(c1[:, None], N, 1)
        self.nold = np.array([O.gather(self.og, shape, f7[3:4], x[:, i])[0] for i in range(N)])

        def packed(a, rows):  # rows of the bound count, packed, in a capacity-sized buffer
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

    def step(self, dt, c0, u_rad=0.0):
        self.p.gather_push(0.0, dt, 1)
        self.p.spec_update(dt, c0, u_rad)
        f = O.lp_rk2_step if self.order == 2 else O.lp_rk3_step
        self.x, nn, b2, gm = f(self.og, self.shape, self.f7[:3], self.f7[3:4], self.f7[4:],
                               self.x, dt)
        self.chi, self.eng, self.nold = O.spec_update(self.chi, self.eng, self.nold, nn, b2, gm,
                                                      dt, c0, u_rad)

    def compare(self, xtol, stol):
        self.p.sync()
        xg, cg, eg, ng = self.plain()
        assert np.max(np.abs(_pdiff(xg, self.x))) <= xtol
        assert _rel(eg, self.eng) <= stol
        assert _rel(cg, self.chi) <= stol
        assert _rel(ng, self.nold) <= stol


def _fluid(dim, n, seed, v_rms=0.05):
    vel, rho, B = synth.fluid_snapshot(dim, n, seed, v_rms=v_rms)
    return np.concatenate([vel, rho, B]).reshape(7, -1)


def _uniform_lps(dim, N, seed):
    rng = np.random.default_rng(seed)
    x = np.zeros((3, N))
    x[:dim] = rng.uniform(-1.0, 1.0, (dim, N))
    return x


@pytest.mark.parametrize("dim,n,shape,order", [(3, 20, P.TSC, 2), (2, 40, P.TSC, 2),
                                               (3, 12, P.CIC, 2), (3, 20, P.TSC, 3),
                                               (2, 24, P.CIC, 3)])
def test_paired_steps_match_oracle(dim, n, shape, order):
    """Five steps (the first gathers v, B at x, the others take them from the
    cache): every LP against the oracle after each step."""
    N = n ** dim * 2 + 5
    run = Run(dim, n, _fluid(dim, n, 41), _uniform_lps(dim, N, 3), 64, shape, order)
    dt = 0.5 * 2.0 / n
    for k in range(5):
        run.step(dt, 2e-3, 0.1)
        run.compare(2e-12 * (k + 1), 1e-12 * (k + 1))


def test_paired_agrees_with_fp64_kernel_to_its_own_precision():
    """The paired and the FP64 GPU steps from the same state: positions within
    1e-14 (a few 2^-48 of the coordinates), samples-driven spectra within
    1e-12."""
    dim, n, nb = 3, 24, 32
    f7 = _fluid(dim, n, 47)
    N = n ** 3
    x = _uniform_lps(dim, N, 8)
    out = []
    for paired in (False, True):
        p = P.Part(P.make_grid(dim, n), P.FP64, P.TSC, P.LP_RK2, capacity=N, nbins=nb)
        p.set_fields(_dev(f7))
        p.set_lp_arith(paired)
        xd = _dev(x)
        chi = torch.ones((nb, N), dtype=torch.float64, device="cuda")
        eng = torch.ones((nb, N), dtype=torch.float64, device="cuda") * 10.0
        nold = _dev(np.array([O.gather(O.make_grid(dim, (n, n, n)), P.TSC, f7[3:4], x[:, i])[0]
                              for i in range(N)]))
        p.bind(N, xd, chi=chi, eng=eng, n_old=nold)
        for _ in range(3):
            p.gather_push(0.0, 0.5 * 2.0 / n, 1)
            p.spec_update(0.5 * 2.0 / n, 2e-3, 0.1)
        p.sync()
        out.append((_host(xd), _host(chi), _host(eng)))
    assert np.max(np.abs(_pdiff(out[0][0], out[1][0]))) <= 1e-14
    assert _rel(out[1][1], out[0][1]) <= 1e-12
    assert _rel(out[1][2], out[0][2]) <= 1e-12


def test_paired_across_flush_injection_and_switching():
    """Steps with a flush, an injection and two changes of arithmetic in
    between (each change drops the cached v, B; spec_update reads the samples
    in the format the last push left): chi, eps, n_old and positions against
    the oracle."""
    dim, n, nb = 3, 16, 32
    f7 = _fluid(dim, n, 43)
    N0, K = 3000, 200
    x0 = _uniform_lps(dim, N0 + K, 5)
    run = Run(dim, n, f7, x0[:, :N0], nb, capacity=N0 + K)
    dt, c0 = 0.5 * 2.0 / n, 3e-3

    def steps(k):
        for _ in range(k):
            run.step(dt, c0, 0.05)

    steps(2)
    run.p.set_lp_arith(False)
    steps(1)
    run.p.set_lp_arith(True)
    steps(1)
    run.p.flush()
    steps(2)
    rng = np.random.default_rng(9)
    xn = x0[:, N0:]
    e1, c1 = O.init_spectrum(nb, 1.0, 1e6, 2.2, 1e-6)
    cn = np.repeat(c1[:, None], K, 1) * rng.uniform(0.5, 2.0, (1, K))
    en_ = np.repeat(e1[:, None], K, 1)
    nn0 = np.array([O.gather(run.og, P.TSC, f7[3:4], xn[:, i])[0] for i in range(K)])
    run.p.inject(K, x=_dev(xn), chi=_dev(cn), eng=_dev(en_), n_old=_dev(nn0))
    run.x = np.concatenate([run.x, xn], 1)
    run.chi, run.eng = np.concatenate([run.chi, cn], 1), np.concatenate([run.eng, en_], 1)
    run.nold = np.concatenate([run.nold, nn0])
    steps(3)
    run.compare(1e-12 * 2 * 9, 1e-11)


def _rh(n, r=40.0 / 11.0, rho_u=50.0, v_u=0.1):
    xc = -1.0 + (np.arange(n) + 0.5) * (2.0 / n)
    down = np.broadcast_to(xc[None, :] > 0.0, (n, n)).reshape(-1)
    f7 = np.zeros((7, n * n))
    f7[0] = np.where(down, v_u / r, v_u)
    f7[3] = np.where(down, r * rho_u, rho_u)
    f7[4] = 1.0
    return f7


@pytest.mark.parametrize("rel", [False, True])
def test_paired_shock_steps_match_oracle(rel):
    """LPs crossing the Rankine-Hugoniot shock in paired arithmetic, with the
    non-relativistic and the relativistic slope: flags bit-exact, spectra
    1e-12 per step."""
    n, N, nb = 40, 3001, 64
    f7 = _rh(n)
    rng = np.random.default_rng(4)
    x = np.zeros((3, N))
    x[0] = rng.uniform(-0.12, 0.02, N)
    x[1] = rng.uniform(-1.0, 1.0, N)
    run = Run(2, n, f7, x, nb, seed_spec=(1e2, 1e4, 9.0))
    st = torch.zeros(N, dtype=torch.uint8, device="cuda")
    if rel:
        run.p.set_shock_slope(True)
    run.p.enable_shocks(1.5, st)
    rc = O.shock_cells(run.og, f7[:3], f7[3:4], 1.5)
    qc = O.shock_slopes(run.og, f7[:3], f7[3:4], rc, rel) if rel else None
    sto = np.zeros(N, np.uint8)
    dt = 0.5 * (2.0 / n) / 0.1
    for k in range(3):
        run.step(dt, 1e-6)
        run.chi, sto = O.lp_shock(run.og, rc, run.x, run.chi, run.eng, sto, q_cell=qc)
        run.compare(2e-12 * (k + 1), 1e-12 * (k + 1))
        assert np.array_equal(_host(st), sto)
    assert int(sto.sum()) > 100            # LPs did cross into the shock


def test_paired_open_axis_with_compaction():
    """An open x axis: LPs drift out through x = +1 in paired arithmetic; the
    outflow mask is bit-exact with the oracle's outside test every step, and
    the compacted survivors match."""
    n, N, nb, r = 64, 2000, 16, 40.0 / 11.0
    f7 = _rh(n)
    rng = np.random.default_rng(9)
    x = np.zeros((3, N))
    x[0] = rng.uniform(0.3, 0.99, N)
    x[1] = rng.uniform(-1.0, 1.0, N)
    run = Run(2, n, f7, x, nb, seed_spec=(1e2, 1e4, 9.0), open_axes=(1, 0, 0))
    out = torch.zeros(N, dtype=torch.uint8, device="cuda")
    run.p.set_outflow(out)
    dt = 2.0 * (2.0 / n) / (0.1 / r)
    for _ in range(6):
        run.step(dt, 1e-6)
        run.p.sync()
        m = O.outside(run.og, run.x)
        assert np.array_equal(_host(out)[: run.x.shape[1]], m)
        k = run.p.compact(out)
        kk, src = O.compact_map(m)
        assert k == kk
        run.x, run.chi, run.eng, run.nold = (run.x[:, src], run.chi[:, src], run.eng[:, src],
                                             run.nold[src])
    run.p.sync()
    k = run.x.shape[1]
    assert 0 < k < N
    xg, cg, _, _ = run.plain()
    assert np.max(np.abs(xg - run.x)) <= 1e-12
    assert np.max(np.abs(cg - run.chi) / np.abs(run.chi)) <= 1e-11


def test_lp_arith_errors():
    pg = P.make_grid(3, 8)
    pb = P.Part(pg, P.FP64, P.TSC, P.BORIS, capacity=4)
    with pytest.raises(P.PartError):
        pb.set_lp_arith(True)                     # Boris mode
    p = P.Part(pg, P.FP64, P.TSC, P.LP_RK2, capacity=4, nbins=2)
    for bad in (-1, 2):
        with pytest.raises(P.PartError):
            p._check(p.L.part_set_lp_arith(p.ctx, bad))
    p.set_lp_arith(True)
    p.set_lp_arith(False)
