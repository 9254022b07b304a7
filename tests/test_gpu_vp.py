"""GPU variable projection solve (Eqs. 2-5, linear CG with device-resident
scalars) against the oracle's FP64 CG on the same seeded problem: the extended
perturbation after k iterations (relative L2 <= 1e-4) and the objective history
(recursively updated on the GPU, evaluated directly by the oracle; within
1e-5 of Phi_0)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_2206_02362_gb300 as fw  # noqa: E402

pytestmark = pytest.mark.gpu


class VP:
    """37 x 300 physical (ragged strips), W=10, nt=250, nh=5, 3 shots; dres = f(m_true) - f(m0)."""

    def __init__(self, nh=5, seed=0):
        nz, nx, W, nt = 37, 300, 10, 250
        self.dt, self.dx = 1e-3, 10.0
        rng = np.random.default_rng(synth.SEED0 + 400 + seed)
        z = np.arange(nz)[:, None]
        x = np.arange(nx)[None, :]
        self.v0 = (1800.0 + 20.0 * z + 0.0 * x).astype(np.float32)
        vt = self.v0 + synth.gaussian_blobs(nz, nx, rng, amp=120.0, sigma_pts=5.0, ring=1)
        self.src_iz, self.src_ix = np.array([0, 2, 1]), np.array([10, 150, 290])
        self.rec_iz, self.rec_ix = np.full(150, 1), 2 * np.arange(150)
        self.w = np.stack([synth.ricker(nt, self.dt, 20.0)] * 3).astype(np.float32)
        self.og = oracle.Grid(nz=nz, nx=nx, W=W, nt=nt, dt=self.dt, dx=self.dx, nh=nh)
        self.ogeo = oracle.Geometry(self.src_iz, self.src_ix, self.rec_iz, self.rec_ix)
        f = lambda v: oracle.forward(self.og, v.astype(np.float64), self.ogeo, self.w.astype(np.float64))
        self.dres = (f(vt) - f(self.v0)).astype(np.float32)
        self.pt0 = (0.01 * rng.standard_normal((nh, nz, nx))).astype(np.float32)
        probe = rng.standard_normal((nh, nz, nx))
        gain = np.linalg.norm(oracle.born_ext(self.og, self.v0.astype(np.float64), self.ogeo,
                                              self.w.astype(np.float64), probe)) / np.linalg.norm(probe)
        self.eps = float(0.1 * gain)
        self.fg = fw.Grid(nz=nz, nx=nx, sponge=W, nt=nt, dt=self.dt, dx=self.dx, nh=nh)
        self.fgeo = fw.Geometry(self.src_iz, self.src_ix, self.rec_iz, self.rec_ix)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32))).cuda()


@pytest.fixture(scope="module")
def case():
    assert torch.cuda.is_available()
    fw.load()
    return VP()


def oracle_vp(c, niter, dres=None):
    return oracle.vp_solve(c.og, c.v0.astype(np.float64), c.ogeo, c.w.astype(np.float64),
                           (c.dres if dres is None else dres).astype(np.float64), c.pt0.astype(np.float64),
                           c.eps, niter)


@pytest.mark.parametrize("niter", [0, 1, 4])
def test_vp_solve_matches_oracle(case, niter):
    c = case
    ctx = fw.Context(c.fg, c.fgeo)
    try:
        pt = dev(c.pt0)
        hist = ctx.vp_solve(dev(c.v0), dev(c.w), dev(c.dres), pt, eps=c.eps, niter=niter)
        p_ref, h_ref = oracle_vp(c, niter)
        p = pt.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(p - p_ref) / np.linalg.norm(p_ref) <= 1e-4
        assert len(hist) == niter + 1
        assert max(abs(a - b) for a, b in zip(hist, h_ref)) <= 1e-5 * h_ref[0], (hist, h_ref)
        assert all(b <= a * (1 + 1e-6) for a, b in zip(hist, hist[1:]))
    finally:
        ctx.close()


def test_vp_solve_batched_equals_plain_schedule(case):
    c = case
    out = []
    for opts in ({}, {"plain": 1}, {"shots_per_batch": 2, "segment": 7}):
        ctx = fw.Context(c.fg, c.fgeo, **opts)
        try:
            pt = dev(c.pt0)
            hist = ctx.vp_solve(dev(c.v0), dev(c.w), dev(c.dres), pt, eps=c.eps, niter=2)
            out.append((pt.cpu().numpy().astype(np.float64), hist))
        finally:
            ctx.close()
    for p, h in out[1:]:
        assert np.linalg.norm(p - out[0][0]) / np.linalg.norm(out[0][0]) <= 1e-5
        assert abs(h[-1] - out[0][1][-1]) <= 1e-6 * out[0][1][0]
