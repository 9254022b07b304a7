"""GPU time-lag extension (B~ / B~* extended with time lags, Eq. 1; FWIME_OPT_TIME_LAG) against the
FP64 oracle: several lag counts and spacings, ragged segments shorter and longer than the lag reach,
ragged shot batches, a generic lag count, the GPU dot test and the VP solve with time lags."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_2206_02362_gb300 as fw  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-4


class TL:
    def __init__(self, nh, lag, nt=260, nshot=3, seed=0):
        nz, nx, W = 30, 150, 10
        rng = np.random.default_rng(synth.SEED0 + 800 + seed)
        z = np.arange(nz)[:, None]; x = np.arange(nx)[None, :]
        self.v = (1800.0 + 25.0 * z + 120.0 * np.sin(x / 13.0) * np.cos(z / 4.0)).astype(np.float32)
        self.src_iz, self.src_ix = np.array([0, 2, 1][:nshot]), np.linspace(5, nx - 6, nshot).astype(int)
        self.rec_iz, self.rec_ix = np.full(75, 1), 2 * np.arange(75)
        self.w = np.stack([synth.ricker(nt, 1e-3, 22.0) * (1 + 0.1 * s) for s in range(nshot)]).astype(np.float32)
        self.pt = rng.standard_normal((nh, nz, nx)).astype(np.float32)
        self.d = rng.standard_normal((nshot, nt, len(self.rec_iz))).astype(np.float32)
        self.og = oracle.Grid(nz=nz, nx=nx, W=W, nt=nt, dt=1e-3, dx=10.0, nh=nh, lag=lag)
        self.ogeo = oracle.Geometry(self.src_iz, self.src_ix, self.rec_iz, self.rec_ix)
        self.fg = fw.Grid(nz=nz, nx=nx, sponge=W, nt=nt, dt=1e-3, dx=10.0, nh=nh)
        self.fgeo = fw.Geometry(self.src_iz, self.src_ix, self.rec_iz, self.rec_ix)
        self.lag = lag

    def ctx(self, **opt):
        return fw.Context(self.fg, self.fgeo, time_lag=self.lag, **opt)


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("nh,lag,opts", [
    (5, 3, {}),
    (5, 3, dict(shots_per_batch=2, segment=7)),     # segments shorter than the lag reach (Hs = 12)
    (21, 1, dict(segment=40)),
    (11, 4, dict(segment=13)),
    (7, 2, {}),                                     # generic lag count
    (1, 1, {}),
    # chunks of 16 outputs of one residue class, the window carried from chunk to chunk: two chunks (30
    # per class), three (45 per class), and the generic kernel (28 per class)
    (5, 1, dict(segment=60)),
    (3, 1, dict(segment=90)),
    (7, 1, dict(segment=56)),
    # 75 outputs per class in chunks of 16: the window carried over four times
    (5, 1, dict(segment=150)),
])
def test_time_lag_born_and_adjoint_match_oracle(nh, lag, opts):
    assert torch.cuda.is_available()
    c = TL(nh, lag)
    v, w = c.v.astype(np.float64), c.w.astype(np.float64)
    ref_d = oracle.born_ext(c.og, v, c.ogeo, w, c.pt.astype(np.float64))
    ref_i = oracle.born_ext_adj(c.og, v, c.ogeo, w, c.d.astype(np.float64))
    with c.ctx(**opts) as ctx:
        d = torch.zeros(c.d.shape, device="cuda")
        ctx.born_ext(T(c.v), T(c.w), T(c.pt), d)
        img = torch.zeros(c.pt.shape, device="cuda")
        ctx.born_ext_adj(T(c.v), T(c.w), T(c.d), img)
    assert rel(d.double().cpu().numpy(), ref_d) <= TOL
    assert rel(img.double().cpu().numpy(), ref_i) <= TOL


def test_time_lag_gpu_dot_product():
    c = TL(11, 2)
    with c.ctx() as ctx:
        d = torch.zeros(c.d.shape, device="cuda")
        ctx.born_ext(T(c.v), T(c.w), T(c.pt), d)
        img = torch.zeros(c.pt.shape, device="cuda")
        ctx.born_ext_adj(T(c.v), T(c.w), T(c.d), img)
    dd, dref = d.double().cpu(), torch.from_numpy(c.d).double()
    lhs = float((dd * dref).sum())
    rhs = float((img.double().cpu() * torch.from_numpy(c.pt).double()).sum())
    # random data against B~ p~ cancel heavily: bound the mismatch by the Cauchy-Schwarz scale
    assert abs(lhs - rhs) <= 1e-5 * float(dd.norm() * dref.norm())


def test_time_lag_vp_solve_matches_oracle():
    c = TL(5, 3, nt=200)
    rng = np.random.default_rng(3)
    dres = (0.1 * rng.standard_normal(c.d.shape)).astype(np.float32)
    pt0 = np.zeros_like(c.pt)
    eps = 0.5
    p_ref, h_ref = oracle.vp_solve(c.og, c.v.astype(np.float64), c.ogeo, c.w.astype(np.float64),
                                   dres.astype(np.float64), pt0.astype(np.float64), eps, 3)
    with c.ctx() as ctx:
        pt = T(pt0)
        hist = ctx.vp_solve(T(c.v), T(c.w), T(dres), pt, eps=eps, niter=3)
    assert rel(pt.double().cpu().numpy(), p_ref) <= TOL
    assert max(abs(a - b) for a, b in zip(hist, h_ref)) <= 1e-5 * h_ref[0]


@pytest.mark.parametrize("nh,lag,opts", [(5, 3, {}), (5, 3, dict(shots_per_batch=2, segment=7)), (11, 2, dict(segment=20)),
                                         (5, 1, dict(segment=100))])
def test_time_lag_tomo_and_gradient_match_oracle(nh, lag, opts):
    c = TL(nh, lag, nt=220)
    rng = np.random.default_rng(21)
    dv = synth.gaussian_blobs(c.og.nz, c.og.nx, rng, amp=40.0, sigma_pts=4.0, ring=1).astype(np.float32)
    pts = (1e-3 * c.pt).astype(np.float32)
    v, w = c.v.astype(np.float64), c.w.astype(np.float64)
    ref_t = oracle.tomo(c.og, v, c.ogeo, w, pts.astype(np.float64), dv.astype(np.float64))
    ref_ta = oracle.tomo_adj(c.og, v, c.ogeo, w, pts.astype(np.float64), c.d.astype(np.float64))
    dobs = (1e-3 * c.d).astype(np.float32)
    J_ref, g_ref = oracle.gradient(c.og, v, c.ogeo, w, pts.astype(np.float64), dobs.astype(np.float64), eps=0.1)
    with c.ctx(**opts) as ctx:
        d = torch.zeros(c.d.shape, device="cuda")
        ctx.tomo(T(c.v), T(c.w), T(pts), T(dv), d)
        ta = torch.zeros((c.og.nz, c.og.nx), device="cuda")
        ctx.tomo_adj(T(c.v), T(c.w), T(pts), T(c.d), ta)
        g = torch.zeros((c.og.nz, c.og.nx), device="cuda")
        J = ctx.gradient(T(c.v), T(c.w), T(pts), T(dobs), g, eps=0.1)
        Jo = ctx.objective(T(c.v), T(c.w), T(pts), T(dobs), eps=0.1)
    assert rel(d.double().cpu().numpy(), ref_t) <= TOL
    assert rel(ta.double().cpu().numpy(), ref_ta) <= TOL
    assert rel(g.double().cpu().numpy(), g_ref) <= TOL
    assert abs(J - J_ref) <= 1e-5 * abs(J_ref) and abs(Jo - J_ref) <= 1e-5 * abs(J_ref)


def test_time_lag_segment_falls_back_when_the_long_one_does_not_fit():
    """The default time-lag segment (4 Hs steps) needs more workspace per shot than 2 Hs; under a budget
    between the two the context plans 2 Hs segments instead of refusing, with the same results."""
    c = TL(5, 3)                      # Hs = 12: default K = 48, fallback K = 24
    v, w = c.v.astype(np.float64), c.w.astype(np.float64)
    ref_i = oracle.born_ext_adj(c.og, v, c.ogeo, w, c.d.astype(np.float64))
    img = torch.zeros(c.pt.shape, device="cuda")
    ws = {}
    for seg in (0, 24):
        with c.ctx(shots_per_batch=1, segment=seg) as ctx:
            ctx.born_ext_adj(T(c.v), T(c.w), T(c.d), img)
            ws[seg] = ctx.get_option("workspace")
    assert ws[0] > ws[24]
    with fw.Context(c.fg, c.fgeo, max_workspace_bytes=(ws[0] + ws[24]) // 2, time_lag=c.lag,
                    shots_per_batch=1) as ctx:
        img.zero_()
        ctx.born_ext_adj(T(c.v), T(c.w), T(c.d), img)
        assert ctx.get_option("workspace") <= (ws[0] + ws[24]) // 2
    assert rel(img.double().cpu().numpy(), ref_i) <= TOL
