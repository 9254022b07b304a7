"""GPU free surface (FWIME_OPT_FREE_SURFACE) against the oracle's free-surface reading: forward data,
B, B*, B~, B~*, T*, the gradient, with receivers on and just below the surface, batched and plain
schedules, plus the GPU dot test of (B~, B~*)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_2206_02362_gb300 as fw  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-4


class FS:
    def __init__(self, nh=5, nt=240, nshot=3, seed=0):
        nz, nx, W = 32, 160, 10
        rng = np.random.default_rng(synth.SEED0 + 900 + seed)
        z = np.arange(nz)[:, None]; x = np.arange(nx)[None, :]
        self.v = (1700.0 + 25.0 * z + 100.0 * np.sin(x / 11.0) * np.cos(z / 5.0)).astype(np.float32)
        self.src_iz, self.src_ix = np.array([1, 3, 2][:nshot]), np.linspace(4, nx - 5, nshot).astype(int)
        # receivers on the surface row, one and two rows below, and deeper
        self.rec_iz = np.concatenate([np.full(40, 0), np.full(40, 1), np.full(40, 2), [20, 25]])
        self.rec_ix = np.concatenate([4 * np.arange(40), 4 * np.arange(40) + 1, 4 * np.arange(40) + 2, [10, 150]])
        self.w = np.stack([synth.ricker(nt, 1e-3, 22.0) * (1 + 0.1 * s) for s in range(nshot)]).astype(np.float32)
        self.dv = synth.gaussian_blobs(nz, nx, rng, amp=40.0, sigma_pts=4.0, ring=1).astype(np.float32)
        self.pt = rng.standard_normal((nh, nz, nx)).astype(np.float32)
        self.d = rng.standard_normal((nshot, nt, len(self.rec_iz))).astype(np.float32)
        self.og = oracle.Grid(nz=nz, nx=nx, W=W, nt=nt, dt=1e-3, dx=10.0, nh=nh, fs=1)
        self.ogeo = oracle.Geometry(self.src_iz, self.src_ix, self.rec_iz, self.rec_ix)
        self.fg = fw.Grid(nz=nz, nx=nx, sponge=W, nt=nt, dt=1e-3, dx=10.0, nh=nh)
        self.fgeo = fw.Geometry(self.src_iz, self.src_ix, self.rec_iz, self.rec_ix)


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def case():
    assert torch.cuda.is_available()
    return FS()


@pytest.mark.parametrize("opts", [{}, dict(shots_per_batch=2, segment=9), dict(plain=1)])
def test_free_surface_operators_match_oracle(case, opts):
    c = case
    v, w = c.v.astype(np.float64), c.w.astype(np.float64)
    ref = {
        "fwd": oracle.forward(c.og, v, c.ogeo, w),
        "born": oracle.born(c.og, v, c.ogeo, w, c.dv.astype(np.float64)),
        "born_adj": oracle.born_adj(c.og, v, c.ogeo, w, c.d.astype(np.float64)),
        "ext": oracle.born_ext(c.og, v, c.ogeo, w, c.pt.astype(np.float64)),
        "ext_adj": oracle.born_ext_adj(c.og, v, c.ogeo, w, c.d.astype(np.float64)),
        "tomo_adj": oracle.tomo_adj(c.og, v, c.ogeo, w, c.pt.astype(np.float64), c.d.astype(np.float64)),
    }
    with fw.Context(c.fg, c.fgeo, free_surface=1, **opts) as ctx:
        out = {}
        d = torch.zeros(c.d.shape, device="cuda"); ctx.forward(T(c.v), T(c.w), d); out["fwd"] = d.double().cpu().numpy()
        d = torch.zeros(c.d.shape, device="cuda"); ctx.born(T(c.v), T(c.w), T(c.dv), d); out["born"] = d.double().cpu().numpy()
        m = torch.zeros(c.v.shape, device="cuda"); ctx.born_adj(T(c.v), T(c.w), T(c.d), m); out["born_adj"] = m.double().cpu().numpy()
        d = torch.zeros(c.d.shape, device="cuda"); ctx.born_ext(T(c.v), T(c.w), T(c.pt), d); out["ext"] = d.double().cpu().numpy()
        e = torch.zeros(c.pt.shape, device="cuda"); ctx.born_ext_adj(T(c.v), T(c.w), T(c.d), e); out["ext_adj"] = e.double().cpu().numpy()
        m = torch.zeros(c.v.shape, device="cuda"); ctx.tomo_adj(T(c.v), T(c.w), T(c.pt), T(c.d), m); out["tomo_adj"] = m.double().cpu().numpy()
    assert np.all(out["fwd"][:, :, :40] == 0.0)      # receivers on the surface row
    for k in ref:
        assert rel(out[k], ref[k]) <= TOL, k


def test_free_surface_gradient_matches_oracle(case):
    c = case
    pts = (1e-3 * c.pt).astype(np.float32)
    dobs = (1e-3 * c.d).astype(np.float32)
    J_ref, g_ref = oracle.gradient(c.og, c.v.astype(np.float64), c.ogeo, c.w.astype(np.float64),
                                   pts.astype(np.float64), dobs.astype(np.float64), eps=0.1)
    with fw.Context(c.fg, c.fgeo, free_surface=1) as ctx:
        g = torch.zeros(c.v.shape, device="cuda")
        J = ctx.gradient(T(c.v), T(c.w), T(pts), T(dobs), g, eps=0.1)
    assert rel(g.double().cpu().numpy(), g_ref) <= TOL
    assert abs(J - J_ref) <= 1e-5 * abs(J_ref)


def test_free_surface_time_lag_and_background_reuse(case):
    """The free surface composes with the time-lag extension and with the background reuse."""
    c = FS(nh=5, nt=200, seed=1)
    og = oracle.Grid(nz=c.og.nz, nx=c.og.nx, W=c.og.W, nt=c.og.nt, dt=c.og.dt, dx=c.og.dx, nh=5, fs=1, lag=2)
    ref = oracle.born_ext_adj(og, c.v.astype(np.float64), c.ogeo, c.w.astype(np.float64), c.d.astype(np.float64))
    with fw.Context(c.fg, c.fgeo, free_surface=1, time_lag=2) as ctx:
        e = torch.zeros(c.pt.shape, device="cuda")
        ctx.born_ext_adj(T(c.v), T(c.w), T(c.d), e)
    assert rel(e.double().cpu().numpy(), ref) <= TOL
    ref2 = oracle.born_ext_adj(c.og, c.v.astype(np.float64), c.ogeo, c.w.astype(np.float64), c.d.astype(np.float64))
    vd, wd, pd, dd = T(c.v), T(c.w), T(c.pt), T(c.d)
    with fw.Context(c.fg, c.fgeo, free_surface=1, reuse_background=1) as ctx:
        ctx.born_ext(vd, wd, pd, torch.zeros_like(dd))
        e = torch.zeros(c.pt.shape, device="cuda")
        ctx.born_ext_adj(vd, wd, dd, e)
        assert ctx.get_option("background_reused") == 1
    assert rel(e.double().cpu().numpy(), ref2) <= TOL
