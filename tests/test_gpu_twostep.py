"""Two time steps per stencil launch (FWIME_OPT_TWO_STEP, temporal blocking) give the same numbers as
one step per launch: the arithmetic of every point is the same, only the launch structure changes.
Checked for the forward data, B~ (background with D2t and point source, scattered field with local
sources), B~* (segment recomputation) and the background reuse, with odd and even segment lengths,
ragged shot batches and grids whose width is not a multiple of the 120-column strips."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_2206_02362_gb300 as fw  # noqa: E402

pytestmark = pytest.mark.gpu


def case(nz=37, nx=300, nt=251, nh=5, nshot=3, seed=0):
    rng = np.random.default_rng(synth.SEED0 + 950 + seed)
    z = np.arange(nz)[:, None]; x = np.arange(nx)[None, :]
    v = (1800.0 + 20.0 * z + 150.0 * np.sin(x / 17.0) * np.cos(z / 5.0)).astype(np.float32)
    src_iz, src_ix = np.array([0, 3, 1][:nshot]), np.linspace(0, nx - 1, nshot).astype(int)
    rec_iz, rec_ix = np.full(nx // 3, 1), 3 * np.arange(nx // 3)
    w = np.stack([synth.ricker(nt, 1e-3, 20.0) * (1 + 0.1 * s) for s in range(nshot)]).astype(np.float32)
    grid = fw.Grid(nz=nz, nx=nx, sponge=10, nt=nt, dt=1e-3, dx=10.0, nh=nh)
    geom = fw.Geometry(src_iz, src_ix, rec_iz, rec_ix)
    pt = rng.standard_normal((nh, nz, nx)).astype(np.float32)
    d = rng.standard_normal((nshot, nt, len(rec_iz))).astype(np.float32)
    return grid, geom, v, w, pt, d


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def run(grid, geom, v, w, pt, d, **opts):
    with fw.Context(grid, geom, **opts) as c:
        vd, wd = T(v), T(w)
        # leave wavefields all over the workspace first: a buffer that the stencil reads without
        # having written or zeroed it then shows up as a difference
        c.born_ext_adj(vd, wd, T(d), torch.zeros(pt.shape, device="cuda"))
        c.tomo_adj(vd, wd, T(pt), T(d), torch.zeros(v.shape, device="cuda"))
        f = torch.zeros(d.shape, device="cuda"); c.forward(vd, wd, f)
        e = torch.zeros(d.shape, device="cuda"); c.born_ext(vd, wd, T(pt), e)
        i = torch.zeros(pt.shape, device="cuda"); c.born_ext_adj(vd, wd, T(d), i)
    return f.cpu().numpy(), e.cpu().numpy(), i.cpu().numpy()


@pytest.mark.parametrize("opts", [dict(), dict(segment=7), dict(shots_per_batch=2, segment=10)])
@pytest.mark.parametrize("shape", [(37, 300, 251), (20, 121, 60), (45, 480, 100)])
def test_two_step_equals_one_step(opts, shape):
    assert torch.cuda.is_available()
    nz, nx, nt = shape
    grid, geom, v, w, pt, d = case(nz, nx, nt)
    one = run(grid, geom, v, w, pt, d, two_step=0, **opts)
    two = run(grid, geom, v, w, pt, d, two_step=1, **opts)
    for a, b in zip(one, two):
        assert np.max(np.abs(a - b)) <= 1e-6 * np.max(np.abs(a)), np.max(np.abs(a - b)) / np.max(np.abs(a))


def test_two_step_matches_oracle_and_reuse():
    grid, geom, v, w, pt, d = case(37, 300, 251)
    og = oracle.Grid(nz=grid.nz, nx=grid.nx, W=grid.sponge, nt=grid.nt, dt=grid.dt, dx=grid.dx, nh=grid.nh)
    ogeo = oracle.Geometry(geom.src_iz, geom.src_ix, geom.rec_iz, geom.rec_ix)
    ref = oracle.born_ext_adj(og, v.astype(np.float64), ogeo, w.astype(np.float64), d.astype(np.float64))
    vd, wd, pd, dd = T(v), T(w), T(pt), T(d)
    with fw.Context(grid, geom, reuse_background=1, two_step=1) as c:
        c.born_ext(vd, wd, pd, torch.zeros_like(dd))
        img = torch.zeros(pt.shape, device="cuda")
        c.born_ext_adj(vd, wd, dd, img)
        assert c.get_option("background_reused") == 1
    img = img.double().cpu().numpy()
    assert np.linalg.norm(img - ref) / np.linalg.norm(ref) <= 1e-4
