"""Background checkpoint reuse (FWIME_OPT_REUSE_BACKGROUND): B~* / B* that start from the
segment-start states kept by the preceding B~ / B on the same v and w must give the results of
the self-contained operators (and of the oracle), launch fewer kernels, and fall back to their
own checkpointing sweep whenever the states may not belong to their inputs."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_2206_02362_gb300 as fw  # noqa: E402

pytestmark = pytest.mark.gpu


def setup(nshot=3, nt=250, nh=5, seed=0):
    nz, nx, W = 37, 300, 10
    rng = np.random.default_rng(synth.SEED0 + 500 + seed)
    z = np.arange(nz)[:, None]; x = np.arange(nx)[None, :]
    v = (1800.0 + 20.0 * z + 150.0 * np.sin(x / 17.0) * np.cos(z / 5.0)).astype(np.float32)
    src_iz, src_ix = np.array([0, 3, 1][:nshot]), np.linspace(0, nx - 1, nshot).astype(int)
    rec_iz, rec_ix = np.full(100, 0), 3 * np.arange(100)
    w = np.stack([synth.ricker(nt, 1e-3, 20.0) * (1 + 0.1 * s) for s in range(nshot)]).astype(np.float32)
    grid = fw.Grid(nz=nz, nx=nx, sponge=W, nt=nt, dt=1e-3, dx=10.0, nh=nh)
    geom = fw.Geometry(src_iz, src_ix, rec_iz, rec_ix)
    pt = rng.standard_normal((nh, nz, nx)).astype(np.float32)
    d = rng.standard_normal((nshot, nt, len(rec_iz))).astype(np.float32)
    return grid, geom, v, w, pt, d


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    a = a.double().cpu().numpy(); b = b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("opts", [dict(), dict(shots_per_batch=2, segment=7), dict(graph=1)])
def test_ext_adjoint_from_cached_background(opts):
    assert torch.cuda.is_available()
    grid, geom, v, w, pt, d = setup()
    vd, wd, ptd, dd = T(v), T(w), T(pt), T(d)
    dout = torch.zeros_like(dd)
    stream = torch.cuda.Stream() if opts.get("graph") else None
    torch.cuda.synchronize()
    with fw.Context(grid, geom, stream=stream, **opts) as plain:
        ref = torch.zeros((grid.nh, grid.nz, grid.nx), device="cuda")
        plain.born_ext_adj(vd, wd, dd, ref)
        n_plain = plain.launches
    with fw.Context(grid, geom, stream=stream, reuse_background=1, **opts) as c:
        for it in range(2):                       # the second round replays graphs in graph mode
            img = torch.zeros_like(ref)
            torch.cuda.synchronize()
            c.born_ext(vd, wd, ptd, dout)
            c.born_ext_adj(vd, wd, dd, img)
            assert rel(img, ref) <= 1e-6
            assert c.launches < n_plain            # no checkpointing sweep
            assert c.get_option("background_reused") == 1
    o = oracle.born_ext_adj(oracle.Grid(nz=grid.nz, nx=grid.nx, W=grid.sponge, nt=grid.nt, dt=grid.dt, dx=grid.dx,
                                        nh=grid.nh),
                            v.astype(np.float64), oracle.Geometry(geom.src_iz, geom.src_ix, geom.rec_iz, geom.rec_ix),
                            w.astype(np.float64), d.astype(np.float64))
    assert np.linalg.norm(img.double().cpu().numpy() - o) / np.linalg.norm(o) <= 1e-4


def test_born_adjoint_from_cached_background():
    grid, geom, v, w, pt, d = setup(nh=1)
    vd, wd, dd = T(v), T(w), T(d)
    dv = T(synth.gaussian_blobs(grid.nz, grid.nx, np.random.default_rng(3), amp=50.0, sigma_pts=4.0,
                                ring=1).astype(np.float32))
    with fw.Context(grid, geom) as plain:
        ref = torch.zeros((grid.nz, grid.nx), device="cuda")
        plain.born_adj(vd, wd, dd, ref)
    with fw.Context(grid, geom, reuse_background=1) as c:
        out = torch.zeros_like(ref)
        c.born(vd, wd, dv, torch.zeros_like(dd))
        c.born_adj(vd, wd, dd, out)
    assert rel(out, ref) <= 1e-6


def test_cache_is_not_used_for_other_inputs():
    grid, geom, v, w, pt, d = setup()
    vd, wd, ptd, dd = T(v), T(w), T(pt), T(d)
    v2 = T(v * np.float32(1.05))
    with fw.Context(grid, geom) as plain:
        ref = torch.zeros((grid.nh, grid.nz, grid.nx), device="cuda")
        plain.born_ext_adj(v2, wd, dd, ref)
        n_plain = plain.launches
    with fw.Context(grid, geom, reuse_background=1) as c:
        img = torch.zeros_like(ref)
        c.born_ext(vd, wd, ptd, torch.zeros_like(dd))
        c.born_ext_adj(v2, wd, dd, img)            # another model: own sweep
        assert rel(img, ref) <= 1e-6 and c.launches == n_plain
        assert c.get_option("background_reused") == 0
        c.born_ext(v2, wd, ptd, torch.zeros_like(dd))
        c.forward(v2, wd, torch.zeros_like(dd))   # any other operator drops the states
        img2 = torch.zeros_like(ref)
        c.born_ext_adj(v2, wd, dd, img2)
        assert rel(img2, ref) <= 1e-6 and c.launches == n_plain
        c.set_option("reuse_background", 0)        # frees them
        assert c.get_option("reuse_background") == 0


def test_host_io_path_reuses_the_staged_background():
    grid, geom, v, w, pt, d = setup()
    with fw.Context(grid, geom) as plain:
        ref = torch.zeros((grid.nh, grid.nz, grid.nx), device="cuda")
        plain.born_ext_adj(T(v), T(w), T(d), ref)
    with fw.Context(grid, geom, reuse_background=1, host_io=1) as c:
        img = np.zeros((grid.nh, grid.nz, grid.nx), np.float32)
        dh = np.zeros_like(d)
        for _ in range(2):                         # the first round may grow (move) the arena
            c.born_ext(v, w, pt, dh)
            c.born_ext_adj(v, w, d, img)
        assert c.get_option("background_reused") == 1
    r = ref.double().cpu().numpy()
    assert np.linalg.norm(img - r) / np.linalg.norm(r) <= 1e-6
