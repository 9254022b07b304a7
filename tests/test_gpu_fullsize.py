"""Full-size checks at the workloads' real sizes, in the launch configuration the
benchmark times (all shots batched, automatic segment length):

* Marmousi2-shaped (350 x 1700, 100 shots, nt 4000, nh 21): B~/B~* dot test over
  all shots; every shot's traces identical alone and inside the 100-shot batch;
  two sampled shots against the oracle on the full grid at a shortened record.
* North-Sea-shaped (400 x 1600, 120 shots, nt 5000, nh 31): the FWIME gradient
  against central finite differences of the objective along 10 random smooth
  perturbations (the workload's own check).
* Salt-shaped (1200 x 5000, nt 8000, nh 41, where the source history does not fit
  in HBM and checkpointing is required): T/T* dot test on 2 shots.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_2206_02362_gb300 as fw  # noqa: E402

pytestmark = pytest.mark.gpu


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def dot64(a, b):
    return float(torch.sum(a.double() * b.double()).item())


@pytest.fixture(scope="module")
def marm():
    assert torch.cuda.is_available()
    wl = synth.marmousi2()
    grid = fw.Grid(nz=wl.nz, nx=wl.nx, sponge=wl.W, nt=wl.nt, dt=wl.dt, dx=wl.dx, nh=wl.nh)
    geom = fw.Geometry(wl.src_iz, wl.src_ix, wl.rec_iz, wl.rec_ix)
    return wl, grid, geom


def test_marmousi2_full_size_dot_and_batch_consistency(marm):
    wl, grid, geom = marm
    rng = np.random.default_rng(synth.SEED0 + 600)
    v = cu(wl.v)
    w = cu(np.broadcast_to(wl.w, (wl.nshot, wl.nt)))
    pt = cu(rng.standard_normal((wl.nh, wl.nz, wl.nx)))
    dr = cu(rng.standard_normal((wl.nshot, wl.nt, wl.nrec)))
    d = torch.zeros((wl.nshot, wl.nt, wl.nrec), device="cuda")
    img = torch.zeros((wl.nh, wl.nz, wl.nx), device="cuda")
    with fw.Context(grid, geom) as ctx:
        ctx.born_ext(v, w, pt, d)
        ctx.born_ext_adj(v, w, dr, img)
        assert ctx.get_option("workspace") > 0
    lhs, rhs = dot64(d, dr), dot64(pt, img)
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), abs(rhs))
    # shots 0, 57 and 99 alone (one shot per context) reproduce the batched traces bit for bit
    for s in (0, 57, 99):
        g1 = fw.Geometry(wl.src_iz[s:s + 1], wl.src_ix[s:s + 1], wl.rec_iz, wl.rec_ix)
        d1 = torch.zeros((1, wl.nt, wl.nrec), device="cuda")
        with fw.Context(grid, g1) as c1:
            c1.born_ext(v, w[s:s + 1].contiguous(), pt, d1)
        assert torch.equal(d1[0], d[s])


def test_marmousi2_full_grid_sampled_shots_against_oracle(marm):
    """Two shots on the full 350 x 1700 grid (receivers every 20 m, nh 21), 300 time steps:
    the oracle's FP64 traces and extended image for exactly these shots."""
    wl, _, _ = marm
    nt = 300
    idx = np.array([11, 73])
    rng = np.random.default_rng(synth.SEED0 + 601)
    grid = fw.Grid(nz=wl.nz, nx=wl.nx, sponge=wl.W, nt=nt, dt=wl.dt, dx=wl.dx, nh=wl.nh)
    geom = fw.Geometry(wl.src_iz[idx], wl.src_ix[idx], wl.rec_iz, wl.rec_ix)
    w = np.stack([wl.w[:nt]] * 2).astype(np.float32)
    pt = rng.standard_normal((wl.nh, wl.nz, wl.nx)).astype(np.float32)
    og = oracle.Grid(nz=wl.nz, nx=wl.nx, W=wl.W, nt=nt, dt=wl.dt, dx=wl.dx, nh=wl.nh)
    ogeo = oracle.Geometry(wl.src_iz[idx], wl.src_ix[idx], wl.rec_iz, wl.rec_ix)
    d_ref = oracle.born_ext(og, wl.v.astype(np.float64), ogeo, w.astype(np.float64), pt.astype(np.float64))
    d_in = d_ref.astype(np.float32)            # the adjoint's input: the oracle's traces, as both sides see them
    d = torch.zeros((2, nt, wl.nrec), device="cuda")
    img = torch.zeros((wl.nh, wl.nz, wl.nx), device="cuda")
    with fw.Context(grid, geom) as ctx:
        ctx.born_ext(cu(wl.v), cu(w), cu(pt), d)
        ctx.born_ext_adj(cu(wl.v), cu(w), cu(d_in), img)
    dg = d.double().cpu().numpy()
    assert np.linalg.norm(dg - d_ref) / np.linalg.norm(d_ref) <= 1e-4
    i_ref = oracle.born_ext_adj(og, wl.v.astype(np.float64), ogeo, w.astype(np.float64), d_in.astype(np.float64))
    ig = img.double().cpu().numpy()
    assert np.linalg.norm(ig - i_ref) / np.linalg.norm(i_ref) <= 1e-4


def test_north_sea_full_size_gradient_against_finite_differences():
    wl, v0 = synth.north_sea()
    grid = fw.Grid(nz=wl.nz, nx=wl.nx, sponge=wl.W, nt=wl.nt, dt=wl.dt, dx=wl.dx, nh=wl.nh)
    geom = fw.Geometry(wl.src_iz, wl.src_ix, wl.rec_iz, wl.rec_ix)
    rng = np.random.default_rng(synth.SEED0 + 602)
    w = cu(np.broadcast_to(wl.w, (wl.nshot, wl.nt)))
    pt = cu(1e-4 * rng.standard_normal((wl.nh, wl.nz, wl.nx)))
    with fw.Context(grid, geom) as ctx:
        dobs = torch.zeros((wl.nshot, wl.nt, wl.nrec), device="cuda")
        ctx.forward(cu(wl.v), w, dobs)                   # observed data from the true model
        g = torch.zeros((wl.nz, wl.nx), device="cuda")
        ctx.gradient(cu(v0), w, pt, dobs, g, eps=1e-3)
        g = g.double().cpu().numpy()
        gn = np.linalg.norm(g)
        errs = []
        for k in range(10):
            dv = synth.gaussian_blobs(wl.nz, wl.nx, rng, nblob=4, amp=1.0, sigma_pts=30.0, ring=2)
            e = 5.0
            jp = ctx.objective(cu(v0 + e * dv), w, pt, dobs, eps=1e-3)
            jm = ctx.objective(cu(v0 - e * dv), w, pt, dobs, eps=1e-3)
            errs.append(abs((jp - jm) / (2 * e) - float((g * dv).sum())) / (gn * np.linalg.norm(dv)))
    assert max(errs) <= 1e-3, errs


def test_salt_full_size_tomographic_dot_test():
    wl = synth.salt(nshot=2)
    grid = fw.Grid(nz=wl.nz, nx=wl.nx, sponge=wl.W, nt=wl.nt, dt=wl.dt, dx=wl.dx, nh=wl.nh)
    geom = fw.Geometry(wl.src_iz, wl.src_ix, wl.rec_iz, wl.rec_ix)
    NZ, NX = wl.padded
    history = wl.nt * NZ * NX * 4
    free, _ = torch.cuda.mem_get_info()
    assert history > 0.5 * free          # the source-wavefield history alone would not fit
    rng = np.random.default_rng(synth.SEED0 + 603)
    w = cu(np.broadcast_to(wl.w, (2, wl.nt)))
    pt = cu(rng.standard_normal((wl.nh, wl.nz, wl.nx)))
    dv = cu(synth.gaussian_blobs(wl.nz, wl.nx, rng, nblob=6, amp=50.0, sigma_pts=40.0, ring=2))
    dr = cu(rng.standard_normal((2, wl.nt, wl.nrec)))
    d = torch.zeros_like(dr)
    g = torch.zeros((wl.nz, wl.nx), device="cuda")
    with fw.Context(grid, geom) as ctx:
        ctx.tomo(cu(wl.v), w, pt, dv, d)
        ctx.tomo_adj(cu(wl.v), w, pt, dr, g)
    lhs, rhs = dot64(d, dr), dot64(dv, g)
    assert np.isfinite(lhs) and abs(lhs - rhs) <= 1e-5 * max(abs(lhs), abs(rhs))
