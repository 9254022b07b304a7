"""GPU linear spline re-parametrisation S / S* (Eq. 1) against the oracle: uniform and non-uniform
nodes, nodes reaching past the grid, a single node per axis and nodes on every grid point (S = I);
GPU dot test; gradient through S with autograd."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_2206_02362_gb300 as fw  # noqa: E402
from paper_2206_02362_gb300.autograd import spline_param  # noqa: E402

pytestmark = pytest.mark.gpu

NZ, NX, DZ, DX = 61, 203, 10.0, 10.0
NODES = {
    "uniform": (np.arange(0, 601, 200.0), np.arange(0, 2021, 450.0)),
    "nonuniform": (np.array([-30.0, 55.0, 120.0, 130.0, 470.0, 640.0]), np.array([5.0, 300.0, 1100.0, 1333.0, 2000.0])),
    "single": (np.array([250.0]), np.array([1000.0])),
    "identity": (np.arange(NZ) * DZ, np.arange(NX) * DX),
}


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available()
    g = fw.Grid(nz=NZ, nx=NX, sponge=8, nt=10, dt=1e-3, dx=DX, dz=DZ)
    geo = fw.Geometry(np.array([1]), np.array([5]), np.array([1]), np.array([7]))
    with fw.Context(g, geo) as c:
        yield c


@pytest.mark.parametrize("name", list(NODES))
def test_spline_matches_oracle(ctx, name):
    zs, xs = NODES[name]
    rng = np.random.default_rng(synth.SEED0 + 600)
    m = (2000.0 + 300.0 * rng.standard_normal((len(zs), len(xs)))).astype(np.float32)
    g = rng.standard_normal((NZ, NX)).astype(np.float32)
    v = torch.zeros((NZ, NX), device="cuda")
    ctx.spline(zs, xs, torch.from_numpy(m).cuda(), v)
    ref = oracle.spline(zs.astype(np.float32), xs.astype(np.float32), NZ, NX, DZ, DX, m.astype(np.float64))
    assert np.abs(v.double().cpu().numpy() - ref).max() <= 1e-6 * np.abs(ref).max()
    ma = torch.zeros((len(zs), len(xs)), device="cuda")
    ctx.spline(zs, xs, torch.from_numpy(g).cuda(), ma, adjoint=True)
    refa = oracle.spline_adj(zs.astype(np.float32), xs.astype(np.float32), NZ, NX, DZ, DX, g.astype(np.float64))
    assert np.linalg.norm(ma.double().cpu().numpy() - refa) <= 1e-5 * np.linalg.norm(refa)
    if name == "identity":
        assert torch.equal(v, torch.from_numpy(m).cuda())


def test_spline_dot_and_accumulate(ctx):
    zs, xs = NODES["nonuniform"]
    rng = np.random.default_rng(7)
    m = torch.from_numpy(rng.standard_normal((len(zs), len(xs))).astype(np.float32)).cuda()
    g = torch.from_numpy(rng.standard_normal((NZ, NX)).astype(np.float32)).cuda()
    v = torch.zeros((NZ, NX), device="cuda")
    a = torch.zeros_like(m)
    ctx.spline(zs, xs, m, v)
    ctx.spline(zs, xs, g, a, adjoint=True)
    lhs = float((v.double() * g.double()).sum()); rhs = float((m.double() * a.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    v2 = v.clone()
    ctx.spline(zs, xs, m, v2, accumulate=True)
    assert torch.allclose(v2, 2 * v, rtol=1e-6, atol=0)


def test_unsorted_nodes_are_rejected(ctx):
    with pytest.raises(fw.FwimeError):
        ctx.spline(np.array([0.0, 50.0, 40.0]), np.array([0.0, 100.0]), torch.zeros((3, 2), device="cuda"),
                   torch.zeros((NZ, NX), device="cuda"))


def test_autograd_through_the_spline(ctx):
    zs, xs = NODES["uniform"]
    rng = np.random.default_rng(9)
    m = torch.from_numpy(rng.standard_normal((len(zs), len(xs))).astype(np.float32)).cuda().requires_grad_(True)
    wgt = torch.from_numpy(rng.standard_normal((NZ, NX)).astype(np.float32)).cuda()
    v = spline_param(ctx, zs, xs, m)
    (v * wgt).sum().backward()
    a = torch.zeros_like(m)
    ctx.spline(zs, xs, wgt, a, adjoint=True)
    assert torch.allclose(m.grad, a, rtol=1e-6, atol=1e-6)


def test_spline_refinement_matches_oracle_and_reproduces_the_coarse_model(ctx):
    """Model-space multiscale step: a 0.2 km x 0.45 km coarse grid refined by halving its spacing twice.
    The carried-over model equals the oracle's, and S on the fine nodes reproduces S on the coarse nodes
    on the finite-difference grid (every coarse node is a fine node)."""
    zc, xc = np.arange(0, 601, 200.0), np.arange(0, 2021, 450.0)
    zf, xf = np.arange(0, 601, 50.0), np.arange(0, 2021, 112.5)
    rng = np.random.default_rng(synth.SEED0 + 601)
    mc = (2000.0 + 300.0 * rng.standard_normal((len(zc), len(xc)))).astype(np.float32)
    mf = torch.zeros((len(zf), len(xf)), device="cuda")
    ctx.spline_refine(zc, xc, torch.from_numpy(mc).cuda(), zf, xf, mf)
    ref = oracle.spline_refine(zc.astype(np.float32), xc.astype(np.float32), mc.astype(np.float64),
                               zf.astype(np.float32), xf.astype(np.float32))
    assert np.abs(mf.double().cpu().numpy() - ref).max() <= 1e-6 * np.abs(ref).max()
    assert torch.equal(mf[::4, ::4], torch.from_numpy(mc).cuda())     # shared nodes keep their values
    vf, vc = torch.zeros((NZ, NX), device="cuda"), torch.zeros((NZ, NX), device="cuda")
    ctx.spline(zf, xf, mf, vf)
    ctx.spline(zc, xc, torch.from_numpy(mc).cuda(), vc)
    assert (vf - vc).abs().max().item() <= 1e-6 * vc.abs().max().item()
