"""Receiver recording and injection folded into the stencil launches, on geometries that stress
the receiver map: receivers spread over many rows (a vertical line, as in a VSP, plus a surface
line), two receivers on the same grid point, and receivers next to the grid's edges.  f, B~ and
B~* (whose adjoint steps inject the data residual) against the FP64 oracle, and the traces of the
repeated receivers identical."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_2206_02362_gb300 as fw  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-4


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("opts", [dict(), dict(shots_per_batch=1, segment=9), dict(plain=1)])
def test_spread_and_repeated_receivers_match_oracle(opts):
    nz, nx, W, nt, nh, dx, dt = 36, 90, 8, 180, 5, 10.0, 1e-3
    rng = np.random.default_rng(synth.SEED0 + 800)
    v = (1700.0 + 20.0 * np.arange(nz)[:, None] + 50.0 * rng.random((nz, nx))).astype(np.float32)
    rec_iz = np.concatenate([np.full(30, 1), np.arange(2, nz, 2), [1, 1, nz - 1, 0], [17, 17]])
    rec_ix = np.concatenate([3 * np.arange(30), np.full(len(range(2, nz, 2)), 60), [9, 9, nx - 1, 0], [44, 44]])
    src_iz, src_ix = np.array([2, 20]), np.array([30, 70])
    w = np.stack([synth.ricker(nt, dt, 20.0)] * 2).astype(np.float32)
    pt = rng.standard_normal((nh, nz, nx)).astype(np.float32)
    grid = fw.Grid(nz=nz, nx=nx, sponge=W, nt=nt, dt=dt, dx=dx, nh=nh)
    geom = fw.Geometry(src_iz, src_ix, rec_iz, rec_ix)
    og = oracle.Grid(nz=nz, nx=nx, W=W, nt=nt, dt=dt, dx=dx, nh=nh)
    ogeo = oracle.Geometry(src_iz, src_ix, rec_iz, rec_ix)
    v64, w64 = v.astype(np.float64), w.astype(np.float64)
    f_ref = oracle.forward(og, v64, ogeo, w64)
    d_ref = oracle.born_ext(og, v64, ogeo, w64, pt.astype(np.float64))
    d_in = rng.standard_normal(d_ref.shape).astype(np.float32)
    i_ref = oracle.born_ext_adj(og, v64, ogeo, w64, d_in.astype(np.float64))
    nrec = len(rec_iz)
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    with fw.Context(grid, geom, **opts) as ctx:
        f = torch.zeros((2, nt, nrec), device="cuda")
        ctx.forward(cu(v), cu(w), f)
        d = torch.zeros((2, nt, nrec), device="cuda")
        ctx.born_ext(cu(v), cu(w), cu(pt), d)
        img = torch.zeros((nh, nz, nx), device="cuda")
        ctx.born_ext_adj(cu(v), cu(w), cu(d_in), img)
    f, d = f.cpu().numpy(), d.cpu().numpy()
    assert rel(f, f_ref) <= TOL and rel(d, d_ref) <= TOL
    assert rel(img.cpu().numpy(), i_ref) <= TOL
    # repeated receivers (columns 30/31 of the extra block, 34/35) record the same traces
    k = 30 + len(range(2, nz, 2))
    assert np.array_equal(f[:, :, k], f[:, :, k + 1]) and np.array_equal(f[:, :, k + 4], f[:, :, k + 5])
