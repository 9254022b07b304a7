"""Shots of uneven size in one launch per time step (fwime_forward_group): three
contexts with different grids, record lengths and shot counts advance together;
each member's traces must equal its own fwime_forward bit for bit (the per-shot
arithmetic is the same), including members whose record ends early, and the
group must match the oracle."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_2206_02362_gb300 as fw  # noqa: E402

pytestmark = pytest.mark.gpu


def member(nz, nx, nt, nshot, seed):
    rng = np.random.default_rng(synth.SEED0 + 700 + seed)
    v = synth.layered(nz, nx, 10.0, synth.SEED0 + 710 + seed)
    src_ix = np.linspace(3, nx - 4, nshot).astype(int)
    geom = fw.Geometry(np.full(nshot, 2), src_ix, np.full(nx // 2, 1), 2 * np.arange(nx // 2))
    grid = fw.Grid(nz=nz, nx=nx, sponge=12, nt=nt, dt=1e-3, dx=10.0)
    w = np.stack([synth.ricker(nt, 1e-3, 18.0) * (1 + 0.05 * rng.random()) for _ in range(nshot)]).astype(np.float32)
    return grid, geom, v, w


def test_group_forward_matches_separate_calls_and_oracle():
    assert torch.cuda.is_available()
    specs = [member(40, 300, 260, 3, 0), member(25, 130, 400, 2, 1), member(60, 520, 150, 4, 2)]
    s = torch.cuda.Stream()
    ctxs, vs, ws, ds, refs = [], [], [], [], []
    with torch.cuda.stream(s):
        for grid, geom, v, w in specs:
            c = fw.Context(grid, geom, stream=s)
            vd, wd = torch.from_numpy(v).cuda(), torch.from_numpy(w).cuda()
            ref = torch.zeros((geom.nshot, grid.nt, geom.nrec), device="cuda")
            c.forward(vd, wd, ref)
            ctxs.append(c); vs.append(vd); ws.append(wd); refs.append(ref)
            ds.append(torch.full_like(ref, 3.0))
        fw.forward_group(ctxs, vs, ws, ds)
        # one model preparation per member, then a stencil and a recording launch per time step
        assert ctxs[0].launches == len(specs) + 2 * (max(g.nt for g, *_ in specs) - 1)
    for (grid, geom, v, w), d, ref in zip(specs, ds, refs):
        assert torch.equal(d, ref)
        og = oracle.Grid(nz=grid.nz, nx=grid.nx, W=grid.sponge, nt=grid.nt, dt=grid.dt, dx=grid.dx)
        ogeo = oracle.Geometry(geom.src_iz, geom.src_ix, geom.rec_iz, geom.rec_ix)
        o = oracle.forward(og, v.astype(np.float64), ogeo, w.astype(np.float64))
        dd = d.double().cpu().numpy()
        assert np.linalg.norm(dd - o) / np.linalg.norm(o) <= 1e-4
    for c in ctxs:
        c.close()


def test_group_members_must_share_a_stream():
    (g1, geo1, v1, w1), (g2, geo2, v2, w2) = member(20, 80, 50, 1, 3), member(20, 90, 60, 1, 4)
    with fw.Context(g1, geo1, stream=torch.cuda.Stream()) as a, fw.Context(g2, geo2, stream=torch.cuda.Stream()) as b:
        d1 = torch.zeros((1, 50, geo1.nrec), device="cuda")
        d2 = torch.zeros((1, 60, geo2.nrec), device="cuda")
        with pytest.raises(fw.FwimeError) as e:
            fw.forward_group([a, b], [torch.from_numpy(v1).cuda(), torch.from_numpy(v2).cuda()],
                             [torch.from_numpy(w1).cuda(), torch.from_numpy(w2).cuda()], [d1, d2])
        assert e.value.code == fw.FWIME_EINVAL
