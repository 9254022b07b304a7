"""The schedule autotuner (segment length x shots per launch x stencil chunking, timed on the GPU):
the chosen schedule is one of its candidates, becomes the context's options, and the operators run
with it still match the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_2206_02362_gb300 as fw  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("op", [fw.OP_BORN_EXT_ADJ, fw.OP_GRADIENT, fw.OP_FORWARD])
def test_schedule_autotuner_picks_a_candidate_and_keeps_parity(op):
    nz, nx, W, nt, nh, dx, dt = 30, 100, 8, 130, 5, 10.0, 1e-3
    rng = np.random.default_rng(synth.SEED0 + 900)
    v = (1800.0 + 25.0 * np.arange(nz)[:, None] + 40.0 * rng.random((nz, nx))).astype(np.float32)
    src_ix = np.array([10, 30, 50, 70, 90, 95])
    geom = fw.Geometry(np.full(6, 2), src_ix, np.full(50, 1), 2 * np.arange(50))
    grid = fw.Grid(nz=nz, nx=nx, sponge=W, nt=nt, dt=dt, dx=dx, nh=nh)
    w = np.stack([synth.ricker(nt, dt, 20.0)] * 6).astype(np.float32)
    pt = rng.standard_normal((nh, nz, nx)).astype(np.float32)
    d_in = rng.standard_normal((6, nt, 50)).astype(np.float32)
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    with fw.Context(grid, geom) as ctx:
        s = ctx.autotune_schedule(op)
        K0 = max(min(int(round(np.sqrt(nt - 1))), 128), 8)
        assert s["segment"] in {K0, max(K0 // 2, 8), min(2 * K0, nt - 1)}
        assert 1 <= s["shots_per_batch"] <= 6 and s["zchunk"] > 0 and s["us_stencil"] > 0
        assert s["us_per_shot"] > 0
        assert ctx.get_option("segment") == s["segment"]
        assert ctx.get_option("shots_per_batch") == s["shots_per_batch"]
        assert ctx.get_option("zchunk") == s["zchunk"]
        img = torch.zeros((nh, nz, nx), device="cuda")
        ctx.born_ext_adj(cu(v), cu(w), cu(d_in), img)
        assert ctx.get_option("batch_used") == s["shots_per_batch"]
    og = oracle.Grid(nz=nz, nx=nx, W=W, nt=nt, dt=dt, dx=dx, nh=nh)
    ogeo = oracle.Geometry(np.full(6, 2), src_ix, np.full(50, 1), 2 * np.arange(50))
    ref = oracle.born_ext_adj(og, v.astype(np.float64), ogeo, w.astype(np.float64), d_in.astype(np.float64))
    assert np.linalg.norm(img.double().cpu().numpy() - ref) / np.linalg.norm(ref) <= 1e-4
