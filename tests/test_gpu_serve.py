"""Continuous-batching request loop: requests of different grid sizes, nt and nh,
forward and gradient, arriving while others run.  Each result must be the same
alone and in the mix (bit-identical: the per-request arithmetic does not depend
on what else is on the GPU), memory admission must hold requests back when the
budget is small, and latencies are reported."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
from paper_2206_02362_gb300 import serve  # noqa: E402

pytestmark = pytest.mark.gpu


def mix(n=10, seed=5):
    reqs = synth.serving_mix(nreq=n, rate=400.0, seed=synth.SEED0 + 300 + seed, nz_range=(20, 40),
                             nx_range=(60, 160), nt_range=(120, 260), nh_choices=(1, 3, 5))
    return [serve.from_synth(r) for r in reqs]


def test_results_same_alone_and_in_the_mix():
    assert torch.cuda.is_available()
    reqs = mix()
    srv = serve.Server(max_active=16)
    try:
        mixed = srv.serve([r for r in reqs], realtime=True)
        alone = [srv.serve([r], realtime=False)[0] for r in reqs]
        burst = srv.serve([r for r in reqs], realtime=False)   # all admitted at once: forwards grouped
    finally:
        srv.close()
    for a, b in zip(alone, burst):
        if a.kind == "forward":
            assert np.array_equal(a.data, b.data)
        else:
            assert np.array_equal(a.grad, b.grad) and a.objective == b.objective
    assert [r.rid for r in mixed] == [r.rid for r in reqs]
    kinds = {r.kind for r in reqs}
    assert kinds == {"forward", "gradient"}
    for a, m in zip(alone, mixed):
        if a.kind == "forward":
            assert np.array_equal(a.data, m.data)
        else:
            assert np.array_equal(a.grad, m.grad) and a.objective == m.objective
    s = serve.summarize(mixed)
    assert s["p99_s"] >= s["p50_s"] > 0 and s["shots_per_s"] > 0


def test_served_forward_matches_oracle():
    req = mix(n=4)[0]
    req.kind = "forward"
    srv = serve.Server()
    try:
        res = srv.serve([req], realtime=False)[0]
    finally:
        srv.close()
    g = oracle.Grid(nz=req.nz, nx=req.nx, W=req.sponge, nt=req.nt, dt=req.dt, dx=req.dx, nh=req.nh)
    geo = oracle.Geometry(np.array([req.src[0]]), np.array([req.src[1]]), req.rec_iz, req.rec_ix)
    ref = oracle.forward(g, req.v.astype(np.float64), geo, req.w.astype(np.float64)[None])[0]
    assert np.linalg.norm(res.data - ref) / np.linalg.norm(ref) <= 1e-4


def test_memory_admission_limits_concurrency():
    reqs = mix(n=6, seed=9)
    biggest = max(serve.request_bytes(r) for r in reqs)
    srv = serve.Server(memory_budget=biggest + (1 << 20))     # room for about one request at a time
    try:
        res = srv.serve(reqs, realtime=False)
    finally:
        srv.close()
    assert len(res) == len(reqs)
    order = sorted(res, key=lambda r: r.admitted)
    for a, b in zip(order, order[1:]):
        # with room for one, a request is admitted only after an earlier one finished, unless both fit
        if serve.request_bytes(next(q for q in reqs if q.rid == a.rid)) + \
                serve.request_bytes(next(q for q in reqs if q.rid == b.rid)) > biggest + (1 << 20):
            assert b.admitted >= a.done - 1e-3


def test_over_budget_request_is_rejected():
    reqs = mix(n=1)
    srv = serve.Server(memory_budget=1 << 20)
    try:
        with pytest.raises(ValueError):
            srv.serve(reqs, realtime=False)
    finally:
        srv.close()


def test_device_pointer_requests_through_the_c_abi():
    """fwime_submit with device buffers (host_io = 0): a forward and a gradient request on different
    grids, submitted together and waited for; each result equals the same operator on its own context
    bit for bit."""
    import ctypes

    import paper_2206_02362_gb300 as fw
    lib = fw.load()
    reqs = mix(n=12, seed=11)
    grd = next(r for r in reqs if r.kind == "gradient")
    fwd = next(r for r in reqs if r is not grd)
    fwd.kind = "forward"                       # (a gradient request's p~ and d_obs are then unused)
    h = ctypes.c_void_p()
    assert lib.fwime_server_create(ctypes.byref(h), ctypes.c_size_t(4 << 30), 8, 0) == fw.FWIME_OK
    keep, tickets, outs = [], [], []
    try:
        for r in (fwd, grd):
            grid = fw.Grid(nz=r.nz, nx=r.nx, sponge=r.sponge, nt=r.nt, dt=r.dt, dx=r.dx, nh=r.nh)
            geom = fw.Geometry(np.array([r.src[0]]), np.array([r.src[1]]), r.rec_iz, r.rec_ix)
            t = {"v": torch.from_numpy(r.v).cuda(), "w": torch.from_numpy(r.w[None]).cuda()}
            if r.kind == "forward":
                t["out"] = torch.zeros((1, r.nt, len(r.rec_iz)), device="cuda")
            else:
                t["pt"] = torch.from_numpy(r.pt).cuda()
                t["dobs"] = torch.from_numpy(r.dobs[None]).cuda()
                t["out"] = torch.zeros((r.nz, r.nx), device="cuda")
            gm, kg = geom.c()
            p = lambda k: t[k].data_ptr() if k in t else None  # noqa: E731
            c = fw.RequestC(fw.REQ_FORWARD if r.kind == "forward" else fw.REQ_GRADIENT, grid.c(), gm, 0,
                            p("v"), p("w"), p("pt"), p("dobs"), p("out") if r.kind == "forward" else None,
                            p("out") if r.kind == "gradient" else None, ctypes.c_float(r.eps))
            tk = ctypes.c_uint64(0)
            assert lib.fwime_submit(h, ctypes.byref(c), ctypes.byref(tk)) == fw.FWIME_OK
            keep.append((c, kg, gm, grid, geom))
            tickets.append(tk.value)
            outs.append(t)
        res = []
        for tk in tickets:
            rr = fw.ResultC()
            assert lib.fwime_wait(h, ctypes.c_uint64(tk), ctypes.byref(rr)) == fw.FWIME_OK
            assert rr.done == 1 and rr.status == fw.FWIME_OK and rr.latency_s >= rr.queued_s >= 0.0
            res.append(rr.objective)
        r = fw.ResultC()
        assert lib.fwime_poll(h, ctypes.c_uint64(tickets[0]), ctypes.byref(r)) == fw.FWIME_EINVAL   # collected once
    finally:
        lib.fwime_destroy(h)
    (c0, _, _, grid0, geom0), (c1, _, _, grid1, geom1) = keep
    with fw.Context(grid0, geom0, shots_per_batch=1) as ctx:
        ref = torch.zeros_like(outs[0]["out"])
        ctx.forward(outs[0]["v"], outs[0]["w"], ref)
    assert torch.equal(ref, outs[0]["out"])
    with fw.Context(grid1, geom1, shots_per_batch=1) as ctx:
        g = torch.zeros_like(outs[1]["out"])
        J = ctx.gradient(outs[1]["v"], outs[1]["w"], outs[1]["pt"], outs[1]["dobs"], g, eps=grd.eps)
    assert torch.equal(g, outs[1]["out"]) and J == res[1]
