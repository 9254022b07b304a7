"""Continuous-batching request loop for FWIME shot requests on one GPU.

A request is one forward-modelling shot (f, Eq. 1) or one FWIME-gradient shot
(Phi and B* r + T* r at fixed p~, Eqs. 1, 7-9) on its own grid, nt and nh.
Requests arrive over time; the loop

  * admits a request as soon as its device memory (workspace from
    fwime_workspace_bytes plus its inputs/outputs) fits the budget and an
    in-flight slot is free -- while other requests are still running;
  * keeps its model, wavelet, p~, data and wavefields resident on the device
    for the life of the request, on a CUDA stream of its own, so the work of
    all admitted requests overlaps on the GPU;
  * enqueues each request's kernels from a worker thread (the C ABI releases
    the GIL), detects completion with a CUDA event, returns the result to
    pinned host memory and releases the memory for the next admissions;
  * reports per-request latency (arrival -> result on the host), p50/p99 and
    throughput.

Device memory is stream-ordered (libfwime allocates with cudaMallocAsync on the
request's stream), so finishing one request never synchronises the others.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class ShotRequest:
    """One shot on its own grid.  v [nz][nx] m/s; w [nt]; for gradients p~ [nh][nz][nx] and d_obs [nt][nrec]."""
    rid: int
    kind: str                      # "forward" | "gradient"
    arrival: float                 # seconds after the start of serving
    nz: int
    nx: int
    dx: float
    dt: float
    nt: int
    nh: int
    sponge: int
    src: tuple
    rec_iz: np.ndarray
    rec_ix: np.ndarray
    v: np.ndarray
    w: np.ndarray
    pt: np.ndarray | None = None
    dobs: np.ndarray | None = None
    eps: float = 0.0


@dataclass
class ShotResult:
    rid: int
    kind: str
    arrival: float
    admitted: float
    done: float
    data: np.ndarray | None = None      # forward: d [nt][nrec]
    grad: np.ndarray | None = None      # gradient: [nz][nx]
    objective: float | None = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class _Active:
    req: ShotRequest
    ctx: object
    stream: object
    event: object
    tensors: dict
    host_out: object
    nbytes: int
    admitted: float
    future: object = None
    J: list = field(default_factory=list)


def request_bytes(req: ShotRequest) -> int:
    """Device bytes a request holds while admitted: workspace + inputs + outputs."""
    import paper_2206_02362_gb300 as fw
    grid = fw.Grid(nz=req.nz, nx=req.nx, sponge=req.sponge, nt=req.nt, dt=req.dt, dx=req.dx, nh=req.nh)
    geom = fw.Geometry(np.array([req.src[0]]), np.array([req.src[1]]), req.rec_iz, req.rec_ix)
    op = fw.OP_FORWARD if req.kind == "forward" else fw.OP_GRADIENT
    ws = fw.workspace_bytes(grid, geom, op, 1, 0)
    io = 4 * (req.v.size + req.nt + req.nt * len(req.rec_iz))
    if req.kind == "gradient":
        io += 4 * (req.pt.size + req.v.size)
    return ws + io + (1 << 20)


class Server:
    """Memory-admitted, stream-overlapped request loop on one CUDA device."""

    def __init__(self, memory_budget: int | None = None, max_active: int = 64, workers: int = 8, device: int = 0,
                 plain: bool = False, group_forward: bool = True):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        if memory_budget is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            memory_budget = int(0.8 * free)
        self.budget = memory_budget
        self.max_active = max_active
        self.plain = plain              # one shot per launch, host-driven steps (the comparison path)
        # forward requests admitted together run as one group: one launch per time step for all of
        # them, whatever their grid sizes and record lengths (fwime_forward_group)
        self.group_forward = group_forward and not plain
        self.pool = cf.ThreadPoolExecutor(max_workers=workers)

    # ---------------------------------------------------------------- one request
    def _admit(self, req: ShotRequest, nbytes: int, now: float) -> _Active:
        import paper_2206_02362_gb300 as fw
        torch = self.torch
        stream = torch.cuda.Stream(device=self.device)
        grid = fw.Grid(nz=req.nz, nx=req.nx, sponge=req.sponge, nt=req.nt, dt=req.dt, dx=req.dx, nh=req.nh)
        geom = fw.Geometry(np.array([req.src[0]]), np.array([req.src[1]]), req.rec_iz, req.rec_ix)
        nrec = len(req.rec_iz)
        with torch.cuda.stream(stream):
            t = {"v": torch.from_numpy(np.ascontiguousarray(req.v, dtype=np.float32)).pin_memory()
                 .to(self.device, non_blocking=True),
                 "w": torch.from_numpy(np.ascontiguousarray(req.w, dtype=np.float32)[None]).pin_memory()
                 .to(self.device, non_blocking=True)}
            if req.kind == "forward":
                t["d"] = torch.empty((1, req.nt, nrec), device=self.device)
                host_out = torch.empty((req.nt, nrec), pin_memory=True)
            else:
                t["pt"] = torch.from_numpy(np.ascontiguousarray(req.pt, dtype=np.float32)).pin_memory() \
                    .to(self.device, non_blocking=True)
                t["dobs"] = torch.from_numpy(np.ascontiguousarray(req.dobs, dtype=np.float32)[None]).pin_memory() \
                    .to(self.device, non_blocking=True)
                t["g"] = torch.empty((req.nz, req.nx), device=self.device)
                host_out = torch.empty((req.nz, req.nx), pin_memory=True)
        ctx = fw.Context(grid, geom, stream=stream, shots_per_batch=1, plain=int(self.plain))
        act = _Active(req, ctx, stream, torch.cuda.Event(), t, host_out, nbytes, now)

        def enqueue():
            with torch.cuda.stream(stream):
                if req.kind == "forward":
                    ctx.forward(t["v"], t["w"], t["d"], sync=False)
                    host_out.copy_(t["d"][0], non_blocking=True)
                else:
                    ctx.gradient(t["v"], t["w"], t["pt"], t["dobs"], t["g"], eps=req.eps, sync=False)
                    host_out.copy_(t["g"], non_blocking=True)
                act.event.record(stream)

        act.future = self.pool.submit(enqueue)
        return act

    def _admit_forward_group(self, reqs: list, sizes: dict, now: float) -> list:
        import paper_2206_02362_gb300 as fw
        torch = self.torch
        stream = torch.cuda.Stream(device=self.device)
        acts, ctxs, vs, ws, ds = [], [], [], [], []
        event = torch.cuda.Event()
        with torch.cuda.stream(stream):
            for req in reqs:
                grid = fw.Grid(nz=req.nz, nx=req.nx, sponge=req.sponge, nt=req.nt, dt=req.dt, dx=req.dx, nh=req.nh)
                geom = fw.Geometry(np.array([req.src[0]]), np.array([req.src[1]]), req.rec_iz, req.rec_ix)
                t = {"v": torch.from_numpy(np.ascontiguousarray(req.v, dtype=np.float32)).pin_memory()
                     .to(self.device, non_blocking=True),
                     "w": torch.from_numpy(np.ascontiguousarray(req.w, dtype=np.float32)[None]).pin_memory()
                     .to(self.device, non_blocking=True),
                     "d": torch.empty((1, req.nt, len(req.rec_iz)), device=self.device)}
                host_out = torch.empty((req.nt, len(req.rec_iz)), pin_memory=True)
                ctx = fw.Context(grid, geom, stream=stream, shots_per_batch=1)
                acts.append(_Active(req, ctx, stream, event, t, host_out, sizes[req.rid], now))
                ctxs.append(ctx); vs.append(t["v"]); ws.append(t["w"]); ds.append(t["d"])

        def enqueue():
            with torch.cuda.stream(stream):
                fw.forward_group(ctxs, vs, ws, ds, sync=False)
                for a in acts:
                    a.host_out.copy_(a.tensors["d"][0], non_blocking=True)
                event.record(stream)

        fut = self.pool.submit(enqueue)
        for a in acts:
            a.future = fut
        return acts

    def _finish(self, act: _Active, now: float) -> ShotResult:
        act.ctx.sync()                       # already complete; reads the status word and the objective
        r = ShotResult(act.req.rid, act.req.kind, act.req.arrival, act.admitted, now)
        if act.req.kind == "forward":
            r.data = act.host_out.numpy().copy()
        else:
            r.grad = act.host_out.numpy().copy()
            r.objective = float(act.ctx._J.value)
        act.ctx.close()
        return r

    # ---------------------------------------------------------------- the loop
    def serve(self, requests: list[ShotRequest], realtime: bool = True) -> list[ShotResult]:
        """Serves requests arriving at req.arrival seconds (realtime) or all at once; returns results in rid order."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        queue: collections.deque = collections.deque()
        active: list[_Active] = []
        used = 0
        results = {}
        sizes = {r.rid: request_bytes(r) for r in requests}
        for r in requests:
            if sizes[r.rid] > self.budget:
                raise ValueError(f"request {r.rid} needs {sizes[r.rid]} bytes, over the budget {self.budget}")
        t0 = time.perf_counter()
        while pending or queue or active:
            now = time.perf_counter() - t0
            while pending and (not realtime or pending[0].arrival <= now):
                req = pending.popleft()
                if not realtime:
                    req.arrival = now
                queue.append(req)
            # admission: FIFO, as memory and slots free up
            admitted = []
            while queue and len(active) + len(admitted) < self.max_active and \
                    used + sizes[queue[0].rid] <= self.budget:
                req = queue.popleft()
                admitted.append(req)
                used += sizes[req.rid]
            fwd = [r for r in admitted if r.kind == "forward"] if self.group_forward else []
            grouped = {r.rid for r in fwd} if len(fwd) > 1 else set()
            if grouped:
                active.extend(self._admit_forward_group(fwd, sizes, time.perf_counter() - t0))
            for req in admitted:
                if req.rid not in grouped:
                    active.append(self._admit(req, sizes[req.rid], time.perf_counter() - t0))
            # completion
            still = []
            for act in active:
                if act.future.done() and act.event.query():
                    act.future.result()
                    results[act.req.rid] = self._finish(act, time.perf_counter() - t0)
                    used -= act.nbytes
                else:
                    still.append(act)
            active = still
            if not (pending and pending[0].arrival <= time.perf_counter() - t0):
                time.sleep(2e-4)
        return [results[k] for k in sorted(results)]

    def close(self):
        self.pool.shutdown(wait=True)


def summarize(results: list[ShotResult], wall: float | None = None) -> dict:
    lat = np.array([r.latency for r in results])
    span = wall if wall is not None else (max(r.done for r in results) - min(r.arrival for r in results))
    return {"requests": len(results), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "shots_per_s": len(results) / span, "span_s": span}


def from_synth(req) -> ShotRequest:
    """Converts a synth.Request (seeded serving-mix entry) into a ShotRequest with its inputs."""
    wl = req.workload
    rng = np.random.default_rng(wl.seed)
    pt = dobs = None
    if req.kind == "gradient":
        pt = (1e-3 * rng.standard_normal((wl.nh, wl.nz, wl.nx))).astype(np.float32)
        dobs = (1e-3 * rng.standard_normal((wl.nt, wl.nrec))).astype(np.float32)
    return ShotRequest(req.rid, req.kind, req.arrival, wl.nz, wl.nx, wl.dx, wl.dt, wl.nt, wl.nh, wl.W,
                       (int(wl.src_iz[0]), int(wl.src_ix[0])), wl.rec_iz, wl.rec_ix, wl.v,
                       wl.w.astype(np.float32), pt, dobs, 1e-3)
