"""Serving FWIME shot requests through libfwime's request server.

A request is one forward-modelling shot (f, Eq. 1) or one FWIME-gradient shot
(Phi and B* r + T* r at fixed p~, Eqs. 1, 7-9) on its own grid, nt and nh.
The continuous batching itself runs natively behind the C ABI
(``fwime_server_create`` / ``fwime_submit`` / ``fwime_poll`` / ``fwime_wait``):
admission by device memory (``fwime_request_bytes``) and in-flight slots while
earlier requests run, one stream and context per request so admitted requests
overlap, grouped launches for forward requests admitted together, completion by
CUDA events.  This module only marshals: it pins each request's host buffers,
submits requests at their arrival times, polls, and reports per-request latency
(arrival -> result in host memory), p50/p99 and throughput.
"""
from __future__ import annotations

import ctypes
import time
from dataclasses import dataclass

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
    enqueue_s: float = 0.0              # host time the server spent enqueuing its launches

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class _Marshalled:
    """A request's pinned host buffers and its fwime_request (kept alive until collected)."""

    def __init__(self, req: ShotRequest):
        import torch

        import paper_2206_02362_gb300 as fw
        self.req = req

        def pin(a):
            t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).pin_memory()
            return t

        nrec = len(req.rec_iz)
        self.t = {"v": pin(req.v), "w": pin(np.asarray(req.w)[None])}
        if req.kind == "forward":
            self.t["d"] = torch.empty((1, req.nt, nrec), pin_memory=True)
        else:
            self.t["pt"] = pin(req.pt)
            self.t["dobs"] = pin(np.asarray(req.dobs)[None])
            self.t["g"] = torch.empty((req.nz, req.nx), pin_memory=True)
        self.grid = fw.Grid(nz=req.nz, nx=req.nx, sponge=req.sponge, nt=req.nt, dt=req.dt, dx=req.dx, nh=req.nh)
        self.geom = fw.Geometry(np.array([req.src[0]]), np.array([req.src[1]]), req.rec_iz, req.rec_ix)
        gm, self._keep = self.geom.c()
        ptr = lambda k: self.t[k].data_ptr() if k in self.t else None  # noqa: E731
        self.c = fw.RequestC(fw.REQ_FORWARD if req.kind == "forward" else fw.REQ_GRADIENT, self.grid.c(), gm, 1,
                             ptr("v"), ptr("w"), ptr("pt"), ptr("dobs"), ptr("d"), ptr("g"),
                             ctypes.c_float(req.eps))


def request_bytes(req: ShotRequest) -> int:
    """Device bytes the server admits a request with: workspace + staging (fwime_request_bytes)."""
    import paper_2206_02362_gb300 as fw
    grid = fw.Grid(nz=req.nz, nx=req.nx, sponge=req.sponge, nt=req.nt, dt=req.dt, dx=req.dx, nh=req.nh)
    geom = fw.Geometry(np.array([req.src[0]]), np.array([req.src[1]]), req.rec_iz, req.rec_ix)
    gm, keep = geom.c()
    c = fw.RequestC(fw.REQ_FORWARD if req.kind == "forward" else fw.REQ_GRADIENT, grid.c(), gm, 1,
                    None, None, None, None, None, None, ctypes.c_float(req.eps))
    out = ctypes.c_size_t(0)
    rc = fw.load().fwime_request_bytes(ctypes.byref(c), ctypes.byref(out))
    if rc != fw.FWIME_OK:
        raise fw.FwimeError(rc, "fwime_request_bytes")
    return int(out.value)


class Server:
    """libfwime's request server on the current CUDA device (fwime_server_create)."""

    def __init__(self, memory_budget: int | None = None, max_active: int = 64, device: int = 0,
                 plain: bool = False):
        import torch

        import paper_2206_02362_gb300 as fw
        self.fw = fw
        torch.cuda.set_device(device)
        if memory_budget is None:
            free, _ = torch.cuda.mem_get_info(device)
            memory_budget = int(0.8 * free)
        self.budget = memory_budget
        self._lib = fw.load()
        self._h = ctypes.c_void_p()
        rc = self._lib.fwime_server_create(ctypes.byref(self._h), ctypes.c_size_t(memory_budget), int(max_active),
                                           fw.SERVE_PLAIN if plain else 0)
        if rc != fw.FWIME_OK:
            raise fw.FwimeError(rc, "fwime_server_create")

    def _error(self) -> str:
        buf = ctypes.create_string_buffer(256)
        self._lib.fwime_server_last_error(buf, 256)
        return buf.value.decode(errors="replace")

    def submit(self, m: _Marshalled) -> int:
        t = ctypes.c_uint64(0)
        rc = self._lib.fwime_submit(self._h, ctypes.byref(m.c), ctypes.byref(t))
        if rc == self.fw.FWIME_ENOMEM:
            raise ValueError(self._error())
        if rc != self.fw.FWIME_OK:
            raise self.fw.FwimeError(rc, "fwime_submit", self._error())
        return int(t.value)

    def poll(self, ticket: int):
        r = self.fw.ResultC()
        rc = self._lib.fwime_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(r))
        if rc != self.fw.FWIME_OK:
            raise self.fw.FwimeError(rc, "fwime_poll")
        return r if r.done else None

    def wait(self, ticket: int):
        r = self.fw.ResultC()
        rc = self._lib.fwime_wait(self._h, ctypes.c_uint64(ticket), ctypes.byref(r))
        if rc != self.fw.FWIME_OK:
            raise self.fw.FwimeError(rc, "fwime_wait")
        return r

    def serve(self, requests: list[ShotRequest], realtime: bool = True) -> list[ShotResult]:
        """Submits each request at req.arrival seconds (realtime) or all at once, collects every result;
        returns the results in rid order."""
        for r in requests:
            need = request_bytes(r)
            if need > self.budget:
                raise ValueError(f"request {r.rid} needs {need} bytes, over the budget {self.budget}")
        marsh = {r.rid: _Marshalled(r) for r in requests}
        pending = sorted(requests, key=lambda r: r.arrival)
        inflight = {}                  # ticket -> (request, submit time)
        results = {}
        t0 = time.perf_counter()
        k = 0
        while k < len(pending) or inflight:
            now = time.perf_counter() - t0
            while k < len(pending) and (not realtime or pending[k].arrival <= now):
                req = pending[k]
                k += 1
                ts = time.perf_counter() - t0
                if not realtime:
                    req.arrival = ts
                inflight[self.submit(marsh[req.rid])] = (req, ts)
            for ticket in list(inflight):
                res = self.poll(ticket)
                if res is None:
                    continue
                req, ts = inflight.pop(ticket)
                done = ts + res.latency_s          # the server's clock: completion of the copy to host memory
                if res.status != self.fw.FWIME_OK:
                    raise self.fw.FwimeError(res.status, f"request {req.rid}")
                m = marsh[req.rid]
                out = ShotResult(req.rid, req.kind, req.arrival, ts + res.queued_s, done, enqueue_s=res.enqueue_s)
                if req.kind == "forward":
                    out.data = m.t["d"][0].numpy().copy()
                else:
                    out.grad = m.t["g"].numpy().copy()
                    out.objective = float(res.objective)
                results[req.rid] = out
            if inflight and not (k < len(pending) and pending[k].arrival <= time.perf_counter() - t0):
                time.sleep(2e-4)
        self.last_wall = time.perf_counter() - t0       # serving time, after the buffers were pinned
        return [results[r] for r in sorted(results)]

    def close(self):
        if self._h.value:
            self._lib.fwime_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def summarize(results: list[ShotResult], wall: float | None = None) -> dict:
    lat = np.array([r.latency for r in results])
    span = wall if wall is not None else (max(r.done for r in results) - min(r.arrival for r in results))
    return {"requests": len(results), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "shots_per_s": len(results) / span, "span_s": span,
            "enqueue_s_total": float(sum(r.enqueue_s for r in results))}


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
