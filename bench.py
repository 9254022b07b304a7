#!/usr/bin/env python
"""FWIME operator benchmark on one GB300 (or N, shot-sharded, weak scaling).

One step = the extended Born operator B~ followed by its adjoint B~* (extended
imaging condition) over every shot of the workload, all shots batched
(Barnier et al., Theory section Eqs. 1-5; the computational-cost analysis
counts each as two wavefield propagations, Eq. 10).  Default workload: the
Marmousi2-shaped synthetic stand-in, 350 x 1700 at 10 m, 100 shots, 850
receivers, nt = 4000, dt = 0.8 ms, nh = 21 subsurface offsets, sponge 50.

value = useful grid-point updates per second: 4 propagations x shots x
(padded NZ x NX) x (nt - 1) per step (the recomputation of the background
wavefield is not counted as useful work), summed over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "Gpt/s per propagation & FWIME-gradient shots/s, batched vs plain; %HBM peak"
UNIT = "Gupd/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nshot", type=int, default=100)
    ap.add_argument("--nt", type=int, default=4000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--segment", type=int, default=0, help="checkpoint/ring segment length (0 = auto)")
    ap.add_argument("--no-grad", action="store_true", help="skip the FWIME-gradient batched-vs-plain section")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (automatic schedule)")
    ap.add_argument("--tune", default="schedule", choices=["schedule", "chunk"],
                    help="schedule: segment x shots per launch x chunking; chunk: the stencil's chunking only")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving-mix section")
    ap.add_argument("--serve-requests", type=int, default=300)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-active", type=int, default=16, help="requests in flight at most")
    ap.add_argument("--grad-shots", type=int, default=120)
    ap.add_argument("--grad-nt", type=int, default=0, help="record length of the gradient section (0 = the workload's)")
    ap.add_argument("--no-tlag", action="store_true", help="skip the time-lag extension section")
    ap.add_argument("--no-salt", action="store_true", help="skip the Salt-shaped batched-gradient section")
    ap.add_argument("--salt-shots", type=int, default=4)
    ap.add_argument("--no-reuse", action="store_true",
                    help="B~* runs its own checkpointing sweep instead of starting from the background states "
                         "kept by the B~ of the same step")
    return ap.parse_args()


def workload(args):
    return synth.marmousi2(nshot=args.nshot, nt=args.nt)


def updates_per_step(wl) -> float:
    NZ, NX = wl.padded
    return 4.0 * wl.nshot * NZ * NX * (wl.nt - 1)


def config(wl, args, n):
    NZ, NX = wl.padded
    return {"workload": wl.name, "nz": wl.nz, "nx": wl.nx, "padded": [NZ, NX], "dx_m": wl.dx, "dt_s": wl.dt,
            "nt": wl.nt, "nshot": wl.nshot, "nrec": wl.nrec, "nh": wl.nh, "sponge": wl.W,
            "operators": "B~ then B~* per step (extended Born + extended imaging), all shots batched",
            "global_batch": wl.nshot * n, "parallelism": f"shots x{n}" if n > 1 else "single GPU",
            "l2": "inputs larger than L2 (wavefields of 100 shots, tens of GB), no flush needed"}


# --------------------------------------------------------------------- clocks

class Clocks:
    """nvidia-smi sampled every 200 ms during the timed region."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait(timeout=10)
        self.f.flush()
        rows = []
        for ln in open(self.f.name):
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            if self.uuid and self.uuid not in parts[0]:
                continue
            rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        power = [float(r[3]) for r in rows if re.match(r"^[0-9.]+$", r[3])]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(power) if power else None}


# ------------------------------------------------------------------ oracle CPU

def oracle_sample(wl, nt_sample: int, nshot_sample: int, threads: int):
    """Times the FP64 oracle (as it stands) on B~ + B~* for a bounded sample of the workload."""
    import oracle
    oracle.build()
    og = oracle.Grid(nz=wl.nz, nx=wl.nx, W=wl.W, nt=nt_sample, dt=wl.dt, dx=wl.dx, nh=wl.nh)
    geo = oracle.Geometry(wl.src_iz[:nshot_sample], wl.src_ix[:nshot_sample], wl.rec_iz, wl.rec_ix)
    rng = np.random.default_rng(synth.SEED0 + 11)
    pt = rng.standard_normal((wl.nh, wl.nz, wl.nx))
    w = np.asarray(wl.w[:nt_sample], dtype=np.float64)
    v = wl.v.astype(np.float64)
    t0 = time.perf_counter()
    d = oracle.born_ext(og, v, geo, w, pt, nthreads=threads)
    oracle.born_ext_adj(og, v, geo, w, d, nthreads=threads)
    dt = time.perf_counter() - t0
    NZ, NX = wl.padded
    upd = 4.0 * nshot_sample * NZ * NX * (nt_sample - 1)
    return upd / dt / 1e9, dt, f"{nshot_sample} shots x nt={nt_sample} of the {wl.name} grid (B~ + B~*)"


# The oracle's CPU sample: B~ + B~* over nt = ORACLE_NT steps of the bench grid, one shot per host core
# (OpenMP over shots), bounded by the host memory its full FP64 histories take.
ORACLE_NT = 32


def oracle_plan(wl):
    """(shots, threads, host cores) of the oracle sample: every host core runs one shot, as long as
    the shots' histories (about 8 padded FP64 fields x nt per shot) fit in half the available memory."""
    try:
        cores = len(os.sched_getaffinity(0))      # the cores this process may run on (nproc)
    except AttributeError:
        cores = os.cpu_count() or 1
    NZ, NX = wl.padded
    per_shot = 8 * NZ * NX * ORACLE_NT * 8
    avail = None
    try:
        for ln in open("/proc/meminfo"):
            if ln.startswith("MemAvailable:"):
                avail = int(ln.split()[1]) * 1024
    except OSError:
        pass
    n = min(cores, wl.nshot)
    if avail:
        n = max(1, min(n, int(0.5 * avail // per_shot)))
    return n, n, cores


def cpu_baseline(wl):
    nshot, threads, cores = oracle_plan(wl)
    val, dt, sample = oracle_sample(wl, ORACLE_NT, nshot, threads)
    return {"value": val, "unit": UNIT, "cores": threads, "host_cores": cores, "kind": "oracle", "sample": sample,
            "seconds": round(dt, 2)}


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands, on the host cores, same metric."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = workload(args)
    nshot, threads, cores = oracle_plan(wl)
    vals = []
    for i in range(args.warmup + args.steps):
        val, dt, sample = oracle_sample(wl, ORACLE_NT, nshot, threads)
        if i >= args.warmup:
            vals.append((val, dt))
    value = statistics.mean(v for v, _ in vals)
    ms = statistics.mean(dt for _, dt in vals) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
            "config": config(wl, args, 1),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "host_cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm

def serving_section(nreq: int, rate: float, active: int = 16):
    """Serving mix: Poisson arrivals at `rate`/s of forward and FWIME-gradient shot requests on grids
    200-600 x 400-2000 at 10 m, nt 2000-6000, nh in {1, 11, 31}, served through libfwime's request
    server (memory admission, up to `active` requests in flight, one stream each, grouped forward
    launches); p50/p99 latency and shots/s, timed from the first submission (the requests' host
    buffers are pinned before).  A steady-state run offers the same mix at 0.7 x the measured
    throughput.  The plain comparison serves a subset of the same requests one at a time, one shot
    per launch, host-driven steps."""
    from paper_2206_02362_gb300 import serve
    reqs = [serve.from_synth(r) for r in synth.serving_mix(nreq=nreq, rate=rate)]
    srv = serve.Server(max_active=active)
    try:
        warm = [serve.from_synth(r) for r in synth.serving_mix(nreq=4, rate=rate, seed=synth.SEED0 + 99)]
        srv.serve(warm, realtime=False)
        res = srv.serve(reqs, realtime=True)
        s1 = serve.summarize(res, srv.last_wall)
        out = {"workload": f"serving mix, {nreq} requests, Poisson {rate}/s (overload: arrivals outpace the GPU)",
               "max_in_flight": active, **s1,
               "enqueue_share": s1["enqueue_s_total"] / (s1["span_s"] * min(12, active))}
        # steady state: the same mix arriving at 0.7x the throughput just measured
        rate2 = 0.7 * out["shots_per_s"]
        reqs2 = [serve.from_synth(r) for r in synth.serving_mix(nreq=max(20, nreq // 2), rate=rate2,
                                                                 seed=synth.SEED0 + 98)]
        res2 = srv.serve(reqs2, realtime=True)
        s2 = serve.summarize(res2, srv.last_wall)
        out["steady_state"] = {"rate_per_s": rate2, "requests": len(reqs2), "p50_s": s2["p50_s"],
                               "p99_s": s2["p99_s"], "shots_per_s": s2["shots_per_s"]}
    finally:
        srv.close()
    out["kinds"] = {k: sum(1 for r in reqs if r.kind == k) for k in ("forward", "gradient")}
    # plain: the same requests alone, one after the other, one shot per launch, on every 8th request of
    # the mix (a subset spread over it, so its forward/gradient and size mix is the mix's)
    sub = reqs[::8] if nreq >= 32 else reqs[: max(4, nreq // 8)]
    plain = serve.Server(max_active=1, plain=True)
    try:
        plain.serve(sub, realtime=False)
        tp = plain.last_wall
    finally:
        plain.close()
    out["plain_shots_per_s"] = len(sub) / tp
    out["plain_sample"] = f"{len(sub)} requests (every 8th of the mix) served alone, one shot per launch"
    out["served_vs_plain"] = out["shots_per_s"] / out["plain_shots_per_s"]
    return out


def time_lag_section(fw, torch, dev, wl, nh=21, lag=2):
    """B~ then B~* with the time-lag extension (nh lags spaced lag * dt) on the bench workload, all
    shots batched, one step: useful Gupd/s (4 propagations per step) and the extension kernels'
    share and GB/s."""
    grid = fw.Grid(nz=wl.nz, nx=wl.nx, sponge=wl.W, nt=wl.nt, dt=wl.dt, dx=wl.dx, nh=nh)
    geom = fw.Geometry(wl.src_iz, wl.src_ix, wl.rec_iz, wl.rec_ix)
    rng = np.random.default_rng(synth.SEED0 + 31)
    v = torch.from_numpy(wl.v).to(dev)
    w = torch.from_numpy(np.ascontiguousarray(np.broadcast_to(wl.w.astype(np.float32), (wl.nshot, wl.nt)))).to(dev)
    pt = torch.from_numpy(rng.standard_normal((nh, wl.nz, wl.nx)).astype(np.float32)).to(dev)
    d = torch.zeros((wl.nshot, wl.nt, wl.nrec), device=dev)
    img = torch.zeros((nh, wl.nz, wl.nx), device=dev)
    with fw.Context(grid, geom, profile=1, time_lag=lag) as c:
        c.autotune(fw.OP_BORN_EXT_ADJ)
        c.born_ext(v, w, pt, d)
        c.born_ext_adj(v, w, d, img)
        c.profile_read(reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        c.born_ext(v, w, pt, d, sync=False)
        c.born_ext_adj(v, w, d, img, sync=False)
        e1.record()
        c.sync()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        prof = c.profile_read(reset=True)
    kern = sum(p["ms"] for p in prof.values())
    return {"workload": f"{wl.name} with {nh} time lags every {lag} dt (+-{(nh - 1) // 2 * lag * wl.dt * 1e3:.1f} ms)",
            "ms_per_step": ms, "value": updates_per_step(wl) / (ms * 1e-3) / 1e9, "unit": "Gupd/s",
            "time_share": {k: round(p["ms"] / kern, 4) for k, p in prof.items()} if kern else None,
            "family_gbs": {k: round(p["bytes"] / (p["ms"] * 1e-3) / 1e9, 1) for k, p in prof.items() if p["ms"] > 0}}


def gradient_section(fw, torch, dev, nshot, tune=True, nt=0):
    """FWIME gradient (objective + B* r + T* r, checkpointed) on the North-Sea-shaped workload,
    400 x 1600 at 12.5 m, nt 5000, nh 31: all shots batched, the call captured once in a CUDA graph
    and replayed on its own stream (timed), vs the plain path (one shot per launch, host-driven steps)
    on 2 shots.  Shots/s of each and their ratio; kernel-family shares from one more call in profile
    mode (an event pair around every launch, no graph)."""
    wl, v0 = synth.north_sea(nshot=nshot, nt=nt) if nt > 0 else synth.north_sea(nshot=nshot)
    grid = fw.Grid(nz=wl.nz, nx=wl.nx, sponge=wl.W, nt=wl.nt, dt=wl.dt, dx=wl.dx, nh=wl.nh)
    rng = np.random.default_rng(synth.SEED0 + 21)
    v = torch.from_numpy(v0).to(dev)
    w = torch.from_numpy(np.ascontiguousarray(np.broadcast_to(wl.w.astype(np.float32), (wl.nshot, wl.nt)))).to(dev)
    pt = torch.from_numpy((1e-3 * rng.standard_normal((wl.nh, wl.nz, wl.nx))).astype(np.float32)).to(dev)
    dobs = torch.from_numpy((1e-3 * rng.standard_normal((wl.nshot, wl.nt, wl.nrec))).astype(np.float32)).to(dev)
    g = torch.zeros((wl.nz, wl.nx), device=dev)
    geom = fw.Geometry(wl.src_iz, wl.src_ix, wl.rec_iz, wl.rec_ix)
    out = {"workload": wl.name, "nshot": wl.nshot, "segment": "auto"}
    stream = torch.cuda.Stream(device=dev)
    with fw.Context(grid, geom, stream=stream, graph=1) as c:
        if tune:                                              # segment x shots per launch x chunking (untimed)
            out["autotune"] = c.autotune_schedule(fw.OP_GRADIENT)
        c.gradient(v, w, pt, dobs, g, eps=1e-3)              # warm-up: workspace, capture, first replay
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("gradient")   # lets ncu --nvtx-include select the timed replay
        e0.record(stream)
        J = c.gradient(v, w, pt, dobs, g, eps=1e-3, sync=False)
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        c.sync()
        tb = e0.elapsed_time(e1) * 1e-3
        out["batched_shots_per_s"] = wl.nshot / tb
        out["batched_seconds"] = tb
        out["launches"] = c.launches
        out["shots_per_batch"] = c.get_option("batch_used")
        out["graph_replay"] = True
        c.set_option("graph", 0)
        c.set_option("profile", 1)
        c.gradient(v, w, pt, dobs, g, eps=1e-3)
        prof = c.profile_read(reset=True)
        kms = sum(p["ms"] for p in prof.values())
        out["time_share"] = {k: round(p["ms"] / kms, 4) for k, p in prof.items()} if kms else None
        out["family_gbs"] = {k: round(p["bytes"] / (p["ms"] * 1e-3) / 1e9, 1) for k, p in prof.items() if p["ms"] > 0}
        out["profiled_seconds"] = kms * 1e-3
    nps = 2
    geom2 = fw.Geometry(wl.src_iz[:nps], wl.src_ix[:nps], wl.rec_iz, wl.rec_ix)
    with fw.Context(grid, geom2, plain=1) as c:
        w2, d2 = w[:nps].contiguous(), dobs[:nps].contiguous()
        c.gradient(v, w2, pt, d2, g, eps=1e-3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c.gradient(v, w2, pt, d2, g, eps=1e-3)
        tp = time.perf_counter() - t0
        out["plain_shots_per_s"] = nps / tp
    out["batched_vs_plain"] = out["batched_shots_per_s"] / out["plain_shots_per_s"]
    NZ, NX = wl.padded
    out["useful_gupd_s"] = 6.0 * wl.nshot * NZ * NX * (wl.nt - 1) / tb / 1e9   # 6 propagations (Eq. 11)
    out["objective"] = J
    return out


def salt_section(fw, torch, dev, nshot):
    """The batched FWIME gradient on the Salt-shaped workload (1200 x 5000 at 6.25 m, nt 8000,
    dt 0.5 ms, nh 41), where one shot's source-wavefield history (~214 GB padded) exceeds HBM, so the
    adjoint sweep recomputes every segment from its checkpoints: a subset of `nshot` shots in one
    batch, timed in profile mode (shares and GB/s of each kernel family) after a warm-up call."""
    wl = synth.salt(nshot=nshot)
    grid = fw.Grid(nz=wl.nz, nx=wl.nx, sponge=wl.W, nt=wl.nt, dt=wl.dt, dx=wl.dx, nh=wl.nh)
    rng = np.random.default_rng(synth.SEED0 + 41)
    NZ, NX = wl.padded
    v = torch.from_numpy(wl.v).to(dev)
    # a smooth initial model: the true one with its salt body and feeder stem removed (sediment trend)
    v0 = torch.from_numpy(np.where(wl.v == 4500.0, np.float32(3000.0), wl.v)).to(dev)
    w = torch.from_numpy(np.ascontiguousarray(np.broadcast_to(wl.w.astype(np.float32), (wl.nshot, wl.nt)))).to(dev)
    pt = torch.from_numpy((1e-3 * rng.standard_normal((wl.nh, wl.nz, wl.nx))).astype(np.float32)).to(dev)
    geom = fw.Geometry(wl.src_iz, wl.src_ix, wl.rec_iz, wl.rec_ix)
    dobs = torch.zeros((wl.nshot, wl.nt, wl.nrec), device=dev)
    g = torch.zeros((wl.nz, wl.nx), device=dev)
    out = {"workload": wl.name + f" (subset: {wl.nshot} of 400 shots)", "nshot": wl.nshot, "nt": wl.nt,
           "nh": wl.nh, "history_gb_per_shot": round(4.0 * NZ * NX * wl.nt / 1e9, 1)}
    with fw.Context(grid, geom, profile=1) as c:
        c.forward(v, w, dobs)                                   # observed data of the salt model
        c.gradient(v0, w, pt, dobs, g, eps=1e-3)                # warm-up (workspace)
        c.profile_read(reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        c.gradient(v0, w, pt, dobs, g, eps=1e-3, sync=False)
        e1.record()
        c.sync()
        t = e0.elapsed_time(e1) * 1e-3
        prof = c.profile_read(reset=True)
        out["segment"] = "auto"
        out["workspace_gb"] = round(c.get_option("workspace") / 1e9, 1)
    kms = sum(p["ms"] for p in prof.values())
    out["seconds"] = t
    out["shots_per_s"] = wl.nshot / t
    out["useful_gupd_s"] = 6.0 * wl.nshot * NZ * NX * (wl.nt - 1) / t / 1e9
    out["time_share"] = {k: round(p["ms"] / kms, 4) for k, p in prof.items()} if kms else None
    out["family_gbs"] = {k: round(p["bytes"] / (p["ms"] * 1e-3) / 1e9, 1) for k, p in prof.items() if p["ms"] > 0}
    return out


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def ncu_traffic():
    """Per-launch DRAM bytes of the stencil kernel from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    src = os.path.join(ROOT, "paper_2206_02362_gb300", "csrc", "k_prop.cu")
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    path = os.path.join(ROOT, "profiles", "k_prop_marmousi2_ncu.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"k_prop\.cu sha256\[:16\]:\s*([0-9a-f]{16})", txt)
    t = re.search(r"dram bytes per full-size launch:\s*([0-9.eE+]+)", txt)
    a = re.search(r"algorithmic bytes of that variant per full-size launch:\s*([0-9.eE+]+)", txt)
    if not m or not t or m.group(1) != h:
        return None
    return {"dram_bytes_per_launch": float(t.group(1)),
            "algorithmic_bytes_per_launch": float(a.group(1)) if a else None,
            "captured": "every k_prop launch of one timed bench step (full-size launches: 100 shots, nt 40), 1-pass ncu",
            "source": "profiles/k_prop_marmousi2_ncu.md"}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    import paper_2206_02362_gb300 as fw
    from paper_2206_02362_gb300.shard import rank_step

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    wl = workload(args)
    grid = fw.Grid(nz=wl.nz, nx=wl.nx, sponge=wl.W, nt=wl.nt, dt=wl.dt, dx=wl.dx, nh=wl.nh)
    geom = fw.Geometry(wl.src_iz, wl.src_ix, wl.rec_iz, wl.rec_ix)
    rng = np.random.default_rng(synth.SEED0 + 11 + rank)
    pt_h = rng.standard_normal((wl.nh, wl.nz, wl.nx)).astype(np.float32)
    w_h = np.ascontiguousarray(np.broadcast_to(wl.w.astype(np.float32), (wl.nshot, wl.nt)))
    dev = torch.device("cuda", local)
    v = torch.from_numpy(wl.v).to(dev)
    w = torch.from_numpy(w_h).to(dev)
    pt = torch.from_numpy(pt_h).to(dev)
    d = torch.zeros((wl.nshot, wl.nt, wl.nrec), device=dev)
    img = torch.zeros((wl.nh, wl.nz, wl.nx), device=dev)
    reuse = 0 if args.no_reuse else 1
    ctx = fw.Context(grid, geom, profile=1, segment=args.segment, reuse_background=reuse)
    tuned = None
    if not args.no_tune:
        if args.tune == "schedule":   # segment x shots per launch x chunking, timed on this GPU (untimed here)
            tuned = ctx.autotune_schedule(fw.OP_BORN_EXT_ADJ)
        else:                         # stencil chunking only
            zc, us = ctx.autotune(fw.OP_BORN_EXT_ADJ)
            tuned = {"zchunk": zc, "us_stencil": us}
    launches = [0]

    reused = [0]

    def step(c, vv, ww, pp, dd, ii, ranks=world):
        # weak scaling: wl.nshot shots per rank; shard.rank_step hands this rank its block of the
        # ranks x wl.nshot shots (the context's own shots) and sums the images over all ranks
        def apply(a, b):
            assert b - a == c.geom.nshot
            c.born_ext(vv, ww, pp, dd, sync=False)
            n = c.launches
            c.born_ext_adj(vv, ww, dd, ii, sync=False)
            reused[0] = c.get_option("background_reused")
            launches[0] += n + c.launches
            return ii
        rank_step(apply, c.geom.nshot * ranks, ranks, rank if ranks > 1 else 0)

    for _ in range(args.warmup):
        step(ctx, v, w, pt, d, img)
        ctx.sync()
    ctx.profile_read(reset=True)
    launches[0] = 0
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clk = Clocks(uuid)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")     # lets ncu --nvtx-include select the timed launches
    e0.record()
    for _ in range(args.steps):
        step(ctx, v, w, pt, d, img)
    e1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ctx.sync()
    clocks = clk.stop()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_step = ms / args.steps
    value = updates_per_step(wl) * world / (ms_step * 1e-3) / 1e9
    prof = ctx.profile_read(reset=True)
    kern_ms = sum(p["ms"] for p in prof.values())
    pk = prof["prop"]
    peak, peak_kind = peaks()
    achieved = pk["bytes"] / (pk["ms"] * 1e-3) / 1e9 if pk["ms"] > 0 else None
    traffic = ncu_traffic()
    roofline = {"bound": "hbm", "kernel": "k_prop (wave-equation time step, forward and adjoint)",
                "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)",
                "traffic": traffic["dram_bytes_per_launch"] if traffic else None,
                "traffic_source": traffic,
                "launches": pk["launches"], "avg_launch_us": 1e3 * pk["ms"] / max(pk["launches"], 1),
                "algorithmic_bytes_per_launch": pk["bytes"] / max(pk["launches"], 1),
                "time_share": {k: round(p["ms"] / kern_ms, 4) for k, p in prof.items()} if kern_ms else None,
                "family_gbs": {k: round(p["bytes"] / (p["ms"] * 1e-3) / 1e9, 1) for k, p in prof.items()
                               if p["ms"] > 0},
                "bytes_rule": "12 B per shot-point (q^n, q^n-1 in, q^n+1 out) over the padded NZ x NX points "
                              "+ 4 B per grid point per launch for c (shared by all shots) + 4 B per shot-point "
                              "per D2t or local-source field over the physical rows (nz x NX points)"}
    shots_per_s = wl.nshot * world / (ms_step * 1e-3)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded Marmousi2-shaped stand-in)",
            "config": config(wl, args, world), "roofline": roofline, "gpu_launches": launches[0],
            "clocks": clocks, "shots_per_s": shots_per_s,
            "autotune": tuned,
            "executed_gupd_s": value * (4.0 if reused[0] else 5.0) / 4.0,
            "background_reuse": {"used": bool(reused[0]),
                                 "note": "B~* starts from the background states kept by the B~ of the same step "
                                         "(4 propagations per step instead of 5); --no-reuse disables it"}}

    # the same step without the background reuse (B~* with its own checkpointing sweep), one step
    if reuse and world == 1:
        ctx.set_option("reuse_background", 0)
        step(ctx, v, w, pt, d, img)
        ctx.sync()
        torch.cuda.synchronize()
        e0.record()
        step(ctx, v, w, pt, d, img)
        e1.record()
        ctx.sync()
        torch.cuda.synchronize()
        ms_nr = e0.elapsed_time(e1)
        line["no_reuse"] = {"ms_per_step": ms_nr, "value": updates_per_step(wl) / (ms_nr * 1e-3) / 1e9,
                            "unit": UNIT, "steps": 1}
        ctx.set_option("reuse_background", 1)
        ctx.profile_read(reset=True)

    # plain path: one shot per launch, host-driven steps, same per-shot work
    if not args.no_plain and rank == 0:
        nps = 2
        geom2 = fw.Geometry(wl.src_iz[:nps], wl.src_ix[:nps], wl.rec_iz, wl.rec_ix)
        with fw.Context(grid, geom2, plain=1, reuse_background=reuse) as cp:
            d2 = torch.zeros((nps, wl.nt, wl.nrec), device=dev)
            step(cp, v, w[:nps].contiguous(), pt, d2, img, ranks=1)
            cp.sync()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            step(cp, v, w[:nps].contiguous(), pt, d2, img, ranks=1)
            cp.sync()
            tp = time.perf_counter() - t0
        line["plain"] = {"shots_per_s": nps / tp, "sample": f"{nps} shots, one shot per launch, no graph"}
        line["batched_vs_plain"] = shots_per_s / world / (nps / tp)

    # end to end through the C ABI with host buffers (copies inside the timed region)
    if not args.no_e2e:
        ctx.set_option("profile", 0)
        ctx.set_option("host_io", 1)
        vh = torch.from_numpy(wl.v).pin_memory()
        wh = torch.from_numpy(w_h).pin_memory()
        ph = torch.from_numpy(pt_h).pin_memory()
        dh = torch.zeros((wl.nshot, wl.nt, wl.nrec)).pin_memory()
        ih = torch.zeros((wl.nh, wl.nz, wl.nx)).pin_memory()
        arr = lambda t: t.numpy()  # noqa: E731
        ctx.born_ext(arr(vh), arr(wh), arr(ph), arr(dh))     # warm (staging allocation)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ne = 3
        for _ in range(ne):
            ctx.born_ext(arr(vh), arr(wh), arr(ph), arr(dh))
            ctx.born_ext_adj(arr(vh), arr(wh), arr(dh), arr(ih))
        te = (time.perf_counter() - t0) / ne
        nb = 4
        h2d = 2 * (wl.v.nbytes + w_h.nbytes) + pt_h.nbytes + dh.numel() * nb
        d2h = dh.numel() * nb + ih.numel() * nb
        line["e2e"] = {"value": updates_per_step(wl) / te / 1e9, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                       "d2h_bytes_per_step": int(d2h), "seconds_per_step": te}
        ctx.set_option("host_io", 0)

    if not args.no_cpu and rank == 0 and world == 1:
        line["cpu_baseline"] = cpu_baseline(wl)
    ctx.close()
    del d, img, pt, w, v
    torch.cuda.empty_cache()
    # FWIME gradient (Eqs. 7-9) on the North-Sea-shaped workload: batched vs plain shots/s
    if not args.no_grad and rank == 0:
        line["gradient"] = gradient_section(fw, torch, dev, args.grad_shots,
                                            tune=not args.no_tune and args.tune == "schedule", nt=args.grad_nt)
    if not args.no_tlag and rank == 0 and world == 1:
        line["time_lag"] = time_lag_section(fw, torch, dev, wl)
    # Salt-shaped batched gradient with checkpoint/recompute (a shot subset)
    if not args.no_salt and rank == 0 and world == 1:
        line["salt"] = salt_section(fw, torch, dev, args.salt_shots)
    # serving mix: continuous batching with memory admission, p50/p99 (Poisson arrivals)
    if not args.no_serve and rank == 0:
        line["serving"] = serving_section(args.serve_requests, args.serve_rate, args.serve_active)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
