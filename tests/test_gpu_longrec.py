"""Parity with the FP64 oracle at the workloads' full record lengths.

FP32 leapfrog error grows with the number of time steps, and the imaging
conditions and the gradient are FP32 reductions over nt terms (Theory section,
Eqs. 2-9), so a check at a few hundred steps says little about nt = 4000-8000.
These tests run the operators at the real nt, dt, spacing, sponge, velocity
range and nh of three workloads, on grids cropped (rows from the top of the
model and from its fastest part, stacked, so the crop keeps the full velocity
range) until the FP64 oracle finishes in minutes:

* Marmousi2-shaped: 110 x 300 at 10 m, nt 4000, dt 0.8 ms, nh 21, 2 shots,
  8 Hz low-cut Ricker; B~ (traces) and B~* (image, also offset plane by offset
  plane) in the benchmark's configuration (batched, automatic segment,
  B~* starting from the background states kept by B~).
* North-Sea-shaped: 60 x 160 at 12.5 m, nt 5000, dt 1 ms, nh 31, 2 shots; the
  FWIME objective and gradient at the 1-D initial model against data of the
  layered model with its chalk layer, and T* of those data.
* Salt-shaped: 60 x 160 at 6.25 m, nt 8000, dt 0.5 ms, nh 41, 10 Hz; B~* with
  segments of 50 steps (every segment recomputed from its checkpoint), and the
  gradient of one shot.

Bars: rel. L2 <= 1e-4 on traces, images (also per offset plane) and gradients; the
objective within the change that a 1e-4 relative error on the predicted traces can
make to it (``objective_bound``).
The oracle's jobs start on host threads when the module's fixture is first
used (ctypes releases the GIL, OpenMP runs each job's shots in parallel) and
run while the GPU computes; jobs are admitted by an estimate of their FP64
history memory against the host's available memory.
"""
import concurrent.futures as cf
import threading

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_2206_02362_gb300 as fw  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-4


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def f32(a):
    """The values the GPU sees, in float64 for the oracle."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


# ------------------------------------------------------------------ crops

def marmousi_crop():
    """Rows 0-59 (water and the first layers) over rows 300-349 (the fastest layers) of the
    Marmousi2-shaped model, columns 700-999: 110 x 300, 1.5-4.7 km/s."""
    v = synth.marmousi_like()
    return np.concatenate([v[:60, 700:1000], v[300:350, 700:1000]], axis=0)


def north_sea_crop():
    """True model: rows 0-29 over the 30 rows around the chalk layer; initial model: the 1-D trend
    at the same rows (60 x 160 at 12.5 m)."""
    vt, v0 = synth.north_sea_like()
    ch = int(np.where(vt[:, 0] == 4500.0)[0][0])
    rows = np.r_[0:30, ch - 10:ch + 20]
    return vt[rows, 600:760], v0[rows, 600:760]


def salt_crop():
    """Rows 0-19 (water) over 40 rows across the rugose salt top, 160 columns over the feeder stem
    (60 x 160 at 6.25 m, 1.5-4.5 km/s)."""
    v = synth.salt_like()
    col = int(np.argmax((v == 4500.0).sum(axis=0)))
    top = int(np.argmax(v[:, col] == 4500.0))
    rows = np.r_[0:20, top - 20:top + 20]
    return v[rows, col - 80:col + 80]


def spread(nx, nshot):
    """Sources at depth index 2, evenly inside the crop; receivers every 2 points at depth 2."""
    src_ix = np.round(np.linspace(0.2, 0.8, nshot) * (nx - 1)).astype(int)
    rec_ix = 2 * np.arange(nx // 2)
    return np.full(nshot, 2), src_ix, np.full(len(rec_ix), 2), rec_ix


# ------------------------------------------------------------------ oracle jobs

class OracleJobs:
    """Runs oracle calls on host threads, admitted by estimated memory."""

    def __init__(self):
        avail = None
        try:
            for ln in open("/proc/meminfo"):
                if ln.startswith("MemAvailable:"):
                    avail = int(ln.split()[1]) * 1024
        except OSError:
            pass
        self.budget = 0.6 * (avail or 32 << 30)
        self.used = 0.0
        self.cv = threading.Condition()
        self.pool = cf.ThreadPoolExecutor(max_workers=8)

    def submit(self, est_bytes, fn, *args, **kw):
        est = min(float(est_bytes), self.budget)

        def run():
            with self.cv:
                self.cv.wait_for(lambda: self.used + est <= self.budget or self.used == 0.0)
                self.used += est
            try:
                return fn(*args, **kw)
            finally:
                with self.cv:
                    self.used -= est
                    self.cv.notify_all()

        return self.pool.submit(run)


def hist_bytes(g, nshot, fields):
    """FP64 bytes of `fields` full time histories of one padded field per shot."""
    return 8.0 * fields * nshot * g.nt * g.NZ * g.NX


@pytest.fixture(scope="module")
def cases():
    jobs = OracleJobs()
    out = {}

    # Marmousi2-shaped
    v = marmousi_crop()
    nz, nx = v.shape
    nt, dt, dx, nh = 4000, 8e-4, 10.0, 21
    siz, six, riz, rix = spread(nx, 2)
    w = synth.lowcut(synth.ricker(nt, dt, 8.0), dt, 2.0, 4.0)
    rng = np.random.default_rng(synth.SEED0 + 700)
    pt = rng.standard_normal((nh, nz, nx))
    og = oracle.Grid(nz=nz, nx=nx, W=50, nt=nt, dt=dt, dx=dx, nh=nh)
    geo = oracle.Geometry(siz, six, riz, rix)
    W2 = np.stack([f32(w)] * 2)
    d_obs = oracle.forward(og, f32(v), geo, W2)          # data for B~* (a few seconds)
    m = dict(v=v, w=W2, pt=pt, d_in=f32(d_obs), grid=(nz, nx, 50, nt, dt, dx, nh), geom=(siz, six, riz, rix))
    m["born_ext"] = jobs.submit(hist_bytes(og, 2, 4), oracle.born_ext, og, f32(v), geo, W2, f32(pt))
    m["born_ext_adj"] = jobs.submit(hist_bytes(og, 2, 4), oracle.born_ext_adj, og, f32(v), geo, W2, m["d_in"])
    out["marmousi"] = m

    # North-Sea-shaped
    vt, v0 = north_sea_crop()
    nz, nx = vt.shape
    nt, dt, dx, nh = 5000, 1e-3, 12.5, 31
    siz, six, riz, rix = spread(nx, 2)
    w = synth.ricker(nt, dt, 8.0)
    rng = np.random.default_rng(synth.SEED0 + 701)
    pt = 1e-4 * rng.standard_normal((nh, nz, nx))
    og = oracle.Grid(nz=nz, nx=nx, W=50, nt=nt, dt=dt, dx=dx, nh=nh)
    geo = oracle.Geometry(siz, six, riz, rix)
    W2 = np.stack([f32(w)] * 2)
    d_obs = f32(oracle.forward(og, f32(vt), geo, W2))
    n = dict(v=v0, w=W2, pt=pt, d_in=d_obs, grid=(nz, nx, 50, nt, dt, dx, nh), geom=(siz, six, riz, rix), eps=1e-3)
    n["gradient"] = jobs.submit(hist_bytes(og, 2, 11), oracle.gradient, og, f32(v0), geo, W2, f32(pt), d_obs, 1e-3)
    n["tomo_adj"] = jobs.submit(hist_bytes(og, 2, 10), oracle.tomo_adj, og, f32(v0), geo, W2, f32(pt), d_obs)
    out["north_sea"] = n

    # Salt-shaped
    v = salt_crop()
    nz, nx = v.shape
    nt, dt, dx, nh = 8000, 5e-4, 6.25, 41
    siz, six, riz, rix = spread(nx, 2)
    w = synth.ricker(nt, dt, 10.0)
    rng = np.random.default_rng(synth.SEED0 + 702)
    og = oracle.Grid(nz=nz, nx=nx, W=50, nt=nt, dt=dt, dx=dx, nh=nh)
    geo = oracle.Geometry(siz, six, riz, rix)
    W2 = np.stack([f32(w)] * 2)
    d_in = f32(oracle.forward(og, f32(v), geo, W2))
    pt = 1e-4 * rng.standard_normal((nh, nz, nx))
    s = dict(v=v, w=W2, pt=pt, d_in=d_in, grid=(nz, nx, 50, nt, dt, dx, nh), geom=(siz, six, riz, rix), eps=1e-3)
    s["born_ext_adj"] = jobs.submit(hist_bytes(og, 2, 4), oracle.born_ext_adj, og, f32(v), geo, W2, d_in)
    geo1 = oracle.Geometry(siz[:1], six[:1], riz, rix)
    dobs1 = np.ascontiguousarray(0.5 * d_in[:1])           # data of a model the crop does not match
    s["dobs1"] = dobs1
    s["gradient1"] = jobs.submit(hist_bytes(og, 1, 11), oracle.gradient, og, f32(v), geo1, W2[:1], f32(pt), dobs1,
                                 1e-3)
    out["salt"] = s
    yield out
    jobs.pool.shutdown(wait=True)


def fw_setup(c, nshot=None, **opts):
    nz, nx, W, nt, dt, dx, nh = c["grid"]
    siz, six, riz, rix = c["geom"]
    if nshot is not None:
        siz, six = siz[:nshot], six[:nshot]
    grid = fw.Grid(nz=nz, nx=nx, sponge=W, nt=nt, dt=dt, dx=dx, nh=nh)
    return fw.Context(grid, fw.Geometry(siz, six, riz, rix), **opts), grid


def plane_errors(img, ref):
    return [rel(img[i], ref[i]) for i in range(ref.shape[0])]


def objective_bound(c, J_ref, dobs, nshot=None):
    """Largest |Phi_gpu - Phi_oracle| the trace contract allows: Phi = 1/2 ||r||^2 + (DSO term), r = pred -
    d_obs, and a relative error of at most TOL on the predicted traces moves ||r|| by at most
    TOL ||pred|| <= TOL (||r|| + ||d_obs||), hence Phi by at most ||r|| TOL (||r|| + ||d_obs||) to first order."""
    nz, nx, W, nt, dt, dx, nh = c["grid"]
    og = oracle.Grid(nz=nz, nx=nx, W=W, nt=nt, dt=dt, dx=dx, nh=nh)
    r = np.sqrt(2.0 * (J_ref - oracle.dso_penalty(og, f32(c["pt"]), c["eps"])))
    return TOL * r * (r + np.linalg.norm(dobs))


def test_marmousi2_full_record_born_ext_and_adjoint(cases):
    c = cases["marmousi"]
    ctx, g = fw_setup(c, reuse_background=1)
    d = torch.zeros((2, g.nt, len(c["geom"][2])), device="cuda")
    img = torch.zeros((g.nh, g.nz, g.nx), device="cuda")
    with ctx:
        v, w = cu(c["v"]), cu(c["w"])
        ctx.born_ext(v, w, cu(c["pt"]), d)
        ctx.born_ext_adj(v, w, cu(c["d_in"]), img)
        assert ctx.get_option("background_reused") == 1
    d_ref = c["born_ext"].result()
    i_ref = c["born_ext_adj"].result()
    e_d = rel(d.double().cpu().numpy(), d_ref)
    ig = img.double().cpu().numpy()
    e_i = rel(ig, i_ref)
    planes = plane_errors(ig, i_ref)
    print(f"marmousi2 nt 4000: B~ traces {e_d:.3e}, B~* image {e_i:.3e}, worst plane {max(planes):.3e}")
    assert e_d <= TOL
    assert e_i <= TOL
    assert max(planes) <= TOL, planes


def test_north_sea_full_record_gradient(cases):
    c = cases["north_sea"]
    ctx, g = fw_setup(c)
    grad = torch.zeros((g.nz, g.nx), device="cuda")
    with ctx:
        J = ctx.gradient(cu(c["v"]), cu(c["w"]), cu(c["pt"]), cu(c["d_in"]), grad, eps=c["eps"])
    J_ref, g_ref = c["gradient"].result()
    e_g = rel(grad.double().cpu().numpy(), g_ref)
    print(f"north sea nt 5000: objective {abs(J - J_ref) / abs(J_ref):.3e}, gradient {e_g:.3e}")
    assert abs(J - J_ref) <= objective_bound(c, J_ref, c["d_in"])
    assert e_g <= TOL


def test_north_sea_full_record_tomo_adj(cases):
    c = cases["north_sea"]
    ctx, g = fw_setup(c)
    out = torch.zeros((g.nz, g.nx), device="cuda")
    with ctx:
        ctx.tomo_adj(cu(c["v"]), cu(c["w"]), cu(c["pt"]), cu(c["d_in"]), out)
    ref = c["tomo_adj"].result()
    e = rel(out.double().cpu().numpy(), ref)
    print(f"north sea nt 5000: T* {e:.3e}")
    assert e <= TOL


def test_salt_full_record_born_ext_adj_recomputed_segments(cases):
    c = cases["salt"]
    ctx, g = fw_setup(c, segment=50)
    img = torch.zeros((g.nh, g.nz, g.nx), device="cuda")
    with ctx:
        ctx.born_ext_adj(cu(c["v"]), cu(c["w"]), cu(c["d_in"]), img)
    ref = c["born_ext_adj"].result()
    ig = img.double().cpu().numpy()
    e = rel(ig, ref)
    planes = plane_errors(ig, ref)
    print(f"salt nt 8000: B~* image {e:.3e}, worst plane {max(planes):.3e}")
    assert e <= TOL
    assert max(planes) <= TOL, planes


def test_salt_full_record_gradient(cases):
    c = cases["salt"]
    ctx, g = fw_setup(c, nshot=1, segment=50)
    grad = torch.zeros((g.nz, g.nx), device="cuda")
    with ctx:
        J = ctx.gradient(cu(c["v"]), cu(c["w"][:1]), cu(c["pt"]), cu(c["dobs1"]), grad, eps=c["eps"])
    J_ref, g_ref = c["gradient1"].result()
    e_g = rel(grad.double().cpu().numpy(), g_ref)
    print(f"salt nt 8000: objective {abs(J - J_ref) / abs(J_ref):.3e}, gradient {e_g:.3e}")
    assert abs(J - J_ref) <= objective_bound(c, J_ref, c["dobs1"])
    assert e_g <= TOL
