"""GPU parity: every operator of libfwime (FP32, sm_103a) against the FP64 oracle,
element by element, at sizes the oracle finishes in seconds that span several
stencil strips/chunks with ragged tails, ragged time segments and ragged shot
batches.  Tolerances: relative L2 <= 1e-4 on traces and images, dot-product
tests <= 1e-5 (FP32 path, FP64 inner products)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_2206_02362_gb300 as fw  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-4
DOT_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    fw.load()


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64); b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32))).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


class Case:
    """A small seeded problem: 37 x 300 physical (3 ragged 128-point strips), W=10,
    nt=250 (249 steps: ragged segments), 3 shots (ragged batches of 2)."""

    def __init__(self, nz=37, nx=300, W=10, nt=250, nh=5, nshot=3, seed=0, f0=20.0):
        rng = np.random.default_rng(synth.SEED0 + 100 + seed)
        self.nz, self.nx, self.W, self.nt, self.nh = nz, nx, W, nt, nh
        self.dx, self.dt = 10.0, 1e-3
        z = np.arange(nz)[:, None]; x = np.arange(nx)[None, :]
        self.v = (1800.0 + 20.0 * z + 150.0 * np.sin(x / 17.0) * np.cos(z / 5.0)).astype(np.float32)
        self.src_iz = np.array([0, 3, 1][:nshot] + [2] * max(0, nshot - 3))
        self.src_ix = np.linspace(0, nx - 1, nshot).astype(int)
        self.rec_iz = np.concatenate([np.full(nx // 3, 0), [nz - 1, nz // 2]])
        self.rec_ix = np.concatenate([3 * np.arange(nx // 3), [nx - 1, 0]])
        w = synth.ricker(nt, self.dt, f0)
        self.w = np.stack([w * (1.0 + 0.1 * s) for s in range(nshot)]).astype(np.float32)
        self.dv = synth.gaussian_blobs(nz, nx, rng, amp=50.0, sigma_pts=4.0, ring=1).astype(np.float32)
        self.pt = rng.standard_normal((nh, nz, nx)).astype(np.float32)
        self.d = rng.standard_normal((nshot, nt, len(self.rec_iz))).astype(np.float32)
        self.og = oracle.Grid(nz=nz, nx=nx, W=W, nt=nt, dt=self.dt, dx=self.dx, nh=nh)
        self.ogeo = oracle.Geometry(self.src_iz, self.src_ix, self.rec_iz, self.rec_ix)
        self.fg = fw.Grid(nz=nz, nx=nx, sponge=W, nt=nt, dt=self.dt, dx=self.dx, nh=nh)
        self.fgeo = fw.Geometry(self.src_iz, self.src_ix, self.rec_iz, self.rec_ix)

    @property
    def nshot(self):
        return len(self.src_iz)

    @property
    def nrec(self):
        return len(self.rec_iz)

    def ctx(self, **opt):
        return fw.Context(self.fg, self.fgeo, **opt)

    def dshape(self):
        return (self.nshot, self.nt, self.nrec)

    # --- GPU calls returning float64 host arrays
    def g_forward(self, c):
        d = torch.zeros(self.dshape(), device="cuda")
        c.forward(dev(self.v), dev(self.w), d)
        return host(d)

    def g_born(self, c, dv=None):
        d = torch.zeros(self.dshape(), device="cuda")
        c.born(dev(self.v), dev(self.w), dev(self.dv if dv is None else dv), d)
        return host(d)

    def g_born_adj(self, c, d=None):
        out = torch.zeros((self.nz, self.nx), device="cuda")
        c.born_adj(dev(self.v), dev(self.w), dev(self.d if d is None else d), out)
        return host(out)

    def g_ext(self, c, pt=None):
        d = torch.zeros(self.dshape(), device="cuda")
        c.born_ext(dev(self.v), dev(self.w), dev(self.pt if pt is None else pt), d)
        return host(d)

    def g_ext_adj(self, c, d=None):
        out = torch.zeros((self.nh, self.nz, self.nx), device="cuda")
        c.born_ext_adj(dev(self.v), dev(self.w), dev(self.d if d is None else d), out)
        return host(out)

    def g_tomo(self, c):
        d = torch.zeros(self.dshape(), device="cuda")
        c.tomo(dev(self.v), dev(self.w), dev(self.pt), dev(self.dv), d)
        return host(d)

    def g_tomo_adj(self, c, d=None):
        out = torch.zeros((self.nz, self.nx), device="cuda")
        c.tomo_adj(dev(self.v), dev(self.w), dev(self.pt), dev(self.d if d is None else d), out)
        return host(out)


@pytest.fixture(scope="module")
def case():
    return Case()


@pytest.fixture(scope="module")
def ref(case):
    """Oracle results (FP64) on the same float32 inputs."""
    c = case
    v, w = c.v.astype(np.float64), c.w.astype(np.float64)
    out = {}
    out["forward"] = oracle.forward(c.og, v, c.ogeo, w)
    out["born"] = oracle.born(c.og, v, c.ogeo, w, c.dv.astype(np.float64))
    out["born_adj"] = oracle.born_adj(c.og, v, c.ogeo, w, c.d.astype(np.float64))
    out["ext"] = oracle.born_ext(c.og, v, c.ogeo, w, c.pt.astype(np.float64))
    out["ext_adj"] = oracle.born_ext_adj(c.og, v, c.ogeo, w, c.d.astype(np.float64))
    out["tomo"] = oracle.tomo(c.og, v, c.ogeo, w, c.pt.astype(np.float64), c.dv.astype(np.float64))
    out["tomo_adj"] = oracle.tomo_adj(c.og, v, c.ogeo, w, c.pt.astype(np.float64), c.d.astype(np.float64))
    return out


# ----------------------------------------------------------------- parity

@pytest.mark.parametrize("opts", [dict(), dict(shots_per_batch=2, segment=16), dict(plain=1, segment=37)])
def test_forward_parity(case, ref, opts):
    with case.ctx(**opts) as c:
        d = case.g_forward(c)
    assert rel_l2(d, ref["forward"]) <= TOL
    assert np.all(d[:, 0, :] == 0.0)


@pytest.mark.parametrize("opts", [dict(), dict(shots_per_batch=2)])
def test_born_parity(case, ref, opts):
    with case.ctx(**opts) as c:
        assert rel_l2(case.g_born(c), ref["born"]) <= TOL


@pytest.mark.parametrize("opts", [dict(), dict(shots_per_batch=2, segment=16), dict(plain=1, segment=50)])
def test_born_adj_parity(case, ref, opts):
    with case.ctx(**opts) as c:
        assert rel_l2(case.g_born_adj(c), ref["born_adj"]) <= TOL


@pytest.mark.parametrize("opts", [dict(), dict(shots_per_batch=2, segment=16), dict(plain=1, segment=7)])
def test_born_ext_parity(case, ref, opts):
    with case.ctx(**opts) as c:
        assert rel_l2(case.g_ext(c), ref["ext"]) <= TOL


@pytest.mark.parametrize("opts", [dict(), dict(shots_per_batch=2, segment=16), dict(plain=1, segment=60)])
def test_born_ext_adj_parity(case, ref, opts):
    with case.ctx(**opts) as c:
        img = case.g_ext_adj(c)
    assert rel_l2(img, ref["ext_adj"]) <= TOL
    for ih in range(case.nh):       # every offset plane on its own
        assert rel_l2(img[ih], ref["ext_adj"][ih]) <= TOL


@pytest.mark.parametrize("opts", [dict(), dict(shots_per_batch=2, segment=16)])
def test_tomo_parity(case, ref, opts):
    with case.ctx(**opts) as c:
        assert rel_l2(case.g_tomo(c), ref["tomo"]) <= TOL


@pytest.mark.parametrize("opts", [dict(), dict(shots_per_batch=2, segment=16), dict(plain=1, segment=23)])
def test_tomo_adj_parity(case, ref, opts):
    with case.ctx(**opts) as c:
        assert rel_l2(case.g_tomo_adj(c), ref["tomo_adj"]) <= TOL


@pytest.mark.parametrize("opts", [dict(), dict(shots_per_batch=2, segment=16)])
def test_gradient_parity(case, opts):
    c = case
    dobs = (c.d * 0.05).astype(np.float32)
    J_o, g_o = oracle.gradient(c.og, c.v.astype(np.float64), c.ogeo, c.w.astype(np.float64),
                               (1e-3 * c.pt).astype(np.float64), dobs.astype(np.float64), eps=0.3)
    with c.ctx(**opts) as ctx:
        grad = torch.zeros((c.nz, c.nx), device="cuda")
        J = ctx.gradient(dev(c.v), dev(c.w), dev(1e-3 * c.pt), dev(dobs), grad, eps=0.3)
    assert rel_l2(host(grad), g_o) <= TOL
    assert abs(J - J_o) <= 1e-5 * abs(J_o)


# ----------------------------------------------------------------- dot tests on the GPU

def _dot(a, b):
    return float(np.dot(np.ravel(a).astype(np.float64), np.ravel(b).astype(np.float64)))


def test_gpu_dot_born(case):
    with case.ctx() as c:
        lhs = _dot(case.g_born(c), case.d)
        rhs = _dot(case.dv, case.g_born_adj(c))
    assert abs(lhs - rhs) <= DOT_TOL * max(abs(lhs), abs(rhs))


def test_gpu_dot_born_ext(case):
    with case.ctx(segment=16) as c:
        lhs = _dot(case.g_ext(c), case.d)
        rhs = _dot(case.pt, case.g_ext_adj(c))
    assert abs(lhs - rhs) <= DOT_TOL * max(abs(lhs), abs(rhs))


def test_gpu_dot_tomo(case):
    with case.ctx(segment=16) as c:
        lhs = _dot(case.g_tomo(c), case.d)
        rhs = _dot(case.dv, case.g_tomo_adj(c))
    assert abs(lhs - rhs) <= DOT_TOL * max(abs(lhs), abs(rhs))


# ----------------------------------------------------------------- schedule invariance

def test_batching_and_segments_do_not_change_traces(case):
    """Per-shot arithmetic is the same in every schedule: data outputs are bit-identical."""
    with case.ctx() as a, case.ctx(plain=1, segment=5) as b, case.ctx(shots_per_batch=2, segment=33) as c:
        for fn in (case.g_forward, case.g_born, case.g_ext, case.g_tomo):
            ra, rb, rc = fn(a), fn(b), fn(c)
            assert np.array_equal(ra, rb) and np.array_equal(ra, rc), fn.__name__


def test_graph_replay_and_host_io_match(case):
    s = torch.cuda.Stream()
    with case.ctx() as a:
        ref_img = case.g_ext_adj(a)
        ref_d = case.g_ext(a)
    with fw.Context(case.fg, case.fgeo, stream=s, graph=1) as g:
        with torch.cuda.stream(s):
            for _ in range(2):        # capture, then replay
                d = torch.zeros(case.dshape(), device="cuda")
                g.born_ext(dev(case.v), dev(case.w), dev(case.pt), d)
                assert np.array_equal(host(d), ref_d)
        assert g.launches > 0
    with fw.Context(case.fg, case.fgeo, host_io=1) as h:
        img = np.zeros((case.nh, case.nz, case.nx), dtype=np.float32)
        h.born_ext_adj(case.v, case.w.astype(np.float32), case.d, img)
        assert np.array_equal(img.astype(np.float64), ref_img)


# ----------------------------------------------------------------- reductions and edge cases

def test_nh1_extension_equals_born(case):
    c1 = Case(nh=1)
    with c1.ctx() as c:
        b = c1.g_born(c)
        e = c1.g_ext(c, pt=c1.dv[None])
        ba = c1.g_born_adj(c)
        ea = c1.g_ext_adj(c)
    assert rel_l2(e, b) <= 1e-6
    assert rel_l2(ea[0], ba) <= 1e-6


@pytest.mark.parametrize("nh,W", [(7, 10), (41, 6), (3, 0)])
def test_offsets_past_the_sponge_and_generic_nh(nh, W):
    """nh=7 takes the generic (non-templated) kernels; nh=41 with W=6 reaches past the
    active region, where terms are dropped; W=0 has no sponge at all."""
    c = Case(nz=20, nx=140, W=W, nt=120, nh=nh, nshot=2, seed=3)
    v, w = c.v.astype(np.float64), c.w.astype(np.float64)
    with c.ctx(segment=13) as ctx:
        assert rel_l2(c.g_ext(ctx), oracle.born_ext(c.og, v, c.ogeo, w, c.pt.astype(np.float64))) <= TOL
        assert rel_l2(c.g_ext_adj(ctx), oracle.born_ext_adj(c.og, v, c.ogeo, w, c.d.astype(np.float64))) <= TOL
        # T*: the transposed scatter also emits the second adjoint field's source (generic kernel + a
        # separate second difference at nh 7, two outputs per lane at nh 41)
        assert rel_l2(c.g_tomo_adj(ctx), oracle.tomo_adj(c.og, v, c.ogeo, w, c.pt.astype(np.float64),
                                                         c.d.astype(np.float64))) <= TOL


def test_scatter_pairs_split_over_warps():
    """Few (row, column block) tasks and long segments: the scatter splits every task's pairs (shots,
    for the transposed one of T*) over several warps to fill the last wave of resident CTAs."""
    c = Case(nz=64, nx=600, W=10, nt=121, nh=5, nshot=4, seed=8)
    v, w = c.v.astype(np.float64), c.w.astype(np.float64)
    with c.ctx(segment=60) as ctx:
        assert rel_l2(c.g_ext(ctx), oracle.born_ext(c.og, v, c.ogeo, w, c.pt.astype(np.float64))) <= TOL
        assert rel_l2(c.g_ext_adj(ctx), oracle.born_ext_adj(c.og, v, c.ogeo, w, c.d.astype(np.float64))) <= TOL
        assert rel_l2(c.g_tomo_adj(ctx), oracle.tomo_adj(c.og, v, c.ogeo, w, c.pt.astype(np.float64),
                                                         c.d.astype(np.float64))) <= TOL


@pytest.mark.parametrize("segment", [1, 2, 3])
def test_tomo_adj_short_segments(segment):
    """Segments of one to three steps: the source of the second adjoint field at a segment's last
    steps takes one or two samples of the transposed scatter from the segment after it."""
    c = Case(nz=16, nx=120, W=6, nt=40, nh=5, nshot=3, seed=6)
    v, w = c.v.astype(np.float64), c.w.astype(np.float64)
    ref = oracle.tomo_adj(c.og, v, c.ogeo, w, c.pt.astype(np.float64), c.d.astype(np.float64))
    with c.ctx(segment=segment, shots_per_batch=2) as ctx:
        assert rel_l2(c.g_tomo_adj(ctx), ref) <= TOL


def test_two_time_samples():
    c = Case(nz=8, nx=40, W=2, nt=2, nh=3, nshot=2, seed=4)
    v, w = c.v.astype(np.float64), c.w.astype(np.float64)
    with c.ctx() as ctx:
        d = c.g_forward(ctx)
        ref = oracle.forward(c.og, v, c.ogeo, w)
        assert np.all(d[:, 0, :] == 0.0) and np.abs(ref[:, 1, :]).max() > 0
        assert rel_l2(d, ref) <= TOL
        assert rel_l2(c.g_ext_adj(ctx), oracle.born_ext_adj(c.og, v, c.ogeo, w, c.d.astype(np.float64))) <= TOL


def test_cfl_violation_is_reported(case):
    with case.ctx() as c:
        d = torch.zeros(case.dshape(), device="cuda")
        with pytest.raises(fw.FwimeError) as e:
            c.forward(dev(case.v * 10.0), dev(case.w), d)
        assert e.value.code == fw.FWIME_ECFL
        with pytest.raises(fw.FwimeError) as e:
            c.forward(dev(-case.v), dev(case.w), d)
        assert e.value.code == fw.FWIME_ECFL
        c.forward(dev(case.v), dev(case.w), d)     # the context stays usable


def test_workspace_budget_enforced(case):
    with fw.Context(case.fg, case.fgeo, max_workspace_bytes=1 << 16) as c:
        d = torch.zeros(case.dshape(), device="cuda")
        with pytest.raises(fw.FwimeError) as e:
            c.forward(dev(case.v), dev(case.w), d)
        assert e.value.code == fw.FWIME_ENOMEM


def test_autotuner_picks_a_chunking_without_changing_results(case):
    with case.ctx() as a, case.ctx() as b:
        zc, us = b.autotune(fw.OP_BORN_EXT)
        assert zc >= 8 and us > 0
        assert b.get_option("zchunk") == zc
        assert np.array_equal(case.g_ext(a), case.g_ext(b))
        assert np.array_equal(case.g_forward(a), case.g_forward(b))
