"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test would fail for a plausible mistake in the oracle (a dropped term, a
wrong sign, a transposed operand, an off-by-one in time):
  - Laplacian exact on polynomials (coefficients, spacing)
  - dot-product tests of every primitive and operator pair (exact transposes)
  - 2-D analytic Green's function under grid refinement (source scaling,
    c = v^2 dt^2, recording time convention, 2nd-order convergence)
  - Born = Jacobian of f, T = Jacobian of B~ p~, gradient = dPhi/dm (Eqs. 7-9)
  - source-receiver reciprocity, time-shift invariance, mirror symmetry
  - reductions nh=1 / h=0 of the extension to the non-extended Born operator
  - scattering kinematics of the subsurface-offset extension (sign of h)
  - the paper's printed cost table (Eqs. 10-11)
"""
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_grid(nh=5, nt=120, nz=16, nx=24, W=6):
    return oracle.Grid(nz=nz, nx=nx, W=W, nt=nt, dt=1e-3, dx=10.0, nh=nh)


def small_model(g, seed=1):
    rng = np.random.default_rng(seed)
    v = 2000.0 + 300.0 * rng.random((g.nz, g.nx))
    return v


def small_geo(g):
    return oracle.Geometry(np.array([2, 3]), np.array([5, g.nx - 6]),
                           np.concatenate([np.full(g.nx // 2, 1), [g.nz - 3]]),
                           np.concatenate([2 * np.arange(g.nx // 2), [g.nx // 2]]))


def rel(a, b):
    return abs(a - b) / max(abs(a), abs(b), 1e-300)


# ----------------------------------------------------------------- Laplacian

def test_laplacian_exact_on_polynomials():
    """8th-order central differences differentiate polynomials of degree <= 9 exactly."""
    g = oracle.Grid(nz=10, nx=12, W=2, nt=3, dt=1e-3, dx=3.0, dz=2.0)
    Z, X = np.meshgrid(np.arange(g.NZ) * 2.0, np.arange(g.NX) * 3.0, indexing="ij")
    act = oracle.prep(g, np.full((g.nz, g.nx), 1000.0))[0] != 0
    worst = {}
    for k in range(0, 11):
        for axis in ("x", "z"):
            s = X / (g.NX * 3.0) if axis == "x" else Z / (g.NZ * 2.0)
            scale = (g.NX * 3.0) if axis == "x" else (g.NZ * 2.0)
            q = s ** k
            exact = k * (k - 1) * s ** max(k - 2, 0) / scale ** 2 if k >= 2 else np.zeros_like(q)
            h = 3.0 if axis == "x" else 2.0
            # round-off reference: the size of the individual stencil terms, max|q| / h^2
            err = np.abs(oracle.lap(g, q) - exact)[act].max() / (np.abs(q).max() / h ** 2)
            worst[k] = max(worst.get(k, 0.0), err)
    exact_part = max(worst[k] for k in range(10))
    assert exact_part < 1e-12, worst
    # degree 10 is NOT differentiated exactly: the pin is sharp (a wrong coefficient shows up
    # as an error at a degree <= 9 instead)
    assert worst[10] > 1e3 * exact_part, worst


def test_laplacian_symmetric_on_active_fields():
    g = small_grid()
    rng = np.random.default_rng(3)
    c, gam, b = oracle.prep(g, small_model(g))
    act = (c != 0).astype(float)
    a = rng.standard_normal((g.NZ, g.NX)) * act
    bb = rng.standard_normal((g.NZ, g.NX)) * act
    assert rel((oracle.lap(g, a) * bb).sum(), (a * oracle.lap(g, bb)).sum()) < 1e-13


# ----------------------------------------------------------- primitive dots

def test_dot_step_and_prop():
    g = small_grid()
    rng = np.random.default_rng(4)
    c, gam, _ = oracle.prep(g, small_model(g))
    act = (c != 0).astype(float)
    qc, qp, s, qn = [rng.standard_normal((g.NZ, g.NX)) * act for _ in range(4)]
    fw = oracle.step(g, c, gam, qc, qp, s)
    tc, tp, ts = oracle.step_T(g, c, gam, qn)
    assert rel((fw * qn).sum(), (tc * qc).sum() + (tp * qp).sum() + (ts * s).sum()) < 1e-13
    S = rng.standard_normal((g.nt - 1, g.NZ, g.NX)) * act
    A = rng.standard_normal((g.nt, g.NZ, g.NX)) * act
    assert rel((oracle.prop(g, c, gam, S) * A).sum(), (S * oracle.prop_T(g, c, gam, A)).sum()) < 1e-12


def test_dot_d2t():
    g = small_grid(nt=30)
    rng = np.random.default_rng(5)
    q = rng.standard_normal((g.nt, g.NZ, g.NX))
    z = rng.standard_normal((g.nt - 1, g.NZ, g.NX))
    assert rel((oracle.d2t(g, q) * z).sum(), (q * oracle.d2t_T(g, z)).sum()) < 1e-13


def test_dot_scatter_all_arguments():
    """<E(W,D), e*> = <W, E_W^T(D,e*)> = <D, E_D^T(W,e*)>, including offsets that leave the grid."""
    for nh in (1, 5, 41):   # nh=41 reaches past the sponge: dropped terms must be dropped alike
        g = small_grid(nh=nh)
        rng = np.random.default_rng(6 + nh)
        c, _, _ = oracle.prep(g, small_model(g))
        act = (c != 0).astype(float)
        Wt = rng.standard_normal((g.nh, g.nz, g.nx))
        D = rng.standard_normal((g.NZ, g.NX)) * act
        es = rng.standard_normal((g.NZ, g.NX)) * act
        lhs = (oracle.scatter(g, Wt, D) * es).sum()
        assert rel(lhs, (Wt * oracle.scatter_TW(g, D, es)).sum()) < 1e-13
        assert rel(lhs, (D * oracle.scatter_TD(g, Wt, es)).sum()) < 1e-13


# ------------------------------------------------------------ operator dots

@pytest.fixture(scope="module")
def op_case():
    g = small_grid(nh=5)
    rng = np.random.default_rng(7)
    v = small_model(g)
    geo = small_geo(g)
    w = synth.ricker(g.nt, g.dt, 25.0)
    d = rng.standard_normal((geo.nshot, g.nt, geo.nrec))
    dv = rng.standard_normal((g.nz, g.nx))
    pt = rng.standard_normal((g.nh, g.nz, g.nx))
    return g, v, geo, w, d, dv, pt


def test_dot_born(op_case):
    g, v, geo, w, d, dv, pt = op_case
    lhs = (oracle.born(g, v, geo, w, dv) * d).sum()
    rhs = (dv * oracle.born_adj(g, v, geo, w, d)).sum()
    assert rel(lhs, rhs) < 1e-12


def test_dot_born_ext(op_case):
    g, v, geo, w, d, dv, pt = op_case
    lhs = (oracle.born_ext(g, v, geo, w, pt) * d).sum()
    rhs = (pt * oracle.born_ext_adj(g, v, geo, w, d)).sum()
    assert rel(lhs, rhs) < 1e-12


def test_dot_tomo(op_case):
    g, v, geo, w, d, dv, pt = op_case
    lhs = (oracle.tomo(g, v, geo, w, pt, dv) * d).sum()
    rhs = (dv * oracle.tomo_adj(g, v, geo, w, pt, d)).sum()
    assert rel(lhs, rhs) < 1e-12


# --------------------------------------------------- analytic Green function

def _green_2d(r, t, v0, f0):
    """w * G2D with G2D = H(t - r/v)/(2 pi sqrt(t^2 - r^2/v^2)), by the substitution
    tau = (r/v) cosh u, which removes the wavefront singularity."""
    out = np.zeros_like(t)
    for i, tt in enumerate(t):
        if tt * v0 <= r:
            continue
        u = np.linspace(0.0, math.acosh(v0 * tt / r), 4001)
        out[i] = np.trapezoid(synth.ricker_at(tt - (r / v0) * np.cosh(u), f0), u) / (2 * math.pi)
    return out


def test_green_function_convergence():
    """Homogeneous medium: traces converge to the 2-D Green's-function convolution at 2nd order
    (dx = 20, 10, 5 m at a fixed Courant number), with boundary echoes outside the window."""
    v0, f0, H, tmax = 2000.0, 10.0, 900.0, 0.55
    offs = [200.0, 400.0, 600.0]
    errs = []
    for dx in (20.0, 10.0, 5.0):
        n = int(round(2 * H / dx)) + 1
        dt = 0.2 * dx / v0
        nt = int(round(tmax / dt)) + 1
        g = oracle.Grid(nz=n, nx=n, W=20, nt=nt, dt=dt, dx=dx)
        c = n // 2
        geo = oracle.Geometry(np.array([c]), np.array([c]), np.array([c] * 3),
                              np.array([c + int(round(o / dx)) for o in offs]))
        d = oracle.forward(g, np.full((n, n), v0), geo, synth.ricker(nt, dt, f0))[0]
        t = np.arange(nt) * dt
        errs.append([np.linalg.norm(d[:, k] - a) / np.linalg.norm(a)
                     for k, a in enumerate(_green_2d(o, t, v0, f0) for o in offs)])
    errs = np.array(errs)
    ratios = errs[:-1] / errs[1:]
    assert np.all(ratios > 3.3) and np.all(ratios < 4.6), ratios       # 2nd order
    assert errs[-1].max() < 2e-3 and errs[-1][0] < 6e-4, errs[-1]


# ---------------------------------------------------------------- Jacobians

def _fd_slopes(fun, lin, eps_list):
    errs = []
    for e in eps_list:
        fd = (fun(e) - fun(-e)) / (2 * e)
        errs.append(np.linalg.norm(fd - lin) / np.linalg.norm(lin))
    return np.array(errs)


def test_born_is_jacobian_of_forward(op_case):
    g, v, geo, w, d, dv, pt = op_case
    rng = np.random.default_rng(11)
    dvs = synth.gaussian_blobs(g.nz, g.nx, rng, amp=100.0, sigma_pts=3.0, ring=1)
    lin = oracle.born(g, v, geo, w, dvs)
    errs = _fd_slopes(lambda e: oracle.forward(g, v + e * dvs, geo, w), lin, [1.0, 0.1, 0.01, 0.001])
    assert errs[0] / errs[1] > 80 and errs[1] / errs[2] > 80, errs    # slope 2 in eps
    assert errs[-1] < 1e-7, errs


def test_born_with_edge_perturbation_is_not_jacobian(op_case):
    """Sharpness: a dv on the outermost physical ring also perturbs the replicated padding,
    which B (zero-embedded dv) does not see."""
    g, v, geo, w, d, dv, pt = op_case
    dve = np.zeros((g.nz, g.nx)); dve[:, 0] = 100.0
    lin = oracle.born(g, v, geo, w, dve)
    errs = _fd_slopes(lambda e: oracle.forward(g, v + e * dve, geo, w), lin, [0.01])
    assert errs[0] > 1e-3


def test_tomo_is_jacobian_of_extended_born(op_case):
    g, v, geo, w, d, dv, pt = op_case
    rng = np.random.default_rng(12)
    dvs = synth.gaussian_blobs(g.nz, g.nx, rng, amp=100.0, sigma_pts=3.0, ring=1)
    lin = oracle.tomo(g, v, geo, w, pt, dvs)
    errs = _fd_slopes(lambda e: oracle.born_ext(g, v + e * dvs, geo, w, pt), lin, [1.0, 0.1, 0.01, 0.001])
    assert errs[0] / errs[1] > 80 and errs[1] / errs[2] > 80, errs
    assert errs[-1] < 1e-7, errs


def test_gradient_matches_finite_differences(op_case):
    """Phi(m) at fixed p~ and grad = B* r + T* r (Eqs. 7-9) along random smooth directions."""
    g, v, geo, w, d, dv, pt = op_case
    rng = np.random.default_rng(13)
    dobs = oracle.forward(g, v * 1.03, geo, w) + 0.01 * rng.standard_normal((geo.nshot, g.nt, geo.nrec))
    pts = 1e-3 * pt
    J0, grad = oracle.gradient(g, v, geo, w, pts, dobs, eps=1e-2)
    for k in range(3):
        dvs = synth.gaussian_blobs(g.nz, g.nx, rng, amp=10.0, sigma_pts=3.0, ring=1)
        e = 0.01
        Jp, _ = oracle.gradient(g, v + e * dvs, geo, w, pts, dobs, eps=1e-2)
        Jm, _ = oracle.gradient(g, v - e * dvs, geo, w, pts, dobs, eps=1e-2)
        fd = (Jp - Jm) / (2 * e)
        an = float((grad * dvs).sum())
        assert rel(fd, an) < 1e-6, (k, fd, an)


def test_gradient_splits_into_born_and_tomo(op_case):
    """grad = B* r + T* r with r = f + B~ p~ - d (Eq. 7), the objective being 1/2||r||^2 + DSO term."""
    g, v, geo, w, d, dv, pt = op_case
    dobs = 0.5 * d
    J, grad = oracle.gradient(g, v, geo, w, pt, dobs, eps=0.0)
    r = oracle.forward(g, v, geo, w) + oracle.born_ext(g, v, geo, w, pt) - dobs
    assert rel(J, 0.5 * (r ** 2).sum()) < 1e-12
    ref = oracle.born_adj(g, v, geo, w, r) + oracle.tomo_adj(g, v, geo, w, pt, r)
    assert np.linalg.norm(grad - ref) / np.linalg.norm(ref) < 1e-12


# ------------------------------------------------------------- symmetries

def test_reciprocity():
    g = oracle.Grid(nz=30, nx=40, W=8, nt=300, dt=1e-3, dx=10.0)
    rng = np.random.default_rng(14)
    v = 1800.0 + 800.0 * rng.random((g.nz, g.nx))
    w = synth.ricker(g.nt, g.dt, 20.0)
    A, B = (2, 5), (21, 33)
    dAB = oracle.forward(g, v, oracle.Geometry(np.array([A[0]]), np.array([A[1]]),
                                               np.array([B[0]]), np.array([B[1]])), w)[0, :, 0]
    dBA = oracle.forward(g, v, oracle.Geometry(np.array([B[0]]), np.array([B[1]]),
                                               np.array([A[0]]), np.array([A[1]])), w)[0, :, 0]
    assert np.abs(dAB).max() > 0
    assert np.abs(dAB - dBA).max() <= 1e-11 * np.abs(dAB).max()


def test_time_shift_is_exact(op_case):
    g, v, geo, w, d, dv, pt = op_case
    k = 7
    ws = np.concatenate([np.zeros(k), w[:-k]])
    d0 = oracle.born_ext(g, v, geo, w, pt)
    d1 = oracle.born_ext(g, v, geo, ws, pt)
    assert np.array_equal(d1[:, k:, :], d0[:, :-k, :])
    assert np.all(d1[:, :k, :] == 0.0)


def test_mirror_symmetry():
    g = oracle.Grid(nz=20, nx=31, W=6, nt=150, dt=1e-3, dx=10.0)
    rng = np.random.default_rng(15)
    half = 1800.0 + 600.0 * rng.random((g.nz, 16))
    v = np.concatenate([half, half[:, -2::-1]], axis=1)
    assert np.array_equal(v, v[:, ::-1])
    geo = oracle.Geometry(np.array([3]), np.array([15]), np.full(g.nx, 2), np.arange(g.nx))
    d = oracle.forward(g, v, geo, synth.ricker(g.nt, g.dt, 20.0))[0]
    assert np.abs(d).max() > 0
    assert np.array_equal(d, d[:, ::-1])


# ------------------------------------------------------------- reductions

def test_extension_reduces_to_born(op_case):
    """nh=1 (and p~ non-zero only at h=0) reduce B~ and B~* to B and B*."""
    g, v, geo, w, d, dv, pt = op_case
    g1 = small_grid(nh=1)
    bd = oracle.born(g1, v, geo, w, dv)
    assert np.linalg.norm(oracle.born_ext(g1, v, geo, w, dv[None]) - bd) <= 1e-13 * np.linalg.norm(bd)
    pt0 = np.zeros((g.nh, g.nz, g.nx)); pt0[g.nh // 2] = dv
    assert np.linalg.norm(oracle.born_ext(g, v, geo, w, pt0) - bd) <= 1e-13 * np.linalg.norm(bd)
    ba = oracle.born_adj(g1, v, geo, w, d)
    ea = oracle.born_ext_adj(g, v, geo, w, d)
    assert np.linalg.norm(ea[g.nh // 2] - ba) <= 1e-13 * np.linalg.norm(ba)
    assert np.all(oracle.born_ext(g, v, geo, w, np.zeros_like(pt)) == 0.0)


def test_extended_born_is_linear(op_case):
    g, v, geo, w, d, dv, pt = op_case
    rng = np.random.default_rng(16)
    p2 = rng.standard_normal(pt.shape)
    a = oracle.born_ext(g, v, geo, w, 2.0 * pt - 3.0 * p2)
    b = 2.0 * oracle.born_ext(g, v, geo, w, pt) - 3.0 * oracle.born_ext(g, v, geo, w, p2)
    assert np.linalg.norm(a - b) <= 1e-13 * np.linalg.norm(a)


# ------------------------------------------------------------- kinematics

def _xcorr_shift(a, b):
    """Lag (in samples, sub-sample by a parabola) that best aligns b to a."""
    n = len(a)
    cc = np.correlate(b, a, mode="full")
    k = int(np.argmax(cc))
    if 0 < k < len(cc) - 1:
        y0, y1, y2 = cc[k - 1], cc[k], cc[k + 1]
        k = k + 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2)
    return k - (n - 1)


def test_subsurface_offset_kinematics():
    """A spike of p~ at (z0, x0, h0) couples the source field at x0-h0 to the receiver side at x0+h0
    (Eq. 1 extension): the arrival-time difference between h0 and -h0 follows the travel paths."""
    v0, dx, f0 = 2000.0, 10.0, 15.0
    g = oracle.Grid(nz=50, nx=121, W=10, nt=900, dt=1e-3, dx=dx, nh=17)
    v = np.full((g.nz, g.nx), v0)
    z0, x0, h = 40, 60, 8
    xs, xr = x0 + 40, x0 - 40
    geo = oracle.Geometry(np.array([2]), np.array([xs]), np.array([2]), np.array([xr]))
    w = synth.ricker(g.nt, g.dt, f0)

    def trace(hh):
        pt = np.zeros((g.nh, g.nz, g.nx)); pt[hh + g.nh // 2, z0, x0] = 1.0
        return oracle.born_ext(g, v, geo, w, pt)[0, :, 0]

    def path(hh):
        return (math.hypot((x0 - hh - xs) * dx, (z0 - 2) * dx)
                + math.hypot((x0 + hh - xr) * dx, (z0 - 2) * dx)) / v0

    lag = _xcorr_shift(trace(-h), trace(+h)) * g.dt
    pred = path(+h) - path(-h)
    assert abs(pred) > 20 * g.dt          # the two conventions differ clearly
    assert abs(lag - pred) < 2 * g.dt, (lag, pred)


# ------------------------------------------------------------- sponge

def test_sponge_absorbs():
    """Energy that reaches the Cerjan-type sponge leaves the domain; without it, it stays."""
    def late_fraction(W):
        g = oracle.Grid(nz=41, nx=41, W=W, nt=900, dt=1e-3, dx=10.0)
        zz, xx = np.meshgrid(np.arange(g.nz), np.arange(g.nx), indexing="ij")
        geo = oracle.Geometry(np.array([20]), np.array([20]), zz.ravel(), xx.ravel())
        d = oracle.forward(g, np.full((g.nz, g.nx), 2000.0), geo, synth.ricker(g.nt, g.dt, 15.0))[0]
        e = (d ** 2).sum(axis=1)
        return e[-50:].max() / e.max()
    assert late_fraction(30) < 1e-3
    assert late_fraction(0) > 1e-1


# ------------------------------------------------------------- DSO penalty

def test_dso_penalty_closed_form():
    g = small_grid(nh=5)
    pt = np.ones((g.nh, g.nz, g.nx))
    # weights |h|+1 over h = -2..2: 3,2,1,2,3 -> sum of squares 27
    assert rel(oracle.dso_penalty(g, pt, 0.5), 0.5 * 0.25 * 27 * g.nz * g.nx) < 1e-14


@pytest.mark.parametrize("nh", [1, 5, 21, 41])
def test_dso_operator_properties(nh):
    """The paper asks only that D be an invertible, modified DSO operator (Theory, Eq. 1): a penalty
    that vanishes nowhere, treats +h and -h alike and grows away from zero offset.  Probe the oracle's
    C arithmetic one offset plane at a time (a unit spike on plane ih gives 1/2 D(ih)^2 at eps = 1):
    D > 0, symmetric in h, smallest at h = 0 and strictly increasing in |h| -- a shifted centre, a
    zero weight or a sign slip fails one of these."""
    g = small_grid(nh=nh)
    hm = (nh - 1) // 2
    d = []
    for ih in range(nh):
        pt = np.zeros((g.nh, g.nz, g.nx))
        pt[ih, g.nz // 2, g.nx // 3] = 1.0
        d.append(np.sqrt(2.0 * oracle.dso_penalty(g, pt, 1.0)))
    d = np.array(d)
    assert np.all(d > 0.0)
    assert np.array_equal(d, d[::-1])
    assert np.argmin(d) == hm and np.sum(d == d.min()) == 1
    assert np.all(np.diff(d[hm:]) > 0.0)
    # linear in p~ planes: the penalty of a sum over planes is the sum of the planes' penalties
    pt = np.ones((g.nh, g.nz, g.nx))
    assert rel(oracle.dso_penalty(g, pt, 1.0), 0.5 * float(np.sum(d ** 2)) * g.nz * g.nx) < 1e-12


# ------------------------------------------------------------- cost table

def test_cost_table_matches_paper():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "cost_table.txt")) if ln.strip() and ln[0] != "#"]
    fwi = [r for r in rows if r[0] == "FWI"][0]
    c_fwi = float(fwi[4])
    assert c_fwi == 4
    for r in rows:
        if r[0] != "FWIME":
            continue
        n_vp, c_ext, c_vp, c_tot, share, ratio = int(r[1]), float(r[2]) / 100, *map(float, r[3:])
        assert oracle.cost_vp(n_vp, c_ext) == pytest.approx(c_vp, abs=1e-9)
        assert oracle.cost_fwime(n_vp, c_ext) == pytest.approx(c_tot, abs=1e-9)
        assert abs(100 * c_vp / c_tot - share) <= 0.5
        assert abs(oracle.cost_fwime(n_vp, c_ext) / c_fwi - ratio) <= 0.5   # printed ratios are rounded
