"""Pins of the oracle's time-lag extension (B~ "extended with time lags", Eq. 1, and its adjoint).

- the adjoint is the transpose (dot test);
- a single zero lag is the non-extended Born operator with dv = p~;
- a p~ concentrated on one lag i produces the zero-lag data delayed by exactly 2 s_i samples,
  s_i = (i - hm) lag (the propagation is time-invariant), which fixes the factor 2, the sign of the
  lag and its spacing;
- linearity in p~.
"""
import numpy as np

import oracle


def setup(nh=5, lag=3, nt=240):
    g = oracle.Grid(nz=24, nx=36, W=6, nt=nt, dt=1e-3, dx=10.0, nh=nh, lag=lag)
    rng = np.random.default_rng(4)
    v = 2000.0 + 200.0 * rng.random((g.nz, g.nx))
    geo = oracle.Geometry(np.array([2, 3]), np.array([5, 30]), np.full(18, 1), 2 * np.arange(18))
    t = np.arange(nt) * g.dt
    # a wavelet that is exactly zero for the first 20 samples
    w = np.stack([np.where(t >= 0.02, np.sin(2 * np.pi * 25.0 * (t - 0.05)) * np.exp(-((t - 0.05) / 0.012) ** 2), 0.0)] * 2)
    return g, v, geo, w, rng


def test_adjoint_dot_product():
    g, v, geo, w, rng = setup()
    pt = rng.standard_normal((g.nh, g.nz, g.nx))
    d = rng.standard_normal((geo.nshot, g.nt, geo.nrec))
    lhs = np.sum(oracle.born_ext(g, v, geo, w, pt) * d)
    rhs = np.sum(pt * oracle.born_ext_adj(g, v, geo, w, d))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_single_zero_lag_is_born():
    g, v, geo, w, rng = setup(nh=1)
    dv = rng.standard_normal((g.nz, g.nx))
    g0 = oracle.Grid(nz=g.nz, nx=g.nx, W=g.W, nt=g.nt, dt=g.dt, dx=g.dx)
    a = oracle.born_ext(g, v, geo, w, dv[None])
    b = oracle.born(g0, v, geo, w, dv)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    d = rng.standard_normal((geo.nshot, g.nt, geo.nrec))
    assert np.abs(oracle.born_ext_adj(g, v, geo, w, d)[0] - oracle.born_adj(g0, v, geo, w, d)).max() <= \
        1e-12 * np.abs(oracle.born_adj(g0, v, geo, w, d)).max()


def test_one_lag_delays_the_zero_lag_data_by_twice_the_lag():
    g, v, geo, w, rng = setup(nh=5, lag=3)
    hm = (g.nh - 1) // 2
    q = np.zeros((g.nz, g.nx))
    q[18:21, 14:20] = rng.standard_normal((3, 6))      # scatterers far enough from both sources that the
    base = np.zeros((g.nh, g.nz, g.nx)); base[hm] = q   # background there is exactly zero for the first steps
    d0 = oracle.born_ext(g, v, geo, w, base)
    for i in range(g.nh):
        pt = np.zeros((g.nh, g.nz, g.nx)); pt[i] = q
        di = oracle.born_ext(g, v, geo, w, pt)
        sh = 2 * (i - hm) * g.lag
        if sh >= 0:        # delayed: the first sh samples are silent
            ref, got = np.concatenate([np.zeros_like(d0[:, :sh]), d0[:, :g.nt - sh]], axis=1), di
        else:              # advanced: the last -sh samples would need d0 beyond the record
            ref, got = d0[:, -sh:], di[:, :g.nt + sh]
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(d0).max(), i


def test_linear_in_the_extended_perturbation():
    g, v, geo, w, rng = setup()
    p1, p2 = rng.standard_normal((2, g.nh, g.nz, g.nx))
    lhs = oracle.born_ext(g, v, geo, w, 2.0 * p1 - 0.5 * p2)
    rhs = 2.0 * oracle.born_ext(g, v, geo, w, p1) - 0.5 * oracle.born_ext(g, v, geo, w, p2)
    assert np.abs(lhs - rhs).max() <= 1e-12 * np.abs(rhs).max()


# ---------------------------------------------------- tomographic operator and gradient with time lags

def op_case_tlag():
    g = oracle.Grid(nz=16, nx=24, W=6, nt=120, dt=1e-3, dx=10.0, nh=5, lag=2)
    rng = np.random.default_rng(7)
    v = 2000.0 + 300.0 * rng.random((g.nz, g.nx))
    geo = oracle.Geometry(np.array([2, 3]), np.array([5, g.nx - 6]),
                          np.concatenate([np.full(g.nx // 2, 1), [g.nz - 3]]),
                          np.concatenate([2 * np.arange(g.nx // 2), [g.nx // 2]]))
    import synth
    w = synth.ricker(g.nt, g.dt, 25.0)
    return g, v, geo, w, rng


def test_tomo_adjoint_dot_product_with_lags():
    g, v, geo, w, rng = op_case_tlag()
    pt = rng.standard_normal((g.nh, g.nz, g.nx)); dv = rng.standard_normal((g.nz, g.nx))
    d = rng.standard_normal((geo.nshot, g.nt, geo.nrec))
    lhs = np.sum(oracle.tomo(g, v, geo, w, pt, dv) * d)
    rhs = np.sum(dv * oracle.tomo_adj(g, v, geo, w, pt, d))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_tomo_is_jacobian_of_time_lag_born():
    import synth
    g, v, geo, w, rng = op_case_tlag()
    pt = rng.standard_normal((g.nh, g.nz, g.nx))
    dvs = synth.gaussian_blobs(g.nz, g.nx, rng, amp=100.0, sigma_pts=3.0, ring=1)
    lin = oracle.tomo(g, v, geo, w, pt, dvs)
    errs = []
    for e in (1.0, 0.1, 0.01):
        fd = (oracle.born_ext(g, v + e * dvs, geo, w, pt) - oracle.born_ext(g, v - e * dvs, geo, w, pt)) / (2 * e)
        errs.append(np.linalg.norm(fd - lin) / np.linalg.norm(lin))
    assert errs[0] / errs[1] > 80 and errs[1] / errs[2] > 80, errs      # second order
    assert errs[-1] < 1e-6, errs


def test_gradient_with_lags_matches_finite_differences():
    import synth
    g, v, geo, w, rng = op_case_tlag()
    pts = 1e-3 * rng.standard_normal((g.nh, g.nz, g.nx))
    dobs = oracle.forward(g, v * 1.03, geo, w) + 0.01 * rng.standard_normal((geo.nshot, g.nt, geo.nrec))
    J0, grad = oracle.gradient(g, v, geo, w, pts, dobs, eps=1e-2)
    r = oracle.forward(g, v, geo, w) + oracle.born_ext(g, v, geo, w, pts) - dobs
    ref = oracle.born_adj(g, v, geo, w, r) + oracle.tomo_adj(g, v, geo, w, pts, r)
    assert np.linalg.norm(grad - ref) <= 1e-12 * np.linalg.norm(ref)
    for k in range(2):
        dvs = synth.gaussian_blobs(g.nz, g.nx, rng, amp=10.0, sigma_pts=3.0, ring=1)
        e = 0.01
        Jp, _ = oracle.gradient(g, v + e * dvs, geo, w, pts, dobs, eps=1e-2)
        Jm, _ = oracle.gradient(g, v - e * dvs, geo, w, pts, dobs, eps=1e-2)
        fd, an = (Jp - Jm) / (2 * e), float((grad * dvs).sum())
        assert abs(fd - an) <= 1e-6 * abs(an), (k, fd, an)
