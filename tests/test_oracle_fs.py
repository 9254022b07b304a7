"""Pins of the oracle's free-surface reading (pressure release at the top physical row; Marmousi2
free-surface test of the paper).

- image principle: in a medium symmetric about the surface the free-surface field equals the
  whole-space field of the source minus that of its mirror image with the wavelet negated, exactly
  (the discrete scheme keeps odd fields odd), which fixes the surface position, the mirror and the
  sign of the reflection;
- the surface row stays zero;
- the adjoints are the transposes (dot tests of the propagation, B, B~ and T);
- B is the Jacobian of f with the free surface.
"""
import numpy as np

import oracle
import synth


def test_image_source_principle_is_exact():
    nz, nx, W, nt, dx = 20, 40, 8, 220, 10.0
    zs, xs = 6, 19
    rec_z, rec_x = np.full(nx, 3), np.arange(nx)
    w = synth.ricker(nt, 1e-3, 25.0)
    gfs = oracle.Grid(nz=nz, nx=nx, W=W, nt=nt, dt=1e-3, dx=dx, fs=1)
    vfs = np.full((nz, nx), 2000.0)
    dfs = oracle.forward(gfs, vfs, oracle.Geometry(np.array([zs]), np.array([xs]), rec_z, rec_x), w[None])
    # whole space, symmetric about the surface row (row nz - 1 of a 2 nz - 1 row grid), same sponges
    gfull = oracle.Grid(nz=2 * nz - 1, nx=nx, W=W, nt=nt, dt=1e-3, dx=dx)
    vfull = np.full((2 * nz - 1, nx), 2000.0)
    s = nz - 1
    geo = oracle.Geometry(np.array([s + zs, s - zs]), np.array([xs, xs]), s + rec_z, rec_x)
    dfull = oracle.forward(gfull, vfull, geo, np.stack([w, -w]))
    ref = dfull[0] + dfull[1]
    assert np.abs(ref).max() > 0
    assert np.abs(dfs[0] - ref).max() <= 1e-12 * np.abs(ref).max()


def fs_case():
    g = oracle.Grid(nz=16, nx=24, W=6, nt=120, dt=1e-3, dx=10.0, nh=5, fs=1)
    rng = np.random.default_rng(8)
    v = 2000.0 + 300.0 * rng.random((g.nz, g.nx))
    geo = oracle.Geometry(np.array([2, 3]), np.array([5, g.nx - 6]),
                          np.concatenate([np.full(g.nx // 2, 1), [0]]),      # one receiver on the surface row
                          np.concatenate([2 * np.arange(g.nx // 2), [g.nx // 2]]))
    return g, v, geo, synth.ricker(g.nt, g.dt, 25.0), rng


def test_surface_row_is_silent_and_propagation_transposes():
    g, v, geo, w, rng = fs_case()
    d = oracle.forward(g, v, geo, w)
    assert np.all(d[:, :, -1] == 0.0)                # the receiver on the surface records nothing
    c, gam, _ = oracle.prep(g, v)
    act = (c != 0).astype(float)
    S = rng.standard_normal((g.nt - 1, g.NZ, g.NX)) * act
    A = rng.standard_normal((g.nt, g.NZ, g.NX)) * act
    q = oracle.prop(g, c, gam, S)
    o = g.W + 4
    assert np.all(q[:, o, :] == 0.0)
    assert np.array_equal(q[:, o - 3, :], -q[:, o + 3, :])
    lhs, rhs = (q * A).sum(), (S * oracle.prop_T(g, c, gam, A)).sum()
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_operator_dot_products_with_the_free_surface():
    g, v, geo, w, rng = fs_case()
    d = rng.standard_normal((geo.nshot, g.nt, geo.nrec))
    dv = rng.standard_normal((g.nz, g.nx)); pt = rng.standard_normal((g.nh, g.nz, g.nx))
    pairs = [
        ((oracle.born(g, v, geo, w, dv) * d).sum(), (dv * oracle.born_adj(g, v, geo, w, d)).sum()),
        ((oracle.born_ext(g, v, geo, w, pt) * d).sum(), (pt * oracle.born_ext_adj(g, v, geo, w, d)).sum()),
        ((oracle.tomo(g, v, geo, w, pt, dv) * d).sum(), (dv * oracle.tomo_adj(g, v, geo, w, pt, d)).sum()),
    ]
    for lhs, rhs in pairs:
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_born_is_the_jacobian_with_the_free_surface():
    g, v, geo, w, rng = fs_case()
    dvs = synth.gaussian_blobs(g.nz, g.nx, rng, amp=60.0, sigma_pts=3.0, ring=1)
    lin = oracle.born(g, v, geo, w, dvs)
    errs = []
    for e in (0.1, 0.01, 0.001):
        fd = (oracle.forward(g, v + e * dvs, geo, w) - oracle.forward(g, v - e * dvs, geo, w)) / (2 * e)
        errs.append(np.linalg.norm(fd - lin) / np.linalg.norm(lin))
    assert errs[0] / errs[1] > 80 and errs[1] / errs[2] > 80, errs
    assert errs[-1] < 1e-7, errs
