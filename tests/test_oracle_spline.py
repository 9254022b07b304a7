"""Pins of the oracle's linear spline re-parametrisation S (v = S m, Eq. 1) and its adjoint.

Linear splines reproduce linear functions exactly between the end nodes, their weights sum to
one, S with nodes on every grid point is the identity, the hat functions of uniform nodes
reduce to the classic bilinear weights, and S* is the transpose of S (dot test)."""
import numpy as np

import oracle


def test_linear_functions_are_reproduced():
    nz, nx, dz, dx = 41, 57, 10.0, 12.5
    zs = np.array([0.0, 70.0, 95.0, 200.0, 400.0])      # non-uniform, the last node at the grid's end
    xs = np.linspace(0.0, 700.0, 6)
    m = 1500.0 + 2.0 * zs[:, None] - 0.7 * xs[None, :]
    v = oracle.spline(zs, xs, nz, nx, dz, dx, m)
    z = np.arange(nz)[:, None] * dz
    x = np.arange(nx)[None, :] * dx
    assert np.abs(v - (1500.0 + 2.0 * z - 0.7 * x)).max() <= 1e-9


def test_partition_of_unity_and_constant_extension():
    zs = np.array([15.0, 40.0, 90.0])
    A = oracle.spline_matrix(zs, np.arange(12) * 10.0)
    assert np.allclose(A.sum(axis=1), 1.0, atol=1e-15)
    assert A[0, 0] == 1.0 and A[1, 0] == 1.0          # 0 m and 10 m lie before the first node
    assert A[-1, -1] == 1.0 and A[-2, -1] == 1.0      # 100 m and 110 m lie after the last node
    assert np.allclose(A[3], [0.4, 0.6, 0.0])         # 30 m: 15 m past the 15 m node, 10 m before 40 m


def test_nodes_on_the_grid_give_the_identity():
    nz, nx, dz, dx = 9, 13, 30.0, 30.0
    m = np.random.default_rng(1).standard_normal((nz, nx))
    assert np.array_equal(oracle.spline(np.arange(nz) * dz, np.arange(nx) * dx, nz, nx, dz, dx, m), m)


def test_uniform_nodes_give_bilinear_weights():
    # nodes every 4 points: grid point j lies at fraction (j mod 4) / 4 of its interval
    A = oracle.spline_matrix(np.arange(0, 41, 4) * 10.0, np.arange(41) * 10.0)
    for j in range(40):
        k, f = j // 4, (j % 4) / 4.0
        assert abs(A[j, k] - (1 - f)) < 1e-15 and abs(A[j, k + 1] - f) < 1e-15


def test_adjoint_dot_product():
    rng = np.random.default_rng(2)
    nz, nx, dz, dx = 50, 64, 10.0, 10.0
    zs = np.sort(rng.uniform(-20.0, 520.0, 7)); xs = np.sort(rng.uniform(0.0, 640.0, 9))
    m = rng.standard_normal((7, 9)); g = rng.standard_normal((nz, nx))
    lhs = np.sum(oracle.spline(zs, xs, nz, nx, dz, dx, m) * g)
    rhs = np.sum(m * oracle.spline_adj(zs, xs, nz, nx, dz, dx, g))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def nested_grids():
    """A coarse node set (0.2 km x 1 km, as the paper's first Marmousi2 spline grid), its refinement by
    halving the spacing twice, and a finite-difference grid of 10 m."""
    zc = np.arange(0.0, 1401.0, 200.0)
    xc = np.arange(0.0, 6001.0, 1000.0)
    zm, xm = np.arange(0.0, 1401.0, 100.0), np.arange(0.0, 6001.0, 500.0)
    zf, xf = np.arange(0.0, 1401.0, 50.0), np.arange(0.0, 6001.0, 250.0)
    return zc, xc, zm, xm, zf, xf


def test_refinement_reproduces_the_coarse_model_exactly():
    """Coarse nodes that are also fine nodes: S on the fine nodes applied to the carried-over model equals S
    on the coarse nodes (a piecewise-linear function on a partition is piecewise linear on any refinement),
    also beyond the grid's end nodes (constant extension)."""
    zc, xc, zm, xm, zf, xf = nested_grids()
    rng = np.random.default_rng(42)
    mc = 1500.0 + 3000.0 * rng.random((len(zc), len(xc)))
    nz, nx, dz, dx = 150, 620, 10.0, 10.0                    # the FD grid reaches past the last nodes
    for z2, x2 in ((zm, xm), (zf, xf), (zf, xm)):
        mf = oracle.spline_refine(zc, xc, mc, z2, x2)
        a = oracle.spline(z2, x2, nz, nx, dz, dx, mf)
        b = oracle.spline(zc, xc, nz, nx, dz, dx, mc)
        assert np.abs(a - b).max() <= 1e-10 * np.abs(b).max()
    # the fine nodes that coincide with coarse ones keep their values exactly
    mf = oracle.spline_refine(zc, xc, mc, zf, xf)
    assert np.array_equal(mf[::4, ::4], mc)


def test_refinement_composes_and_is_the_identity_on_the_same_nodes():
    zc, xc, zm, xm, zf, xf = nested_grids()
    rng = np.random.default_rng(7)
    mc = rng.standard_normal((len(zc), len(xc)))
    assert np.array_equal(oracle.spline_refine(zc, xc, mc, zc, xc), mc)
    two = oracle.spline_refine(zm, xm, oracle.spline_refine(zc, xc, mc, zm, xm), zf, xf)
    one = oracle.spline_refine(zc, xc, mc, zf, xf)
    assert np.abs(two - one).max() <= 1e-12 * np.abs(one).max()


def test_refinement_of_a_linear_model_samples_it():
    zc, xc, zm, xm, zf, xf = nested_grids()
    lin = lambda z, x: 1500.0 + 1.5 * z[:, None] + 0.25 * x[None, :]  # noqa: E731
    mf = oracle.spline_refine(zc, xc, lin(zc, xc), zf, xf)
    assert np.abs(mf - lin(zf, xf)).max() <= 1e-9
    # a coarse grid that is not a subset: the transfer still samples the coarse spline exactly
    zo, xo = zf + 17.0, xf + 33.0
    mo = oracle.spline_refine(zc, xc, lin(zc, xc), zo[:-1], xo[:-1])
    assert np.abs(mo - lin(zo[:-1], xo[:-1])).max() <= 1e-9
