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
