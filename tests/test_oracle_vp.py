"""Pins of the oracle's variable projection solve (linear CG on Eqs. 2-5).

The CG iterates are checked against a characterisation that does not use the
CG recurrences: after k iterations from p_0, conjugate gradients minimise the
quadratic Phi over p_0 + K_k(H, r_0) (the Krylov space of the residual), and
the minimiser over an explicit orthonormal basis of that space is computed here
from a dense copy of B~ built column by column.  A wrong step length, a wrong
sign in a recurrence, a dropped D term or a transposed product moves the
iterate off that minimiser.  With a large eps the system is well conditioned
and CG must reach the dense solve of the normal equations.
"""
import numpy as np

import oracle


def vp_case(eps_scale=1.0, seed=3):
    g = oracle.Grid(nz=6, nx=8, W=4, nt=90, dt=1e-3, dx=10.0, nh=3)
    rng = np.random.default_rng(seed)
    v = 2000.0 + 300.0 * rng.random((g.nz, g.nx))
    geo = oracle.Geometry(np.array([1, 2]), np.array([1, g.nx - 2]), np.full(g.nx, 0), np.arange(g.nx))
    w = np.stack([np.sin(np.arange(g.nt) * 0.21) * np.exp(-((np.arange(g.nt) - 20) / 8.0) ** 2)] * 2)
    n = g.nh * g.nz * g.nx
    B = np.empty((geo.nshot * g.nt * geo.nrec, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        B[:, j] = oracle.born_ext(g, v, geo, w, e.reshape(g.nh, g.nz, g.nx)).ravel()
    scale = np.linalg.norm(B, 2)
    dres = B @ rng.standard_normal(n) + 0.3 * scale * rng.standard_normal(B.shape[0]) / np.sqrt(B.shape[0])
    dres = dres.reshape(geo.nshot, g.nt, geo.nrec)
    eps = eps_scale * scale
    return g, v, geo, w, B, dres, eps


def dense_H(g, B, eps):
    D2 = np.repeat(oracle.dso_weights(g).ravel() ** 2, g.nz * g.nx)
    return B.T @ B + eps * eps * np.diag(D2)


def phi_dense(g, B, dres, eps, p):
    r = B @ p - dres.ravel()
    Dp = np.repeat(oracle.dso_weights(g).ravel(), g.nz * g.nx) * p
    return 0.5 * r @ r + 0.5 * eps * eps * Dp @ Dp


def test_dense_copy_is_the_operator_and_its_adjoint():
    g, v, geo, w, B, dres, eps = vp_case()
    img = oracle.born_ext_adj(g, v, geo, w, dres).ravel()
    assert np.linalg.norm(img - B.T @ dres.ravel()) <= 1e-12 * np.linalg.norm(img)


def test_cg_iterates_minimise_phi_over_the_krylov_space():
    g, v, geo, w, B, dres, eps = vp_case(eps_scale=0.05)
    rng = np.random.default_rng(11)
    p0 = 0.1 * rng.standard_normal((g.nh, g.nz, g.nx))
    H = dense_H(g, B, eps)
    r0 = B.T @ dres.ravel() - H @ p0.ravel()
    # orthonormal basis of K_k(H, r0) by Arnoldi with full re-orthogonalisation
    Q = [r0 / np.linalg.norm(r0)]
    for _ in range(5):
        u = H @ Q[-1]
        for _rep in range(2):
            for q in Q:
                u = u - (q @ u) * q
        Q.append(u / np.linalg.norm(u))
    for k in (1, 2, 3, 5):
        p, hist = oracle.vp_solve(g, v, geo, w, dres, p0, eps, niter=k)
        Qk = np.stack(Q[:k], axis=1)
        y = np.linalg.solve(Qk.T @ H @ Qk, Qk.T @ r0)
        pk = p0.ravel() + Qk @ y
        assert np.linalg.norm(p.ravel() - pk) <= 1e-8 * np.linalg.norm(pk), k
        assert abs(hist[-1] - phi_dense(g, B, dres, eps, pk)) <= 1e-10 * hist[0], k
        assert abs(hist[0] - phi_dense(g, B, dres, eps, p0.ravel())) <= 1e-12 * hist[0]
        assert all(b <= a * (1 + 1e-13) for a, b in zip(hist, hist[1:]))   # CG never increases Phi


def test_cg_reaches_the_dense_solution_when_well_conditioned():
    g, v, geo, w, B, dres, eps = vp_case(eps_scale=2.0)
    H = dense_H(g, B, eps)
    pstar = np.linalg.solve(H, B.T @ dres.ravel())
    p, hist = oracle.vp_solve(g, v, geo, w, dres, np.zeros((g.nh, g.nz, g.nx)), eps, niter=25)
    assert np.linalg.norm(p.ravel() - pstar) <= 1e-9 * np.linalg.norm(pstar)
    # at the minimiser Phi = 1/2 ||dres||^2 - 1/2 b.p*  (normal equations)
    b = B.T @ dres.ravel()
    assert abs(hist[-1] - (0.5 * dres.ravel() @ dres.ravel() - 0.5 * b @ pstar)) <= 1e-9 * hist[0]


def test_zero_residual_keeps_zero_extension():
    g, v, geo, w, B, dres, eps = vp_case()
    p, hist = oracle.vp_solve(g, v, geo, w, np.zeros_like(dres), np.zeros((g.nh, g.nz, g.nx)), eps, niter=3)
    assert not p.any() and hist == [0.0] * 4
