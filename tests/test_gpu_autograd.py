"""The differentiable FWIME objective (Eq. 1 at fixed p~, gradient Eqs. 7-9):
torch.autograd forward = the forward sweep alone, backward = B* r + T* r from
the hand-written adjoint kernels, checked against the FP64 oracle gradient,
against central finite differences of the objective along 10 random smooth
model perturbations, and by kernel-family launch counts (no adjoint kernel in
the forward pass)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_2206_02362_gb300 as fw  # noqa: E402
from paper_2206_02362_gb300.autograd import fwime_objective  # noqa: E402

pytestmark = pytest.mark.gpu


class Problem:
    """North-Sea-shaped in miniature: flat layers with a fast chalk layer, a 1-D trend as the
    current model, 4 shots, nh=7 offsets, checkpoint segments of 16 steps."""

    def __init__(self):
        self.nz, self.nx, self.W, self.nt, self.nh, self.dx, self.dt = 30, 120, 8, 220, 7, 12.5, 1e-3
        vt, v0 = synth.north_sea_like(self.nz, self.nx, self.dx)
        self.vtrue, self.v0 = vt, v0
        rng = np.random.default_rng(synth.SEED0 + 2)
        self.src_iz, self.src_ix = np.full(4, 1), np.array([5, 40, 80, 114])
        self.rec_iz, self.rec_ix = np.full(60, 1), 2 * np.arange(60)
        self.w = np.stack([synth.ricker(self.nt, self.dt, 15.0)] * 4).astype(np.float32)
        self.pt = (1e-4 * rng.standard_normal((self.nh, self.nz, self.nx))).astype(np.float32)
        og = oracle.Grid(nz=self.nz, nx=self.nx, W=self.W, nt=self.nt, dt=self.dt, dx=self.dx, nh=self.nh)
        self.og = og
        self.ogeo = oracle.Geometry(self.src_iz, self.src_ix, self.rec_iz, self.rec_ix)
        self.dobs = oracle.forward(og, vt.astype(np.float64), self.ogeo, self.w.astype(np.float64)).astype(np.float32)
        self.grid = fw.Grid(nz=self.nz, nx=self.nx, sponge=self.W, nt=self.nt, dt=self.dt, dx=self.dx, nh=self.nh)
        self.geom = fw.Geometry(self.src_iz, self.src_ix, self.rec_iz, self.rec_ix)
        self.eps = 1e-2


@pytest.fixture(scope="module")
def prob():
    assert torch.cuda.is_available()
    return Problem()


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_autograd_gradient_matches_oracle(prob):
    p = prob
    J_o, g_o = oracle.gradient(p.og, p.v0.astype(np.float64), p.ogeo, p.w.astype(np.float64),
                               p.pt.astype(np.float64), p.dobs.astype(np.float64), eps=p.eps)
    with fw.Context(p.grid, p.geom, segment=16) as ctx:
        v = cu(p.v0).requires_grad_(True)
        J = fwime_objective(ctx, v, cu(p.w), cu(p.pt), cu(p.dobs), p.eps)
        J.backward()
        g = v.grad.double().cpu().numpy()
        J_only = ctx.objective(cu(p.v0), cu(p.w), cu(p.pt), cu(p.dobs), eps=p.eps)
    assert abs(J.item() - J_o) <= 1e-5 * J_o
    assert abs(J_only - J_o) <= 1e-5 * J_o
    assert np.linalg.norm(g - g_o) / np.linalg.norm(g_o) <= 1e-4


def test_gradient_against_central_finite_differences(prob):
    """10 random smooth perturbations (zero on the edge ring), FP32 objective."""
    p = prob
    rng = np.random.default_rng(synth.SEED0 + 77)
    with fw.Context(p.grid, p.geom, segment=16) as ctx:
        v = cu(p.v0).requires_grad_(True)
        J = fwime_objective(ctx, v, cu(p.w), cu(p.pt), cu(p.dobs), p.eps)
        J.backward()
        g = v.grad.double().cpu().numpy()
        errs, rels = [], []
        gn = np.linalg.norm(g)
        for k in range(10):
            dv = synth.gaussian_blobs(p.nz, p.nx, rng, nblob=3, amp=1.0, sigma_pts=5.0, ring=1)
            e = 5.0
            jp = ctx.objective(cu(p.v0 + e * dv), cu(p.w), cu(p.pt), cu(p.dobs), eps=p.eps)
            jm = ctx.objective(cu(p.v0 - e * dv), cu(p.w), cu(p.pt), cu(p.dobs), eps=p.eps)
            fd = (jp - jm) / (2 * e)
            an = float((g * dv).sum())
            scale = gn * np.linalg.norm(dv)
            # error on the scale of a generic directional derivative; random smooth directions can be
            # almost orthogonal to the gradient, where FP32 noise in Phi swamps (fd - an) / an
            errs.append(abs(fd - an) / scale)
            if abs(an) > 1e-2 * scale:
                rels.append(abs(fd - an) / abs(an))
    assert max(errs) <= 1e-4, errs
    assert len(rels) >= 5 and max(rels) <= 2e-3, rels


def test_forward_runs_no_adjoint_kernel_and_backward_matches_oracle(prob):
    """Under requires_grad the forward pass runs the forward sweep only (the same stencil launches as
    the objective alone, no imaging launch); backward runs the adjoint sweep from the kept state and
    matches the oracle gradient, scaled by a non-scalar-shaped incoming gradient."""
    p = prob
    J_o, g_o = oracle.gradient(p.og, p.v0.astype(np.float64), p.ogeo, p.w.astype(np.float64),
                               p.pt.astype(np.float64), p.dobs.astype(np.float64), eps=p.eps)
    with fw.Context(p.grid, p.geom, segment=16, shots_per_batch=3, profile=1) as ctx:
        w, pt, dobs = cu(p.w), cu(p.pt), cu(p.dobs)
        ctx.objective(cu(p.v0), w, pt, dobs, eps=p.eps)
        obj = ctx.profile_read(reset=True)
        v = cu(p.v0).requires_grad_(True)
        J = fwime_objective(ctx, v, w, pt, dobs, p.eps)
        fwd = ctx.profile_read(reset=True)
        assert fwd["prop"]["launches"] == obj["prop"]["launches"]
        assert fwd["image"]["launches"] == 0
        J.reshape(1).backward(torch.tensor([2.0], dtype=torch.float64, device="cuda"))
        bwd = ctx.profile_read(reset=True)
        assert ctx.get_option("background_reused") == 1      # started from the kept state
        assert bwd["image"]["launches"] > 0
        # the adjoint half recomputes 2 fields and runs 2 adjoint fields: 4 stencil launches per step
        assert bwd["prop"]["launches"] == 4 * (p.nt - 1) * 2     # 2 batches of 3 and 1 shots
        g = v.grad.double().cpu().numpy() / 2.0
    assert abs(J.item() - J_o) <= 1e-5 * J_o
    assert np.linalg.norm(g - g_o) / np.linalg.norm(g_o) <= 1e-4


def test_backward_without_kept_state_recomputes(prob):
    """gradient_backward on pointers the forward half did not see runs the whole gradient."""
    p = prob
    J_o, g_o = oracle.gradient(p.og, p.v0.astype(np.float64), p.ogeo, p.w.astype(np.float64),
                               p.pt.astype(np.float64), p.dobs.astype(np.float64), eps=p.eps)
    with fw.Context(p.grid, p.geom, segment=16) as ctx:
        g = torch.zeros((p.nz, p.nx), device="cuda")
        ctx.gradient_backward(cu(p.v0), cu(p.w), cu(p.pt), cu(p.dobs), g, eps=p.eps)
        assert ctx.get_option("background_reused") == 0
        g2 = g.clone()                       # accumulate onto values of the gradient's own size
        v, w, pt, dobs = cu(p.v0), cu(p.w), cu(p.pt), cu(p.dobs)
        J = ctx.gradient_forward(v, w, pt, dobs, eps=p.eps)
        ctx.gradient_backward(v, w, pt, dobs, g2, eps=p.eps, accumulate=True)
        assert ctx.get_option("background_reused") == 1
    g, g2 = g.double().cpu().numpy(), g2.double().cpu().numpy()
    assert abs(J - J_o) <= 1e-5 * J_o
    assert np.linalg.norm(g - g_o) / np.linalg.norm(g_o) <= 1e-4
    assert np.linalg.norm(g2 - 2.0 * g_o) / np.linalg.norm(2.0 * g_o) <= 1e-4


def test_no_grad_path_runs_forward_sweep_only(prob):
    p = prob
    with fw.Context(p.grid, p.geom, segment=16) as ctx:
        with torch.no_grad():
            J = fwime_objective(ctx, cu(p.v0), cu(p.w), cu(p.pt), cu(p.dobs), p.eps)
        n_obj = ctx.launches
        grad = torch.zeros_like(cu(p.v0))
        ctx.gradient(cu(p.v0), cu(p.w), cu(p.pt), cu(p.dobs), grad, eps=p.eps)
        assert ctx.launches > 2 * n_obj      # the adjoint sweep was skipped
    assert J.item() > 0
