"""FP64 CPU oracle for the FWIME operators -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``fwime_oracle.c`` (plain C,
double precision, sequential loops) through ctypes and shares no code with the
CUDA path in ``paper_2206_02362_gb300``.

Operators (Barnier et al., Theory section): ``forward`` = f(m) (Eq. 1),
``born``/``born_adj`` = B, B* (Eq. 8), ``born_ext``/``born_ext_adj`` = B~, B~*
(Eqs. 1-2; subsurface-offset extension, or the time-lag extension when
``Grid.lag`` > 0), ``tomo``/``tomo_adj`` = T, T* (Eq. 9),
``gradient`` = (Phi at fixed p~, B* r + T* r) (Eqs. 1, 7-9), ``vp_solve`` =
linear conjugate gradients for the variable projection step (Eqs. 2-5),
``spline``/``spline_adj`` = the linear spline re-parametrisation S, S* (Eq. 1),
``spline_refine`` = the model-space multiscale step (coarse to fine spline nodes),
``cost_fwime`` = Eq. 11.  Primitives (``lap``, ``step``, ``step_T``, ``prop``, ``prop_T``,
``d2t``, ``d2t_T``, ``scatter``, ``scatter_TD``, ``scatter_TW``) are exposed
for dot-product pins.

Parity unpinned: the DSO weights of ``dso_penalty`` (a reading of the
invertible, modified DSO operator of the Theory section; only its arithmetic is pinned).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fwime_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libfwime_oracle.so")

OP_FWD, OP_BORN, OP_BORN_ADJ, OP_EXT, OP_EXT_ADJ, OP_TOMO, OP_TOMO_ADJ, OP_GRAD = range(8)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fast-math, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Grid(ctypes.Structure):
    _fields_ = [("nz", ctypes.c_int), ("nx", ctypes.c_int), ("W", ctypes.c_int),
                ("nt", ctypes.c_int), ("nh", ctypes.c_int),
                ("dz", ctypes.c_double), ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("lag", ctypes.c_int),
                ("fs", ctypes.c_int)]


class _Shot(ctypes.Structure):
    _fields_ = [("src_iz", ctypes.c_int), ("src_ix", ctypes.c_int),
                ("w", ctypes.POINTER(ctypes.c_double)), ("nrec", ctypes.c_int),
                ("rec_iz", ctypes.POINTER(ctypes.c_int)), ("rec_ix", ctypes.POINTER(ctypes.c_int))]


_lib = None


def _L():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        D = ctypes.POINTER(ctypes.c_double)
        G = ctypes.POINTER(_Grid)
        _lib.og_shots.restype = ctypes.c_double
        _lib.og_gradient.restype = ctypes.c_double
        _lib.og_dso_penalty.restype = ctypes.c_double
        _lib.og_dso_penalty.argtypes = [G, D, ctypes.c_double]
        _lib.og_cost_vp.restype = ctypes.c_double
        _lib.og_cost_vp.argtypes = [ctypes.c_int, ctypes.c_double]
        _lib.og_cost_fwime.restype = ctypes.c_double
        _lib.og_cost_fwime.argtypes = [ctypes.c_int, ctypes.c_double]
    return _lib


@dataclass(frozen=True)
class Grid:
    """Physical grid nz x nx at spacing dz, dx; sponge W points; nt samples at dt; nh extension points:
    subsurface offsets (lag = 0) or time lags spaced lag * dt (lag > 0); fs = 1: free surface (pressure
    release) at the top physical row instead of a sponge."""
    nz: int
    nx: int
    W: int
    nt: int
    dt: float
    dx: float
    dz: float | None = None
    nh: int = 1
    lag: int = 0
    fs: int = 0

    @property
    def NZ(self) -> int:
        return self.nz + 2 * (self.W + 4)

    @property
    def NX(self) -> int:
        return self.nx + 2 * (self.W + 4)

    @property
    def pad(self) -> int:
        return self.W + 4

    def c(self) -> _Grid:
        dz = self.dx if self.dz is None else self.dz
        return _Grid(self.nz, self.nx, self.W, self.nt, self.nh, float(dz), float(self.dx), float(self.dt), self.lag, self.fs)


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _P(g: Grid) -> int:
    return g.NZ * g.NX


# ----------------------------------------------------------------- primitives

def prep(g: Grid, v):
    v, pv = _d(v)
    c = np.zeros((g.NZ, g.NX)); gam = np.zeros((g.NZ, g.NX)); b = np.zeros((g.nz, g.nx))
    _L().og_prep(ctypes.byref(g.c()), pv, _d(c)[1], _d(gam)[1], _d(b)[1])
    return c, gam, b


def lap(g: Grid, q):
    q, pq = _d(q)
    out = np.zeros((g.NZ, g.NX))
    _L().og_lap(ctypes.byref(g.c()), pq, _d(out)[1])
    return out


def step(g: Grid, c, gam, qc, qp, s):
    args = [_d(a) for a in (c, gam, qc, qp, s)]
    qn = np.zeros((g.NZ, g.NX))
    _L().og_step(ctypes.byref(g.c()), *[a[1] for a in args], _d(qn)[1])
    return qn


def step_T(g: Grid, c, gam, qn_s):
    args = [_d(a) for a in (c, gam, qn_s)]
    outs = [np.zeros((g.NZ, g.NX)) for _ in range(3)]
    _L().og_step_T(ctypes.byref(g.c()), *[a[1] for a in args], *[_d(o)[1] for o in outs])
    return tuple(outs)


def prop(g: Grid, c, gam, s_seq):
    args = [_d(a) for a in (c, gam, s_seq)]
    q = np.zeros((g.nt, g.NZ, g.NX))
    _L().og_prop(ctypes.byref(g.c()), *[a[1] for a in args], _d(q)[1])
    return q


def prop_T(g: Grid, c, gam, a_seq):
    args = [_d(a) for a in (c, gam, a_seq)]
    s = np.zeros((g.nt - 1, g.NZ, g.NX))
    _L().og_prop_T(ctypes.byref(g.c()), *[a[1] for a in args], _d(s)[1])
    return s


def d2t(g: Grid, q_seq):
    q_seq, pq = _d(q_seq)
    D = np.zeros((g.nt - 1, g.NZ, g.NX))
    _L().og_d2t(ctypes.byref(g.c()), pq, _d(D)[1])
    return D


def d2t_T(g: Grid, z_seq):
    z_seq, pz = _d(z_seq)
    a = np.zeros((g.nt, g.NZ, g.NX))
    _L().og_d2t_T(ctypes.byref(g.c()), pz, _d(a)[1])
    return a


def scatter(g: Grid, Wt, D):
    Wt, pw = _d(Wt); D, pD = _d(D)
    e = np.zeros((g.NZ, g.NX))
    _L().og_scatter(ctypes.byref(g.c()), pw, pD, _d(e)[1])
    return e


def scatter_TD(g: Grid, Wt, es):
    Wt, pw = _d(Wt); es, pe = _d(es)
    z = np.zeros((g.NZ, g.NX))
    _L().og_scatter_TD(ctypes.byref(g.c()), pw, pe, _d(z)[1])
    return z


def scatter_TW(g: Grid, D, es):
    D, pD = _d(D); es, pe = _d(es)
    Ws = np.zeros((g.nh, g.nz, g.nx))
    _L().og_scatter_TW_acc(ctypes.byref(g.c()), pD, pe, _d(Ws)[1])
    return Ws


# ------------------------------------------------------------------ operators

@dataclass
class Geometry:
    """Point sources (one per shot) and a fixed receiver spread, physical grid indices."""
    src_iz: np.ndarray
    src_ix: np.ndarray
    rec_iz: np.ndarray
    rec_ix: np.ndarray

    @property
    def nshot(self) -> int:
        return int(len(self.src_iz))

    @property
    def nrec(self) -> int:
        return int(len(self.rec_iz))


def _shots(g: Grid, op: int, v, geo: Geometry, w, in1=None, in2=None, out_shape=None, nthreads=None):
    if nthreads is None:
        nthreads = min(os.cpu_count() or 1, geo.nshot)
    v, pv = _d(v)
    w = np.broadcast_to(np.asarray(w, dtype=np.float64), (geo.nshot, g.nt))
    w, pw = _d(w)
    si, psi = _i(geo.src_iz); sx, psx = _i(geo.src_ix)
    ri, pri = _i(geo.rec_iz); rx, prx = _i(geo.rec_ix)
    keep = []
    p1 = p2 = None
    if in1 is not None:
        a, p1 = _d(in1); keep.append(a)
    if in2 is not None:
        a, p2 = _d(in2); keep.append(a)
    out = np.zeros(out_shape)
    J = _L().og_shots(ctypes.byref(g.c()), ctypes.c_int(op), pv, ctypes.c_int(geo.nshot), psi, psx, pw,
                      ctypes.c_int(geo.nrec), pri, prx, p1, p2, _d(out)[1], ctypes.c_int(nthreads))
    return out, J


def forward(g: Grid, v, geo: Geometry, w, nthreads=None):
    """f(m): data d[nshot][nt][nrec]."""
    return _shots(g, OP_FWD, v, geo, w, out_shape=(geo.nshot, g.nt, geo.nrec), nthreads=nthreads)[0]


def born(g: Grid, v, geo: Geometry, w, dv, nthreads=None):
    """B(m) dv."""
    return _shots(g, OP_BORN, v, geo, w, in1=dv, out_shape=(geo.nshot, g.nt, geo.nrec), nthreads=nthreads)[0]


def born_adj(g: Grid, v, geo: Geometry, w, d, nthreads=None):
    """B*(m) d, summed over shots: [nz][nx]."""
    return _shots(g, OP_BORN_ADJ, v, geo, w, in2=d, out_shape=(g.nz, g.nx), nthreads=nthreads)[0]


def born_ext(g: Grid, v, geo: Geometry, w, pt, nthreads=None):
    """B~(m) p~ with p~[nh][nz][nx]."""
    return _shots(g, OP_EXT, v, geo, w, in1=pt, out_shape=(geo.nshot, g.nt, geo.nrec), nthreads=nthreads)[0]


def born_ext_adj(g: Grid, v, geo: Geometry, w, d, nthreads=None):
    """B~*(m) d, summed over shots: [nh][nz][nx]."""
    return _shots(g, OP_EXT_ADJ, v, geo, w, in2=d, out_shape=(g.nh, g.nz, g.nx), nthreads=nthreads)[0]


def tomo(g: Grid, v, geo: Geometry, w, pt, dv, nthreads=None):
    """T(m, p~) dv."""
    return _shots(g, OP_TOMO, v, geo, w, in1=pt, in2=dv, out_shape=(geo.nshot, g.nt, geo.nrec),
                  nthreads=nthreads)[0]


def tomo_adj(g: Grid, v, geo: Geometry, w, pt, d, nthreads=None):
    """T*(m, p~) d, summed over shots: [nz][nx]."""
    return _shots(g, OP_TOMO_ADJ, v, geo, w, in1=pt, in2=d, out_shape=(g.nz, g.nx), nthreads=nthreads)[0]


def gradient(g: Grid, v, geo: Geometry, w, pt, dobs, eps: float = 0.0, nthreads=None):
    """(Phi, grad): Phi = 1/2||f + B~p~ - d||^2 + eps^2/2||D p~||^2, grad = B* r + T* r."""
    grad, J = _shots(g, OP_GRAD, v, geo, w, in1=pt, in2=dobs, out_shape=(g.nz, g.nx), nthreads=nthreads)
    return J + dso_penalty(g, pt, eps), grad


def dso_penalty(g: Grid, pt, eps: float) -> float:
    pt, pp = _d(pt)
    return float(_L().og_dso_penalty(ctypes.byref(g.c()), pp, ctypes.c_double(eps)))


def cost_vp(n_vp: int, c_ext: float) -> float:
    """Eq. 10: C_vp = 4 N_vp (1 + C_ext)."""
    return float(_L().og_cost_vp(int(n_vp), float(c_ext)))


def cost_fwime(n_vp: int, c_ext: float) -> float:
    """Eq. 11: C_FWIME = 6 + 4 N_vp (1 + C_ext)."""
    return float(_L().og_cost_fwime(int(n_vp), float(c_ext)))


def dso_weights(g: Grid):
    """Diagonal of D on p~[nh][nz][nx]: |ih - (nh-1)/2| + 1 per offset plane (the reading used by dso_penalty)."""
    hm = (g.nh - 1) // 2
    return (np.abs(np.arange(g.nh) - hm) + 1.0)[:, None, None]


def vp_objective(g: Grid, v, geo: Geometry, w, dres, pt, eps: float) -> float:
    """Phi_eps,m(p~) = 1/2 ||B~(m) p~ - dres||^2 + eps^2/2 ||D p~||^2 with dres = d_obs - f(m) (Eq. 2)."""
    r = born_ext(g, v, geo, w, pt) - np.asarray(dres, dtype=np.float64)
    return 0.5 * float(np.sum(r * r)) + 0.5 * eps * eps * float(np.sum((dso_weights(g) * pt) ** 2))


def vp_solve(g: Grid, v, geo: Geometry, w, dres, pt0, eps: float, niter: int):
    """Variable projection step (Eqs. 2-5): niter iterations of linear conjugate gradients on the normal
    equations H p~ = B~* dres, H = B~* B~ + eps^2 D* D, started at pt0.  Textbook CG (Hestenes-Stiefel):
    r = b - H p, d = r; per iteration alpha = r.r / d.Hd, p += alpha d, r -= alpha Hd,
    beta = r'.r' / r.r, d = r' + beta d.  Returns (p~, [Phi at p_0, ..., p_niter]) with every Phi
    evaluated directly from its definition."""
    v = np.asarray(v, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    dres = np.asarray(dres, dtype=np.float64)
    D2 = dso_weights(g) ** 2 * (eps * eps)

    def H(q):
        return born_ext_adj(g, v, geo, w, born_ext(g, v, geo, w, q)) + D2 * q

    p = np.array(pt0, dtype=np.float64)
    r = born_ext_adj(g, v, geo, w, dres) - H(p)
    d = r.copy()
    rr = float(np.sum(r * r))
    hist = [vp_objective(g, v, geo, w, dres, p, eps)]
    for _ in range(niter):
        Hd = H(d)
        dHd = float(np.sum(d * Hd))
        alpha = rr / dHd if dHd > 0 else 0.0
        p = p + alpha * d
        r = r - alpha * Hd
        rr_new = float(np.sum(r * r))
        beta = rr_new / rr if rr > 0 else 0.0
        d = r + beta * d
        rr = rr_new
        hist.append(vp_objective(g, v, geo, w, dres, p, eps))
    return p, hist


def spline_matrix(nodes, coords):
    """Dense [len(coords)][len(nodes)] matrix of the 1-D linear spline (hat) functions on the strictly
    increasing `nodes`, evaluated at `coords`: a point between nodes k and k+1 takes 1-a and a,
    a = (c - node_k) / (node_k+1 - node_k); points beyond the end nodes take the end node's value."""
    nodes = np.asarray(nodes, dtype=np.float64)
    A = np.zeros((len(coords), len(nodes)))
    for i, c in enumerate(np.asarray(coords, dtype=np.float64)):
        if len(nodes) == 1 or c <= nodes[0]:
            A[i, 0] = 1.0
        elif c >= nodes[-1]:
            A[i, -1] = 1.0
        else:
            k = int(np.searchsorted(nodes, c, side="right")) - 1
            a = (c - nodes[k]) / (nodes[k + 1] - nodes[k])
            A[i, k] = 1.0 - a
            A[i, k + 1] = a
    return A


def spline(zs, xs, nz, nx, dz, dx, m):
    """S m (Theory section, Eq. 1: v = S m): the model on the spline grid of node coordinates zs x xs
    (metres) interpolated bilinearly onto the physical grid [nz][nx] at spacing dz, dx."""
    Az = spline_matrix(zs, np.arange(nz) * dz)
    Ax = spline_matrix(xs, np.arange(nx) * dx)
    return Az @ np.asarray(m, dtype=np.float64) @ Ax.T


def spline_adj(zs, xs, nz, nx, dz, dx, g):
    """S* g: a field on the physical grid mapped to the spline nodes (the transpose of `spline`)."""
    Az = spline_matrix(zs, np.arange(nz) * dz)
    Ax = spline_matrix(xs, np.arange(nx) * dx)
    return Az.T @ np.asarray(g, dtype=np.float64) @ Ax


def spline_refine(zc, xc, mc, zf, xf):
    """Model-space multiscale step (Theory section, the model-space multi-scale workflow after Eq. 9; the
    Marmousi2 section halves the spline spacing when the step-length search fails): the model mc on the
    coarse nodes zc x xc carried over to the fine nodes zf x xf as the coarse linear spline evaluated at
    the fine nodes, Az(zf) mc Ax(xf)^T with the hat-function matrices of `spline_matrix`."""
    Az = spline_matrix(zc, np.asarray(zf, dtype=np.float64))
    Ax = spline_matrix(xc, np.asarray(xf, dtype=np.float64))
    return Az @ np.asarray(mc, dtype=np.float64) @ Ax.T
