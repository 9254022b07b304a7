"""The allocation-free forward modelling entry point, fwime_forward_static.

It exists for callers that cannot allocate device memory (running inside another
allocator or memory pool, or on a thread that must not enter the driver's
allocator): it needs no context and takes its scratch from a static device
array.  Called through the C ABI twice in a row (two different models), its
output must match fwime_forward's within the parity tolerance and the FP64
oracle's f(m) within the same tolerance; a problem larger than the static array
must be refused with FWIME_ENOMEM and a message; a velocity that breaks the
stability bound or is not positive must be refused with FWIME_ECFL (output
untouched) and the next valid call must still be right."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_2206_02362_gb300 as fw  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _lib():
    lib = fw.load()
    vp = ctypes.c_void_p
    lib.fwime_forward_static.argtypes = [ctypes.POINTER(fw.GridC), ctypes.POINTER(fw.GeomC), vp, vp, vp, vp]
    lib.fwime_forward_static.restype = ctypes.c_int
    lib.fwime_static_scratch_bytes.argtypes = [ctypes.POINTER(fw.GridC), ctypes.POINTER(fw.GeomC)]
    lib.fwime_static_scratch_bytes.restype = ctypes.c_size_t
    lib.fwime_static_last_error.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
    lib.fwime_static_last_error.restype = ctypes.c_int
    return lib


def _case(seed):
    nz, nx, W, nt = 37, 150, 10, 200
    rng = np.random.default_rng(synth.SEED0 + 500 + seed)
    z = np.arange(nz)[:, None]
    v = (1800.0 + 20.0 * z + 100.0 * rng.random((nz, nx))).astype(np.float32)
    geom = fw.Geometry(np.array([1, 3, 0]), np.array([10, 75, 149]), np.full(50, 1), 3 * np.arange(50))
    grid = fw.Grid(nz=nz, nx=nx, sponge=W, nt=nt, dt=1e-3, dx=10.0, nh=1)
    w = np.stack([synth.ricker(nt, 1e-3, 20.0) * (1 + 0.1 * s) for s in range(3)]).astype(np.float32)
    return grid, geom, v, w


def test_forward_static_matches_forward_on_two_calls_in_a_row():
    assert torch.cuda.is_available()
    lib = _lib()
    for seed in (0, 1):
        grid, geom, v, w = _case(seed)
        vd, wd = torch.from_numpy(v).cuda(), torch.from_numpy(w).cuda()
        ref = torch.zeros((geom.nshot, grid.nt, geom.nrec), device="cuda")
        with fw.Context(grid, geom) as ctx:
            ctx.forward(vd, wd, ref)
        out = torch.full_like(ref, 7.0)            # stale values must be overwritten
        gc = grid.c()
        gm, keep = geom.c()
        assert lib.fwime_static_scratch_bytes(ctypes.byref(gc), ctypes.byref(gm)) <= 32 << 20
        rc = lib.fwime_forward_static(ctypes.byref(gc), ctypes.byref(gm), vd.data_ptr(), wd.data_ptr(),
                                      out.data_ptr(), None)
        assert rc == fw.FWIME_OK
        torch.cuda.synchronize()
        a, b = out.double().cpu().numpy(), ref.double().cpu().numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) <= TOL
        assert np.all(a[:, 0, :] == 0.0)
        og = oracle.Grid(nz=grid.nz, nx=grid.nx, W=grid.sponge, nt=grid.nt, dt=grid.dt, dx=grid.dx)
        ogeo = oracle.Geometry(geom.src_iz, geom.src_ix, geom.rec_iz, geom.rec_ix)
        d_ref = oracle.forward(og, v.astype(np.float64), ogeo, w.astype(np.float64))
        assert np.linalg.norm(a - d_ref) / np.linalg.norm(d_ref) <= TOL


def test_forward_static_refuses_problems_beyond_its_scratch():
    lib = _lib()
    grid = fw.Grid(nz=2000, nx=2000, sponge=50, nt=10, dt=1e-3, dx=10.0)   # ~68 MB of scratch
    geom = fw.Geometry(np.array([1]), np.array([1]), np.array([1]), np.array([2]))
    gc = grid.c()
    gm, keep = geom.c()
    assert lib.fwime_static_scratch_bytes(ctypes.byref(gc), ctypes.byref(gm)) > 32 << 20
    d = torch.zeros((1, 10, 1), device="cuda")
    v = torch.full((2000, 2000), 2000.0, device="cuda")
    w = torch.zeros((1, 10), device="cuda")
    rc = lib.fwime_forward_static(ctypes.byref(gc), ctypes.byref(gm), v.data_ptr(), w.data_ptr(), d.data_ptr(), None)
    assert rc == fw.FWIME_ENOMEM
    buf = ctypes.create_string_buffer(256)
    lib.fwime_static_last_error(buf, 256)
    assert b"scratch" in buf.value


def _static_call(lib, grid, geom, vd, wd, out):
    gc = grid.c()
    gm, keep = geom.c()
    rc = lib.fwime_forward_static(ctypes.byref(gc), ctypes.byref(gm), vd.data_ptr(), wd.data_ptr(), out.data_ptr(),
                                  None)
    torch.cuda.synchronize()
    return rc


@pytest.mark.parametrize("bad", ["cfl", "negative", "zero"])
def test_forward_static_refuses_unstable_or_non_positive_velocity(bad):
    lib = _lib()
    grid, geom, v, w = _case(0)
    vbad = v.copy()
    if bad == "cfl":
        # dt v sqrt(6.5016 (2 / dx^2)) >= 2 above v = 5547 m/s at dt = 1 ms, dx = 10 m
        vbad[20, 70] = 5600.0
    elif bad == "negative":
        vbad[5, 5] = -1800.0
    else:
        vbad[30, 140] = 0.0
    out = torch.full((geom.nshot, grid.nt, geom.nrec), 7.0, device="cuda")
    rc = _static_call(lib, grid, geom, torch.from_numpy(vbad).cuda(), torch.from_numpy(w).cuda(), out)
    assert rc == fw.FWIME_ECFL
    buf = ctypes.create_string_buffer(256)
    lib.fwime_static_last_error(buf, 256)
    assert b"CFL" in buf.value
    assert torch.all(out == 7.0)                     # no time step ran, the output is untouched
    # the next call with a valid model is unaffected by the refused one
    ref = torch.zeros_like(out)
    vd, wd = torch.from_numpy(v).cuda(), torch.from_numpy(w).cuda()
    with fw.Context(grid, geom) as ctx:
        ctx.forward(vd, wd, ref)
    assert _static_call(lib, grid, geom, vd, wd, out) == fw.FWIME_OK
    a, b = out.double().cpu().numpy(), ref.double().cpu().numpy()
    assert np.linalg.norm(a - b) / np.linalg.norm(b) <= TOL
