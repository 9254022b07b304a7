"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/fwime.h declares.  Only host-side paths are called here (no GPU needed):
error strings, workspace sizing and argument validation."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2206_02362_gb300 as fw

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fwime_[a-z_]+)\s*\(", src))
    return sorted(names)


def test_library_builds_and_exports_every_declared_symbol():
    lib = fw.load()
    decl = declared_functions()
    assert len(decl) >= 16
    for name in decl:
        assert hasattr(lib, name), name
    assert set(fw.ABI_FUNCTIONS) <= set(decl)


def test_library_is_built_for_sm_103a_only():
    from paper_2206_02362_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.getsize(fw.lib_path()) > 0


def test_strerror():
    assert fw.strerror(0) == "ok"
    assert "invalid" in fw.strerror(fw.FWIME_EINVAL)
    assert "CFL" in fw.strerror(fw.FWIME_ECFL)


def tiny_grid(**kw):
    base = dict(nz=20, nx=30, sponge=6, nt=50, dt=1e-3, dx=10.0, nh=5)
    base.update(kw)
    return fw.Grid(**base)


def geom(nx=30):
    return fw.Geometry(np.array([2]), np.array([5]), np.full(nx, 1), np.arange(nx))


def test_workspace_bytes_grows_with_shots_and_operator():
    g = tiny_grid()
    gm = fw.Geometry(np.array([2, 2, 2]), np.array([5, 10, 15]), np.full(30, 1), np.arange(30))
    f1 = fw.workspace_bytes(g, gm, fw.OP_FORWARD, 1)
    f3 = fw.workspace_bytes(g, gm, fw.OP_FORWARD, 3)
    assert f3 > f1
    NZ, NXP = 20 + 2 * 10, 64
    assert f3 - f1 == 2 * 2 * NZ * NXP * 4          # two wavefields (q^n, q^n-1) per extra shot
    assert fw.workspace_bytes(g, gm, fw.OP_GRADIENT, 1) > fw.workspace_bytes(g, gm, fw.OP_BORN_EXT_ADJ, 1)
    # checkpoint count follows the segment length
    a = fw.workspace_bytes(g, gm, fw.OP_BORN_EXT_ADJ, 1, 7)
    b = fw.workspace_bytes(g, gm, fw.OP_BORN_EXT_ADJ, 1, 49)
    assert a != b


@pytest.mark.parametrize("bad", [dict(nh=4), dict(nh=0), dict(nt=1), dict(dx=0.0), dict(sponge=-1),
                                 dict(nh=203), dict(nz=0)])
def test_create_rejects_bad_grids_before_touching_the_gpu(bad):
    lib = fw.load()
    g = tiny_grid(**bad).c()
    gm, keep = geom().c()
    h = ctypes.c_void_p()
    assert lib.fwime_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(gm), 0, None) == fw.FWIME_EINVAL
    assert not h.value


@pytest.mark.parametrize("src,rec", [((20, 5), (1, 0)), ((2, 30), (1, 0)), ((2, 5), (1, 30)), ((-1, 5), (1, 0))])
def test_create_rejects_geometry_outside_the_grid(src, rec):
    lib = fw.load()
    g = tiny_grid().c()
    gm, keep = fw.Geometry(np.array([src[0]]), np.array([src[1]]), np.array([rec[0]]), np.array([rec[1]])).c()
    h = ctypes.c_void_p()
    assert lib.fwime_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(gm), 0, None) == fw.FWIME_EINVAL


def test_null_arguments():
    lib = fw.load()
    assert lib.fwime_create(None, None, None, 0, None) == fw.FWIME_EINVAL
    assert lib.fwime_forward(None, None, None, None) == fw.FWIME_EINVAL
    assert lib.fwime_sync(None) == fw.FWIME_EINVAL
    lib.fwime_destroy(None)
