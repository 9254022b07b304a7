"""The request server's host side, through the C ABI and without a GPU: a server
context is created with an explicit memory budget; fwime_submit refuses a
request that alone needs more than the budget (FWIME_ENOMEM, with a message)
and malformed requests (FWIME_EINVAL) before anything is queued; unknown
tickets and operator calls on a server context are refused; fwime_request_bytes
counts the operator's workspace plus host-I/O staging."""
import ctypes

import numpy as np
import pytest

import paper_2206_02362_gb300 as fw


def request(kind=fw.REQ_FORWARD, nz=40, nx=80, nt=100, nh=1, nshot=1, host_io=1):
    grid = fw.Grid(nz=nz, nx=nx, sponge=10, nt=nt, dt=1e-3, dx=10.0, nh=nh)
    geom = fw.Geometry(np.full(nshot, 2), 5 + np.arange(nshot), np.full(20, 2), 2 * np.arange(20))
    gm, keep = geom.c()
    buf = ctypes.c_void_p(16)          # never dereferenced: the requests below are refused or only sized
    grad = kind == fw.REQ_GRADIENT
    c = fw.RequestC(kind, grid.c(), gm, host_io, buf, buf, buf if grad else None, buf if grad else None,
                    None if grad else buf, buf if grad else None, ctypes.c_float(0.0))
    return c, keep, grid, geom


def last_error(lib):
    b = ctypes.create_string_buffer(256)
    lib.fwime_server_last_error(b, 256)
    return b.value.decode()


@pytest.fixture
def server():
    lib = fw.load()
    h = ctypes.c_void_p()
    assert lib.fwime_server_create(ctypes.byref(h), ctypes.c_size_t(4 << 20), 4, 0) == fw.FWIME_OK
    yield lib, h
    lib.fwime_destroy(h)          # nothing queued: returns at once


def test_request_bytes_counts_workspace_and_staging():
    lib = fw.load()
    for kind, op in ((fw.REQ_FORWARD, fw.OP_FORWARD), (fw.REQ_GRADIENT, fw.OP_GRADIENT)):
        dev, keep, grid, geom = request(kind, host_io=0, nh=3)
        host, keep2, _, _ = request(kind, host_io=1, nh=3)
        a, b = ctypes.c_size_t(0), ctypes.c_size_t(0)
        assert lib.fwime_request_bytes(ctypes.byref(dev), ctypes.byref(a)) == fw.FWIME_OK
        assert lib.fwime_request_bytes(ctypes.byref(host), ctypes.byref(b)) == fw.FWIME_OK
        ws = fw.workspace_bytes(grid, geom, op, geom.nshot)
        assert a.value == ws + (1 << 20)
        nm, nd, nw = grid.nz * grid.nx, geom.nshot * grid.nt * geom.nrec, geom.nshot * grid.nt
        al = lambda n: (n + 63) // 64 * 64  # noqa: E731
        stage = al(nm) + al(nw) + al(nd) + (al(grid.nh * nm) + al(nm) if kind == fw.REQ_GRADIENT else 0)
        assert b.value - a.value == 4 * stage


def test_submit_refuses_a_request_beyond_the_budget(server):
    lib, h = server
    c, keep, _, _ = request(nz=400, nx=800, nt=2000)     # far more than 4 MB of workspace
    t = ctypes.c_uint64(0)
    assert lib.fwime_submit(h, ctypes.byref(c), ctypes.byref(t)) == fw.FWIME_ENOMEM
    assert "budget" in last_error(lib)
    assert lib.fwime_sync(h) == fw.FWIME_OK                # nothing was queued


@pytest.mark.parametrize("bad", ["kind", "nh", "geometry", "buffer", "eps"])
def test_submit_refuses_malformed_requests(server, bad):
    lib, h = server
    c, keep, _, _ = request(fw.REQ_GRADIENT, nh=3)
    if bad == "kind":
        c.kind = 7
    elif bad == "nh":
        c.grid.nh = 4
    elif bad == "geometry":
        keep[2][0] = 500                                   # receiver below the grid
    elif bad == "buffer":
        c.dobs = None
    else:
        c.eps = -1.0
    t = ctypes.c_uint64(0)
    assert lib.fwime_submit(h, ctypes.byref(c), ctypes.byref(t)) == fw.FWIME_EINVAL


def test_unknown_tickets_and_operator_calls_are_refused(server):
    lib, h = server
    r = fw.ResultC()
    assert lib.fwime_poll(h, ctypes.c_uint64(12345), ctypes.byref(r)) == fw.FWIME_EINVAL
    assert lib.fwime_wait(h, ctypes.c_uint64(12345), ctypes.byref(r)) == fw.FWIME_EINVAL
    assert lib.fwime_forward(h, ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16)) == fw.FWIME_EINVAL
    assert lib.fwime_set_option(h, fw.OPT_SEGMENT, 8) == fw.FWIME_EINVAL


def test_server_create_rejects_bad_arguments():
    lib = fw.load()
    h = ctypes.c_void_p()
    assert lib.fwime_server_create(ctypes.byref(h), ctypes.c_size_t(1 << 20), 0, 0) == fw.FWIME_EINVAL
    assert lib.fwime_server_create(ctypes.byref(h), ctypes.c_size_t(1 << 20), 4, 8) == fw.FWIME_EINVAL
    assert lib.fwime_server_create(None, ctypes.c_size_t(1 << 20), 4, 0) == fw.FWIME_EINVAL
