"""GPU test of dg_stats_noalloc, the statistics entry point for callers that
cannot allocate device memory when they call (their memory is reserved by
their own pool allocator, or their loop must not pay for an allocation).

It is checked through the C ABI against the existing entry point dg_op_stats
on two calls in a row: a larger P2 mesh, then a smaller P1 mesh, so the second
call runs on scratch that still holds the first call's partial results.  This
file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2409_09620_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _case(N, wl, seed):
    mesh = N.Mesh.from_mesh(wl.mesh)
    u = N.initial_state(mesh, wl)
    rng = np.random.default_rng(seed)
    u[:, 1:, :] += 0.05 * np.abs(u[:, :1, :]) * rng.uniform(-1, 1, u[:, 1:, :].shape)
    solver = N.Solver(mesh, N.config_for(wl), u)
    expect = solver.op_stats(u)            # the existing entry point (allocating solver path)
    return mesh, u, expect


def test_stats_noalloc_matches_existing_entry_point():
    torch = pytest.importorskip("torch")
    from paper_2409_09620_gb300 import native as N
    lib = N.lib()
    cases = [(W.sedov_workload(n=40, k=2), 2, 11),      # 3200 cells: 25 blocks
             (W.vortex_workload(n=9, k=1), 1, 12)]       # 162 cells: 2 blocks (stale slots beyond)
    for wl, k, seed in cases:
        mesh, u, expect = _case(N, wl, seed)
        dev_u = torch.from_numpy(np.ascontiguousarray(u)).cuda()
        out = torch.full((10,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        rc = lib.dg_stats_noalloc(mesh.h, k, ctypes.c_void_p(dev_u.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                  None)
        assert rc == 0, lib.dg_last_error().decode()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got[:4], expect[:4], rtol=1e-12, atol=1e-15 * np.abs(expect[:4]).max())
        np.testing.assert_allclose(got[4:], expect[4:], rtol=1e-12)


def test_stats_noalloc_rejects_bad_arguments():
    from paper_2409_09620_gb300 import native as N
    lib = N.lib()
    mesh = N.Mesh.from_mesh(W.vortex_workload(n=4, k=1).mesh)
    assert lib.dg_stats_noalloc(mesh.h, 3, ctypes.c_void_p(1), ctypes.c_void_p(1), None) == N.DG_EINVAL
    assert lib.dg_stats_noalloc(mesh.h, 1, None, None, None) == N.DG_EINVAL


def test_stats_noalloc_on_a_caller_stream():
    """The work goes to the caller's stream: a torch stream's handle is passed
    and only that stream is synchronised before the result is read."""
    torch = pytest.importorskip("torch")
    from paper_2409_09620_gb300 import native as N
    lib = N.lib()
    mesh, u, expect = _case(N, W.riemann4_workload(n=12, k=2), 13)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        dev_u = torch.from_numpy(np.ascontiguousarray(u)).to("cuda", non_blocking=False)
        out = torch.full((10,), float("nan"), dtype=torch.float64, device="cuda")
    stream.synchronize()
    rc = lib.dg_stats_noalloc(mesh.h, 2, ctypes.c_void_p(dev_u.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                              ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, lib.dg_last_error().decode()
    stream.synchronize()
    got = out.cpu().numpy()
    np.testing.assert_allclose(got[:4], expect[:4], rtol=1e-12, atol=1e-15 * np.abs(expect[:4]).max())
    np.testing.assert_allclose(got[4:], expect[4:], rtol=1e-12)


def test_stats_noalloc_rejects_meshes_larger_than_its_scratch():
    """A mesh of 4,196,352 cells (just over the 4,194,304-cell limit of the
    fixed scratch) is refused with DG_EINVAL before anything is launched; the
    output buffer keeps its contents."""
    torch = pytest.importorskip("torch")
    from paper_2409_09620_gb300 import native as N
    lib = N.lib()
    grid = W.jittered_grid(2049, 1024, seed=3)
    assert grid.nt == 4196352
    mesh = N.Mesh.from_mesh(grid)
    dev_u = torch.zeros((4, 3, grid.nt), dtype=torch.float64, device="cuda")
    out = torch.full((10,), 7.0, dtype=torch.float64, device="cuda")
    rc = lib.dg_stats_noalloc(mesh.h, 1, ctypes.c_void_p(dev_u.data_ptr()), ctypes.c_void_p(out.data_ptr()), None)
    assert rc == N.DG_EINVAL
    assert b"4194304" in lib.dg_last_error()
    torch.cuda.synchronize()
    assert (out.cpu().numpy() == 7.0).all()
