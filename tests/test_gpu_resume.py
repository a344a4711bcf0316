"""Checkpoint and resume: a run continued from a state read with
dg_get_state and written back with dg_set_state (into the same solver or a
new one) is bit for bit the uninterrupted run, in both precision forms.

The double Mach reflection (P2, moving-shock top boundary) limits cells in
every stage, including the last stage of the step before the checkpoint, and
a run to an end time ends on a step clamped to it: both are the cases where
the stage result's traces or exterior time could differ from those a resumed
run recomputes from the stored state.
"""
import numpy as np
import pytest

from paper_2409_09620_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    from paper_2409_09620_gb300 import native
    native.lib()
    return native


@pytest.mark.parametrize("precision", [0, 1])
def test_resume_after_limited_stages_is_bitwise(N, precision):
    wl = W.dmr_workload(nx=96, ny=24, k=2)
    mesh = N.Mesh.from_mesh(wl.mesh)
    u0 = N.initial_state(mesh, wl)
    cfg = N.config_for(wl, precision=precision)
    a = N.Solver(mesh, cfg, u0)
    st, _ = a.advance(1e30, max_steps=6)
    assert st["limited_cells"] > 0
    u, t = a.get_state()
    b = N.Solver(mesh, cfg, u0)
    b.set_state(u, t)
    a.set_state(*a.get_state())            # the same solver, written back onto itself
    c = N.Solver(mesh, cfg, u0)
    c.advance(1e30, max_steps=6)           # uninterrupted
    sa, _ = a.advance(1e30, max_steps=10)
    sb, _ = b.advance(1e30, max_steps=10)
    sc, _ = c.advance(1e30, max_steps=10)
    assert sc["limited_cells"] > 0
    ua, ta = a.get_state()
    ub, tb = b.get_state()
    uc, tc = c.get_state()
    assert ta == tb == tc
    assert np.array_equal(ua, uc) and np.array_equal(ub, uc)


@pytest.mark.parametrize("precision", [0, 1])
def test_resume_after_a_step_clamped_to_the_end_time(N, precision):
    wl = W.dmr_workload(nx=96, ny=24, k=2)
    mesh = N.Mesh.from_mesh(wl.mesh)
    u0 = N.initial_state(mesh, wl)
    cfg = N.config_for(wl, precision=precision)
    a = N.Solver(mesh, cfg, u0)
    t1 = 2.37e-4                           # not a multiple of the step: the last step is clamped
    st, _ = a.advance(t1)
    u, t = a.get_state()
    assert t == t1 and st["steps"] > 1
    b = N.Solver(mesh, cfg, u0)
    b.set_state(u, t)
    sa, _ = a.advance(6.0e-4)
    sb, _ = b.advance(6.0e-4)
    ua, ta = a.get_state()
    ub, tb = b.get_state()
    assert ta == tb == 6.0e-4 and sa["steps"] == sb["steps"]
    assert np.array_equal(ua, ub)
