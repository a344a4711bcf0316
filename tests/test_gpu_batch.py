"""GPU tests of batches: independent ragged meshes (P1 and P2 mixed) advanced
together, by one launch per phase, by one persistent cooperative launch per
RK stage, or by the solves' own step kernels as parallel branches of one
graph.  Each solve of a batch must be bitwise identical to the same solve
advanced alone, for every launch form and any launch shape, with per-solve
end times, in FP64 and in the mixed form; and each solve must match the CPU
oracle advanced from the same state (FP64: 1e-9 relative after several
steps; mixed form: the tolerances of the mixed-form tests)."""
import numpy as np
import pytest

from paper_2409_09620_gb300 import workloads as W
from tests.helpers import rel_err

# mixed form after a few steps against the FP64 oracle: cell averages (FP64
# arithmetic on FP32 flux sums) and all modes, relative to the largest oracle
# magnitude per quantity
MIXED_AVG_TOL, MIXED_MODE_TOL = 1e-5, 1e-3


def check_against_oracle(O, wl, u0, u_gpu, t_gpu, steps, precision, t_end=1e30):
    """The solve's state after `steps` steps (or at t_end) against the oracle
    advanced from the same initial state."""
    om = O.OracleMesh.from_mesh(wl.mesh)
    uo, to, cnt, rc = om.advance(O.config_for(wl), u0, 0.0, t_end, max_steps=steps)
    assert rc == 0 and cnt[3] == steps
    if precision == 0:
        assert abs(t_gpu - to) <= 1e-12 * to, (t_gpu, to)
        err = rel_err(u_gpu, uo)
        assert err < 1e-9, err
    else:
        assert abs(t_gpu - to) <= 1e-5 * to, (t_gpu, to)
        ea, em = rel_err(u_gpu[:, :1], uo[:, :1]), rel_err(u_gpu, uo)
        assert ea < MIXED_AVG_TOL and em < MIXED_MODE_TOL, (ea, em)
    return uo

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    from paper_2409_09620_gb300 import native
    native.lib()
    return native


def _workloads():
    return [W.vortex_workload(n=16, k=1), W.sedov_workload(n=14, k=2), W.riemann4_workload(n=11, k=1),
            W.dmr_workload(nx=24, ny=8, k=2), W.riemann4_workload(n=23, k=2, seed=9)]


def _setup(N, wls, precision, O=None):
    """Meshes, configurations and initial states (the oracle's projection and
    limiter pass when O is given, else the library's projection)."""
    meshes = [N.Mesh.from_mesh(w.mesh) for w in wls]
    cfgs = [N.config_for(w, precision=precision) for w in wls]
    if O is None:
        us = [N.initial_state(m, w) for m, w in zip(meshes, wls)]
    else:
        us = [O.project_workload(O.OracleMesh.from_mesh(w.mesh), w) for w in wls]
    return meshes, cfgs, us


@pytest.mark.parametrize("form", [3, 1, 0])
@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_solo(oracle_mod, N, precision, form):
    wls = _workloads()
    meshes, cfgs, us = _setup(N, wls, precision, oracle_mod)
    batch = N.Batch(meshes, cfgs, us)
    assert batch.shape()["launches_per_stage"] == 3
    batch.set_shape(512, 64, form)
    sh = batch.shape()
    assert sh["launches_per_stage"] == form and sh["cells_per_block"] == 512 and 1 <= sh["blocks_per_sm"] < 64
    st = batch.advance(None, max_steps=7)
    assert all(s["steps"] == 7 for s in st)
    for i in range(len(wls)):
        solo = N.Solver(meshes[i], cfgs[i], us[i])
        solo.advance(1e30, max_steps=7)
        a, ta = batch.solver(i).get_state()
        b, tb = solo.get_state()
        assert ta == tb
        assert np.array_equal(a, b), i
        check_against_oracle(oracle_mod, wls[i], us[i], a, ta, 7, precision)


def test_batch_end_times_and_shapes(oracle_mod, N):
    wls = _workloads()
    meshes, cfgs, us = _setup(N, wls, 0, oracle_mod)
    batch = N.Batch(meshes, cfgs, us)
    # end times a few steps in, different per solve
    t_end = np.array([0.002, 0.0005, 0.003, 0.0002, 0.001])
    batch.set_shape(256, 1)
    st = batch.advance(t_end, max_steps=2)
    batch.set_shape(128, 2, 1)       # change the launch form part-way, twice
    st2 = batch.advance(t_end, max_steps=2)
    batch.set_shape(128, 2, 0)
    st3 = batch.advance(t_end)
    st = [dict(a, steps=a["steps"] + b["steps"] + c["steps"]) for a, b, c in zip(st, st2, st3)]
    for i in range(len(wls)):
        solo = N.Solver(meshes[i], cfgs[i], us[i])
        sst, _ = solo.advance(t_end[i])
        a, ta = batch.solver(i).get_state()
        b, tb = solo.get_state()
        assert ta == t_end[i] and tb == t_end[i]
        assert st[i]["steps"] == sst["steps"]
        assert np.array_equal(a, b), i
        check_against_oracle(oracle_mod, wls[i], us[i], a, ta, sst["steps"], 0, t_end=t_end[i])


def test_batch_autotune_restores_state(N):
    wls = _workloads()
    meshes, cfgs, us = _setup(N, wls, 0)
    batch = N.Batch(meshes, cfgs, us)
    batch.advance(None, max_steps=2)
    before = [batch.solver(i).get_state() for i in range(len(wls))]
    best = batch.autotune(steps=2)
    shape = batch.shape()
    assert best["cells_per_block"] == shape["cells_per_block"] and best["ms_per_step"] > 0
    assert best["launches_per_stage"] == shape["launches_per_stage"] in (0, 1, 3)
    after = [batch.solver(i).get_state() for i in range(len(wls))]
    for (a, ta), (b, tb) in zip(before, after):
        assert ta == tb and np.array_equal(a, b)
    st = batch.advance(None, max_steps=3)
    assert all(s["steps"] == 3 for s in st)
    for i in range(len(wls)):
        solo = N.Solver(meshes[i], cfgs[i], us[i])
        solo.advance(1e30, max_steps=5)
        assert np.array_equal(batch.solver(i).get_state()[0], solo.get_state()[0])


def test_batch_rejects_mixed_precisions(N):
    wls = _workloads()[:2]
    meshes, cfgs, us = _setup(N, wls, 0)
    cfgs[1] = N.config_for(wls[1], precision=1)
    with pytest.raises(N.DGError) as e:
        N.Batch(meshes, cfgs, us)
    assert e.value.code == N.DG_EINVAL


def test_batch_rejects_bad_shapes(N):
    wls = _workloads()[:2]
    meshes, cfgs, us = _setup(N, wls, 0)
    batch = N.Batch(meshes, cfgs, us)
    for bad in ((100, 1, 3), (256, 0, 3), (256, 1, 2)):
        with pytest.raises(N.DGError) as e:
            batch.set_shape(*bad)
        assert e.value.code == N.DG_EINVAL
    st = batch.advance(None, max_steps=2)
    assert all(s["steps"] == 2 for s in st)


def test_barrier_wait_runs_out_and_the_batch_recovers(oracle_mod, N):
    """The cooperative form's grid barrier is the library's one device-side
    wait.  With phantom arrivals added (a fault injected from the host), no
    grid can complete it: every block's wait runs out after its short limit,
    the launch ends early, and dg_batch_advance returns DG_ETIMEOUT within
    seconds.  The host clears the barrier and the finalisation tickets; after
    the states are restored, the next steps are bitwise those of the solves
    run alone and match the oracle."""
    import time
    wls = _workloads()[:3]
    meshes, cfgs, us = _setup(N, wls, 0, oracle_mod)
    batch = N.Batch(meshes, cfgs, us)
    if batch.shape()["launches_per_stage"] != 3:
        pytest.skip("unexpected default form")
    try:
        batch.set_shape(256, 1, 1)
    except N.DGError:
        pytest.skip("no cooperative launch on this device")
    saved = [batch.solver(i).get_state() for i in range(len(wls))]
    batch.set_barrier(timeout_ns=20_000_000, extra_arrivals=1)
    t0 = time.perf_counter()
    with pytest.raises(N.DGError) as e:
        batch.advance(None, max_steps=1)
    assert e.value.code == N.DG_ETIMEOUT
    assert time.perf_counter() - t0 < 10.0
    batch.set_barrier(timeout_ns=2_000_000_000, extra_arrivals=0)
    for i, (u, t) in enumerate(saved):
        batch.solver(i).set_state(u, t)
    st = batch.advance(None, max_steps=3)
    assert all(s["steps"] == 3 for s in st)
    for i in range(len(wls)):
        solo = N.Solver(meshes[i], cfgs[i], us[i])
        solo.set_state(*solo.get_state())       # the same restore path as the batch's solves
        solo.advance(1e30, max_steps=3)
        a, ta = batch.solver(i).get_state()
        b, tb = solo.get_state()
        assert ta == tb and np.array_equal(a, b), i
        check_against_oracle(oracle_mod, wls[i], us[i], a, ta, 3, 0)
