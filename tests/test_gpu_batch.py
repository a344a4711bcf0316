"""GPU tests of batches: independent ragged meshes (P1 and P2 mixed) advanced
together, by one launch per phase or by one persistent cooperative launch per
RK stage.  Each solve of a batch must be bitwise identical to the same solve
advanced alone, for either launch form and any launch shape, with per-solve
end times, in FP64 and in the mixed form."""
import numpy as np
import pytest

from paper_2409_09620_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    from paper_2409_09620_gb300 import native
    native.lib()
    return native


def _workloads():
    return [W.vortex_workload(n=16, k=1), W.sedov_workload(n=14, k=2), W.riemann4_workload(n=11, k=1),
            W.dmr_workload(nx=24, ny=8, k=2), W.riemann4_workload(n=23, k=2, seed=9)]


def _setup(N, wls, precision):
    meshes = [N.Mesh.from_mesh(w.mesh) for w in wls]
    cfgs = [N.config_for(w, precision=precision) for w in wls]
    us = [N.initial_state(m, w) for m, w in zip(meshes, wls)]
    return meshes, cfgs, us


@pytest.mark.parametrize("form", [3, 1])
@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_solo(N, precision, form):
    wls = _workloads()
    meshes, cfgs, us = _setup(N, wls, precision)
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


def test_batch_end_times_and_shapes(N):
    wls = _workloads()
    meshes, cfgs, us = _setup(N, wls, 0)
    batch = N.Batch(meshes, cfgs, us)
    # end times a few steps in, different per solve
    t_end = np.array([0.002, 0.0005, 0.003, 0.0002, 0.001])
    batch.set_shape(256, 1)
    st = batch.advance(t_end, max_steps=2)
    batch.set_shape(128, 2, 1)       # change the launch form part-way
    st2 = batch.advance(t_end)
    st = [dict(a, steps=a["steps"] + b["steps"]) for a, b in zip(st, st2)]
    for i in range(len(wls)):
        solo = N.Solver(meshes[i], cfgs[i], us[i])
        sst, _ = solo.advance(t_end[i])
        a, ta = batch.solver(i).get_state()
        b, tb = solo.get_state()
        assert ta == t_end[i] and tb == t_end[i]
        assert st[i]["steps"] == sst["steps"]
        assert np.array_equal(a, b), i


def test_batch_autotune_restores_state(N):
    wls = _workloads()
    meshes, cfgs, us = _setup(N, wls, 0)
    batch = N.Batch(meshes, cfgs, us)
    batch.advance(None, max_steps=2)
    before = [batch.solver(i).get_state() for i in range(len(wls))]
    best = batch.autotune(steps=2)
    shape = batch.shape()
    assert best["cells_per_block"] == shape["cells_per_block"] and best["ms_per_step"] > 0
    assert best["launches_per_stage"] == shape["launches_per_stage"] in (1, 3)
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
