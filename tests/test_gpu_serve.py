"""GPU tests of the continuous-batching server: results are the same alone and
in a mix of concurrently running requests, and match the CPU oracle run to
the same end time; admission respects the HBM budget, and a request larger
than the budget fails cleanly."""
import numpy as np
import pytest

from paper_2409_09620_gb300 import workloads as W
from tests.test_gpu_batch import check_against_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    from paper_2409_09620_gb300 import native
    native.lib()
    return native


def _request(N, wl, precision=0, O=None):
    """(workload, configuration, initial state): the oracle's projection and
    limiter pass when O is given, else the library's projection."""
    if O is not None:
        u = O.project_workload(O.OracleMesh.from_mesh(wl.mesh), wl)
    else:
        u = N.initial_state(N.Mesh.from_mesh(wl.mesh), wl)
    return wl, N.config_for(wl, precision=precision), u


def _drain(srv, max_ticks=100000):
    for _ in range(max_ticks):
        r, q = srv.tick()
        if r == 0 and q == 0:
            return
    raise AssertionError("server did not drain")


@pytest.mark.parametrize("precision", [0, 1])
def test_same_alone_and_in_the_mix(oracle_mod, N, precision):
    target = _request(N, W.riemann4_workload(n=17, k=2, seed=21), precision, oracle_mod)
    others = [_request(N, w, precision) for w in
              (W.vortex_workload(n=20, k=1), W.sedov_workload(n=16, k=2), W.riemann4_workload(n=9, k=1, seed=5),
               W.dmr_workload(nx=30, ny=10, k=2))]
    t_end = 0.004
    # alone
    srv = N.Server(precision, budget_bytes=1 << 30, steps_per_tick=3)
    rid = srv.submit(target[0].mesh, target[1], target[2], t_end)
    _drain(srv)
    assert srv.info(rid)["state"] == N.REQ_DONE
    alone = srv.result(rid)
    steps_alone = srv.info(rid)["steps"]
    # in the mix: other requests first, the target arrives while they run
    srv = N.Server(precision, budget_bytes=1 << 30, steps_per_tick=3)
    ids = [srv.submit(w.mesh, c, u, 0.002 + 0.001 * i) for i, (w, c, u) in enumerate(others[:2])]
    srv.tick()
    srv.tick()
    rid = srv.submit(target[0].mesh, target[1], target[2], t_end)
    ids += [srv.submit(w.mesh, c, u, 0.003) for (w, c, u) in others[2:]]
    running_max = 0
    for _ in range(100000):
        r, q = srv.tick()
        running_max = max(running_max, r)
        if r == 0 and q == 0:
            break
    assert running_max >= 3              # the target shared launches with other solves
    info = srv.info(rid)
    assert info["state"] == N.REQ_DONE and info["t"] == t_end and info["steps"] == steps_alone
    assert np.array_equal(srv.result(rid), alone)
    for i in ids:
        assert srv.info(i)["state"] == N.REQ_DONE
    # the oracle run to the same end time from the same state
    check_against_oracle(oracle_mod, target[0], target[2], alone, t_end, steps_alone, precision, t_end=t_end)
    # and the same as the solver used on its own
    solo = N.Solver(N.Mesh.from_mesh(target[0].mesh), target[1], target[2])
    solo.advance(t_end)
    assert np.array_equal(solo.get_state()[0], alone)


def test_budget_admission(N):
    reqs = [_request(N, W.riemann4_workload(n=14, k=1 + (i % 2), seed=30 + i)) for i in range(6)]
    # budget for about two solves at a time
    probe = N.Server(0, budget_bytes=1 << 30, steps_per_tick=2)
    pid = probe.submit(reqs[1][0].mesh, reqs[1][1], reqs[1][2], 0.001)
    per_solve = probe.info(pid)["device_bytes"]
    probe.close()
    srv = N.Server(0, budget_bytes=int(2.5 * per_solve), steps_per_tick=2)
    ids = [srv.submit(w.mesh, c, u, 0.002) for (w, c, u) in reqs]
    saw_queue = False
    for _ in range(100000):
        r, q = srv.tick()
        st = srv.stats()
        assert st["bytes_in_use"] <= int(2.5 * per_solve)
        saw_queue |= (r > 0 and q > 0)
        if r == 0 and q == 0:
            break
    assert saw_queue
    for i in ids:
        inf = srv.info(i)
        assert inf["state"] == N.REQ_DONE and inf["t"] == 0.002 and inf["done_s"] >= inf["start_s"] >= inf["submit_s"]
    assert srv.stats()["cell_stages_done"] > 0


def test_oversized_request_fails(N):
    w, c, u = _request(N, W.riemann4_workload(n=10, k=2))
    srv = N.Server(0, budget_bytes=1000, steps_per_tick=1)
    rid = srv.submit(w.mesh, c, u, 0.01)
    srv.tick()
    inf = srv.info(rid)
    assert inf["state"] == N.REQ_FAILED and inf["error"] == N.DG_ENOMEM
