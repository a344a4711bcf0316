"""Domain decomposition of the BP RI-OEDG step across ranks, checked on CPU
with gloo ranks against the unpartitioned oracle.

The method shards by cells: a rank owns a set of cells and keeps a halo of
the edge neighbours of its cells.  One SSP-RK3 step (Sec. 4.5) then needs, per
stage,
  * the viscosity coefficient alpha (eq. 1250) and, once per step, the BP time
    step: a max over ranks;
  * a halo exchange of the stage input before the DG operator L (the edge
    fluxes read the neighbour's trace);
  * the OE statistics (domain means and sup deviations, Sec. 2.3 / 3): the
    means sum every cell average, the deviations are a max over ranks;
  * a halo exchange of the pre-OE state before the OE step (the jumps read
    the neighbour's derivatives);
  * nothing for the limiter (Sec. 4.4 reads the cell alone).

Here each rank is a gloo process that runs the oracle's per-cell phases on
its own cells only, with every coefficient outside its cells and halo set to
NaN, so a read past the halo shows up in the result.  The halo exchange is
point to point (isend / irecv of the boundary cells to the ranks whose halo
holds them); alpha and the deviations are all-reduced with MAX (exact in any
order).  The domain means must round as in the unpartitioned sum, which adds
the cell averages in cell order, so the ranks exchange the cell averages
themselves (an all-reduce SUM in which each average meets only zeros, which
is exact) and every rank sums them in cell order.  The mesh (geometry only)
is replicated.

The partitioned run must equal the oracle's own step bit for bit: state, time
and counters, on periodic, wall, inflow, moving-shock and transmissive
boundaries, P1 and P2, with 3 ranks, one of which may own nothing.  Leaving
out the halo exchange before OE must break that equality.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

# SSP-RK3 (Sec. 4.5): u_h = a u^n + b (v + dt L(v)); stage times t + c dt
RK_A = (0.0, 0.75, 1.0 / 3.0)
RK_B = (1.0, 0.25, 2.0 / 3.0)
C_IN = (0.0, 1.0, 0.5)
C_OUT = (1.0, 0.5, 1.0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _workload(name, k):
    from paper_2409_09620_gb300 import workloads as W
    if name == "vortex":
        return W.vortex_workload(n=8, k=k, radius=0.2)
    if name == "dmr":
        return W.dmr_workload(nx=8, ny=4, k=k)
    if name == "riemann":
        return W.riemann4_workload(n=8, k=k)
    if name == "sedov":
        return W.sedov_workload(n=8, k=k)
    raise KeyError(name)


def partition(wl, nranks, empty_rank=None):
    """Cells split into strips of equal count by centroid x (stable order);
    ``empty_rank`` owns nothing."""
    cx = wl.mesh.xy[wl.mesh.tri].mean(axis=1)[:, 0]
    order = np.argsort(cx, kind="stable")
    active = [r for r in range(nranks) if r != empty_rank]
    parts = np.array_split(order, len(active))
    owned = [np.zeros(0, np.int64) for _ in range(nranks)]
    for r, p in zip(active, parts):
        owned[r] = np.sort(p).astype(np.int64)
    return owned


def halo_plan(nbr, owned):
    """halo[r]: cells outside r that share an edge with a cell of r;
    send[r][q]: r's cells in q's halo; recv[r][q]: q's cells in r's halo."""
    nranks = len(owned)
    owner = np.full(nbr.shape[0], -1, np.int64)
    for r, cells in enumerate(owned):
        owner[cells] = r
    assert (owner >= 0).all()
    halo = []
    for r, cells in enumerate(owned):
        nb = nbr[cells].ravel()
        nb = nb[nb >= 0]
        halo.append(np.unique(nb[owner[nb] != r]).astype(np.int64))
    recv = [{q: halo[r][owner[halo[r]] == q] for q in range(nranks) if q != r} for r in range(nranks)]
    send = [{q: recv[q][r] for q in range(nranks) if q != r} for r in range(nranks)]
    return halo, send, recv


class Comm:
    """The exchanges of one partitioned step, over torch.distributed."""

    def __init__(self, rank, nranks, send, recv):
        import torch.distributed as dist
        self.dist, self.rank, self.n = dist, rank, nranks
        self.send, self.recv = send[rank], recv[rank]
        self.halo_messages = 0

    def allmax(self, x):
        t = torch.tensor(np.atleast_1d(np.asarray(x, np.float64)).copy())
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return t.numpy()

    def allsum_int(self, x):
        t = torch.tensor(np.asarray(x, np.int64).copy())
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return t.numpy()

    def gather_averages(self, u, owned):
        """Every cell's average (mode 0) onto every rank: each rank contributes
        its own cells and zeros elsewhere, so each sum is exact."""
        part = np.zeros((4, u.shape[2]))
        part[:, owned] = u[:, 0, owned]
        t = torch.tensor(part)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        out = u.copy()
        out[:, 0, :] = t.numpy()
        return out

    def exchange(self, u):
        """Halo exchange of the full coefficients: point to point."""
        reqs, bufs = [], {}
        for q, cells in self.recv.items():
            if cells.size:
                bufs[q] = torch.empty((u.shape[0], u.shape[1], cells.size), dtype=torch.float64)
                reqs.append(self.dist.irecv(bufs[q], src=q))
        for q, cells in self.send.items():
            if cells.size:
                reqs.append(self.dist.isend(torch.tensor(np.ascontiguousarray(u[:, :, cells])), dst=q))
                self.halo_messages += 1
        for r in reqs:
            r.wait()
        out = u.copy()
        for q, b in bufs.items():
            out[:, :, self.recv[q]] = b.numpy()
        return out


def _own_only(full, owned):
    out = np.full_like(full, np.nan)
    out[:, :, owned] = full[:, :, owned]
    return out


def partitioned_step(om, cf, u, t, t_end, owned, comm, skip_oe_halo=False):
    """One SSP-RK3 step of the BP OEDG scheme (Sec. 4.5) on a rank's cells,
    in the order of the oracle's own step; returns (u, t, counters)."""
    k = cf.k
    min_ca = om.min_cfl_area(k, cf.decomp)
    un = u
    v = u
    alpha1 = float(comm.allmax(om.alpha(cf, un, t, cells=owned))[0])
    dt = cf.cfl * min_ca / alpha1
    clamped = t + dt >= t_end
    if clamped:
        dt = t_end - t
    lim = np.zeros(2, np.int64)
    breaches = 0
    for s in range(3):
        ts = t + C_IN[s] * dt
        alpha = alpha1 if s == 0 else float(comm.allmax(om.alpha(cf, v, ts, cells=owned))[0])
        if alpha * dt > min_ca * (1.0 + 1e-12):
            breaches += 1
        v = comm.exchange(v)                                       # halo 1: stage input
        uh = _own_only(om.rk_stage(cf, un, v, RK_A[s], RK_B[s], dt, alpha, ts, cells=owned), owned)
        if cf.oe:
            uh = comm.gather_averages(uh, owned)
            st = om.stats(cf, uh, cells=owned)
            st[[4, 5, 6, 8, 9]] = comm.allmax(st[[4, 5, 6, 8, 9]])
            if not skip_oe_halo:
                uh = comm.exchange(uh)                             # halo 2: pre-OE state
            tmp = _own_only(om.oe(cf, uh, dt, st, t + C_OUT[s] * dt, cells=owned), owned)
        else:
            tmp = uh
        if cf.bp:
            out, cnt = om.limit(cf, tmp, cells=owned)
            v = _own_only(out, owned)
            lim += cnt
        else:
            v = tmp
    lim = comm.allsum_int(lim)
    cnt = np.array([lim[0], lim[1], breaches, 1], np.int64)
    return v, (t_end if clamped else t + dt), cnt


CASES = [("vortex", 1, None), ("vortex", 2, None), ("dmr", 2, None), ("dmr", 1, 1),
         ("riemann", 1, None), ("sedov", 2, 2)]
STEPS = 3


def _worker(rank, nranks, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(nranks), "MASTER_ADDR": "127.0.0.1",
                       "MASTER_PORT": str(port), "OMP_NUM_THREADS": "2"})
    import torch.distributed as dist
    from oracle import oracle as O
    dist.init_process_group("gloo", rank=rank, world_size=nranks)
    try:
        results = []
        for name, k, empty in CASES:
            for skip in (False, True) if (name, k) == ("vortex", 2) else (False,):
                wl = _workload(name, k)
                om = O.OracleMesh.from_mesh(wl.mesh)
                cf = O.config_for(wl)
                u0 = O.project_workload(om, wl)
                owned = partition(wl, nranks, empty)
                halo, send, recv = halo_plan(om.neighbors()[0], owned)
                comm = Comm(rank, nranks, send, recv)
                keep = np.concatenate([owned[rank], halo[rank]])
                u = np.full_like(u0, np.nan)
                u[:, :, keep] = u0[:, :, keep]
                t, cnt = 0.0, np.zeros(4, np.int64)
                for _ in range(STEPS):
                    u, t, c = partitioned_step(om, cf, u, t, wl.t_end, owned[rank], comm, skip_oe_halo=skip)
                    cnt += c
                ref, tr, cr, rc = om.advance(cf, u0, 0.0, wl.t_end, max_steps=STEPS)
                mine = owned[rank]
                results.append(dict(case=(name, k, empty, skip), rc=rc,
                                    equal=bool(np.array_equal(u[:, :, mine], ref[:, :, mine])),
                                    t=(t, tr), cnt=(cnt.tolist(), cr.tolist()), n=int(mine.size),
                                    halo=int(halo[rank].size), msgs=comm.halo_messages))
        q.put((rank, results))
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def runs(oracle_mod):
    nranks, port = 3, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, nranks, port, q)) for r in range(nranks)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=600) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return out


@pytest.mark.parametrize("case", [c for c in CASES])
def test_partitioned_step_is_bitwise_the_oracle(runs, case):
    name, k, empty = case
    total = 0
    for rank, results in runs.items():
        r = next(x for x in results if x["case"] == (name, k, empty, False))
        assert r["rc"] == 0
        assert r["equal"], (rank, r)
        assert r["t"][0] == r["t"][1]
        assert r["cnt"][0] == r["cnt"][1], (rank, r["cnt"])
        total += r["n"]
        if rank == empty:
            assert r["n"] == 0 and r["halo"] == 0 and r["msgs"] == 0
        else:
            assert r["halo"] > 0 and r["msgs"] > 0
    assert total == _workload(name, k).mesh.tri.shape[0]


def test_missing_oe_halo_exchange_is_caught(runs):
    """Without the exchange before OE the jumps at the partition boundary read
    NaN (or stale) neighbours: the result differs from the oracle."""
    eq = [next(x for x in res if x["case"] == ("vortex", 2, None, True))["equal"] for res in runs.values()]
    assert not all(eq)


def test_halo_is_the_edge_neighbour_layer(oracle_mod):
    """Unit check of the plan: every halo cell shares an edge with an owned
    cell, is owned elsewhere, and is sent by its owner to exactly this rank."""
    wl = _workload("vortex", 1)
    om = oracle_mod.OracleMesh.from_mesh(wl.mesh)
    nbr = om.neighbors()[0]
    owned = partition(wl, 3)
    halo, send, recv = halo_plan(nbr, owned)
    for r in range(3):
        own = set(owned[r].tolist())
        assert not own & set(halo[r].tolist())
        for h in halo[r]:
            assert any(nbr[h, i] in own for i in range(3))
        got = np.sort(np.concatenate([recv[r][q] for q in recv[r]]))
        assert np.array_equal(got, halo[r])
        for q in send[r]:
            assert np.array_equal(send[r][q], recv[q][r])
