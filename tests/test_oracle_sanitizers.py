"""The CPU oracle under AddressSanitizer, UndefinedBehaviorSanitizer and
LeakSanitizer.  The oracle's C sources and a small driver
(``tests/oracle_sanitize_driver.c``) are built with the sanitizers and with
OpenMP off.  The driver calls every entry point: the mesh builder with good and
rejected meshes, the decomposition of every cell, the stage operators on all
cells and on a subset, and a few steps of the scheme, for Euler and the scalar
laws.  The test passes when the build runs clean (any finding aborts it) and
its steps equal, bit for bit, those of the regular oracle library.  The two
builds share the sources and use no FP contraction, so their results agree
bit for bit."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2409_09620_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
ORACLE = os.path.join(os.path.dirname(HERE), "oracle")
SAN = "-fsanitize=address,undefined"


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    d = tmp_path_factory.mktemp("san")
    exe = str(d / "driver")
    cmd = ["gcc", "-O1", "-g", "-std=c11", SAN, "-fno-sanitize-recover=all", "-fno-omit-frame-pointer",
           "-ffp-contract=off", "-Wall", "-Wno-unknown-pragmas", "-Wno-unused-function", "-I", ORACLE,
           os.path.join(HERE, "oracle_sanitize_driver.c"), os.path.join(ORACLE, "oracle.c"),
           os.path.join(ORACLE, "scalar.c"), "-lm", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and ("asan" in r.stderr or "ubsan" in r.stderr):
        pytest.skip("the sanitizer runtimes are not installed")
    assert r.returncode == 0, r.stderr
    return exe, d


def _run(driver, name, header, mesh, cfg_bytes, u0, t_end):
    exe, d = driver
    fin, fout = str(d / f"{name}.in"), str(d / f"{name}.out")
    with open(fin, "wb") as f:
        f.write(np.asarray(header, np.int64).tobytes())
        f.write(np.ascontiguousarray(mesh.xy, np.float64).tobytes())
        f.write(np.ascontiguousarray(mesh.tri, np.int32).tobytes())
        f.write(np.ascontiguousarray(mesh.canon, np.int32).tobytes())
        f.write(np.ascontiguousarray(mesh.bc, np.int8).tobytes())
        f.write(cfg_bytes)
        f.write(np.ascontiguousarray(u0, np.float64).tobytes())
        f.write(np.float64(t_end).tobytes())
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0:exitcode=23",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    r = subprocess.run([exe, fin, fout], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr[-4000:]
    assert "runtime error" not in r.stderr and "Sanitizer" not in r.stderr, r.stderr[-4000:]
    raw = open(fout, "rb").read()
    n = np.asarray(u0).size
    u = np.frombuffer(raw[: 8 * n], np.float64).reshape(np.asarray(u0).shape)
    t = float(np.frombuffer(raw[8 * n: 8 * n + 8], np.float64)[0])
    cnt = np.frombuffer(raw[8 * n + 8:], np.int64)
    return u, t, cnt


EULER = {
    "vortex_p1": lambda: W.vortex_workload(n=6, k=1, radius=0.2),
    "vortex_p2": lambda: W.vortex_workload(n=6, k=2, radius=0.2),
    "dmr_p2": lambda: W.dmr_workload(nx=6, ny=3, k=2),
    "riemann_p1": lambda: W.riemann4_workload(n=6, k=1),
    "sedov_p2": lambda: W.sedov_workload(n=6, k=2),
}


@pytest.mark.parametrize("variant", ["rioe", "cw_zxs"])
@pytest.mark.parametrize("name", sorted(EULER))
def test_oracle_euler_clean_under_sanitizers(oracle_mod, driver, name, variant):
    O = oracle_mod
    wl = EULER[name]()
    om = O.OracleMesh.from_mesh(wl.mesh)
    u0 = O.project_workload(om, wl)
    cf = O.config_for(wl) if variant == "rioe" else O.config_for(wl, oe=2, decomp=1)
    steps = 3
    u, t, cnt = _run(driver, f"{name}_{variant}", [0, wl.mesh.xy.shape[0], om.nt, wl.k, steps], wl.mesh,
                     bytes(cf), u0, wl.t_end)
    ref, tr, cr, rc = om.advance(cf, u0, 0.0, wl.t_end, max_steps=steps)
    assert rc == 0
    assert np.array_equal(u, ref) and t == tr
    assert cnt.tolist() == cr.tolist()


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("kind", ["linear", "burgers_rm2"])
def test_oracle_scalar_clean_under_sanitizers(oracle_mod, driver, kind, k):
    O = oracle_mod
    wl = W.scalar_linear_workload(level=1, k=k) if kind == "linear" else W.burgers_riemann2_workload(n=6, k=k)
    om = O.OracleMesh.from_mesh(wl.mesh)
    u0 = om.sc_project(k, wl.u0)
    bc = tuple(getattr(wl, "bc_state", (0.0, 0.0, 0.0, 0.0)))
    cf = O.make_sc_config(k, flux=wl.flux, bc_state=bc)
    steps = 3
    u, t, cnt = _run(driver, f"sc_{kind}_{k}", [1, wl.mesh.xy.shape[0], om.nt, k, steps], wl.mesh,
                     bytes(cf), u0, wl.t_end)
    ref, tr = u0.copy(), 0.0
    for _ in range(steps):
        ref, tr, _, rc = om.sc_step(cf, ref, tr, wl.t_end)
        assert rc == 0
    assert np.array_equal(u, ref) and t == tr
    assert cnt[0] == steps
