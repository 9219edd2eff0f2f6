"""Host-side schedules of the symbolic analysis, checked without a GPU: a small
C++ driver (tests/plan_check.cpp) is compiled against csrc/plan.cpp and run on
generated networks."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import gridgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2203_11875_gb300", "csrc")


def _write(net, path):
    with open(path, "wb") as f:
        np.array([net.nb, net.nl, net.ng, net.slack], np.int32).tofile(f)
        for a in (net.Pd, net.Qd, net.Vmin, net.Vmax):
            np.asarray(a, np.float64).tofile(f)
        np.asarray(net.lf, np.int32).tofile(f)
        np.asarray(net.lt, np.int32).tofile(f)
        for a in (net.r, net.x, net.b, net.rate):
            np.asarray(a, np.float64).tofile(f)
        np.asarray(net.gbus, np.int32).tofile(f)
        for a in (net.Pmin, net.Pmax, net.Qmin, net.Qmax, net.c2, net.c1):
            np.asarray(a, np.float64).tofile(f)


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    out = tmp_path_factory.mktemp("plan") / "plan_check"
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, "-o", str(out),
                    os.path.join(ROOT, "tests", "plan_check.cpp"), os.path.join(CSRC, "plan.cpp")],
                   check=True, capture_output=True)
    return out


@pytest.mark.parametrize("name", ["tiny3", "ring30", "grid2000"])
def test_cluster_solve_schedules(checker, tmp_path, name):
    path = tmp_path / f"{name}.bin"
    _write(gridgen.WORKLOADS[name](), str(path))
    res = subprocess.run([str(checker), str(path)], capture_output=True, text=True, timeout=120)
    assert res.returncode == 0 and res.stdout.strip() == "ok", res.stdout + res.stderr


@pytest.fixture(scope="module")
def fs_checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    out = tmp_path_factory.mktemp("fsplan") / "fsplan_check"
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, "-o", str(out),
                    os.path.join(ROOT, "tests", "fsplan_check.cpp"), os.path.join(CSRC, "plan.cpp"),
                    os.path.join(CSRC, "fsplan.cpp")], check=True, capture_output=True)
    return out


@pytest.mark.parametrize("name", ["tiny3", "ring30", "grid2000"])
def test_fullspace_block_plan(fs_checker, tmp_path, name):
    """The block LDL^T plan of the hybrid full-space system: a permutation of
    the unknowns, a symmetric fill-closed block pattern in level order, and
    assembly slots with one source each (tests/fsplan_check.cpp)."""
    net = gridgen.WORKLOADS[name]()
    path = tmp_path / f"{name}.bin"
    _write(net, str(path))
    res = subprocess.run([str(fs_checker), str(path)], capture_output=True, text=True, timeout=120)
    out = res.stdout.split()
    assert res.returncode == 0 and out and out[0] == "ok", res.stdout + res.stderr
    n, nblk, bmax = int(out[1]), int(out[2]), int(out[3])
    from oracle import model
    lay = model.Layout(net)
    assert n == lay.nw + lay.nx + lay.m
    # one block per bus and one per flow-limit row; at most 5 unknowns per bus
    assert nblk == net.nb + 2 * len(lay.lim)
    assert 1 <= bmax <= 5


@pytest.fixture(scope="module")
def reach_checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    out = tmp_path_factory.mktemp("reach") / "reach_check"
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", CSRC, "-o", str(out),
                    os.path.join(ROOT, "tests", "reach_check.cpp"), os.path.join(CSRC, "plan.cpp")],
                   check=True, capture_output=True)
    return out


@pytest.mark.parametrize("name,make", [("ring30", gridgen.ring30),
                                       ("b1500", lambda: gridgen.lattice(1500, 7002, name="b1500")),
                                       ("grid2000", gridgen.grid2000)])
def test_forward_sweep_reach_lists(reach_checker, tmp_path, name, make):
    """The reach lists the forward sweep L Y = P G_u passes rows by: a numeric
    forward solve with random values on both patterns is nonzero only on
    listed rows, every listed row is nonzero or shares a supernode with one,
    and the lists hold only part of the rows (tests/reach_check.cpp)."""
    net = make()
    path = tmp_path / f"{name}.bin"
    _write(net, str(path))
    res = subprocess.run([str(reach_checker), str(path)], capture_output=True, text=True, timeout=300)
    out = res.stdout.split()
    assert res.returncode == 0 and out and out[0] == "ok", res.stdout + res.stderr
    from oracle import model
    nblk, listed, allr, frac = int(out[1]), int(out[2]), int(out[3]), float(out[4])
    assert nblk == model.Layout(net).nu // 32
    if nblk:
        assert 0 < listed < allr and 0 < frac < 0.9
