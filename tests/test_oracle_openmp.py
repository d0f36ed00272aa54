"""The oracle built with OpenMP (the second CPU figure of the bench) computes bitwise what the serial
build computes: its parallel loops each write only their own cell, and every sum stays serial."""
import os
import subprocess
import sys

import numpy as np

import oracle as O
from paper_2209_14889_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import oracle as O
from paper_2209_14889_gb300 import workloads as W
assert O._OPENMP
out = {}
for name, w in [("periodic", W.cfg1()), ("box", W.make(48, 40, rings=[W.ring(20, 4.0, (20.3, 19.6), pull_force=0.0,
                trap=dict(k=0.05, dx=4.0, dy=1.0, t_eq=30, pull=40, width=30))], seed=5, walls_x=1, walls_y=1)),
                ("substeps", W.make(40, 32, rings=[], seed=6, Dp=0.3, diffusion_substeps=2))]:
    s = O.Sim.from_workload(w)
    s.step(30, every=10)
    for k, v in s.fields().items():
        out[name + "_" + k] = v
    out[name + "_X"] = s.X
    out[name + "_series"] = np.array(s.series)
np.savez(sys.argv[2], **out)
"""


def _serial():
    out = {}
    for name, w in [("periodic", W.cfg1()), ("box", W.make(48, 40, rings=[W.ring(20, 4.0, (20.3, 19.6), pull_force=0.0,
                    trap=dict(k=0.05, dx=4.0, dy=1.0, t_eq=30, pull=40, width=30))], seed=5, walls_x=1, walls_y=1)),
                    ("substeps", W.make(40, 32, rings=[], seed=6, Dp=0.3, diffusion_substeps=2))]:
        s = O.Sim.from_workload(w)
        s.step(30, every=10)
        for k, v in s.fields().items():
            out[name + "_" + k] = v
        out[name + "_X"] = s.X
        out[name + "_series"] = np.array(s.series)
    return out


def test_openmp_build_is_bitwise_the_serial_oracle(tmp_path):
    assert not O._OPENMP
    path = str(tmp_path / "omp.npz")
    env = dict(os.environ, VLB_ORACLE_OPENMP="1", OMP_NUM_THREADS="4")
    subprocess.check_call([sys.executable, "-c", _CHILD, ROOT, path], env=env, cwd=ROOT)
    got = np.load(path)
    ref = _serial()
    assert set(got.files) == set(ref)
    for k, v in ref.items():
        assert np.array_equal(got[k], v), k


_CHILD3D = r"""
import sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import oracle.o3d as O3
from paper_2209_14889_gb300 import workloads as W
assert O3._OPENMP
s = O3.Sim3.from_workload(W.make3d(10, 8, 6, seed=4, fext=(1e-5, 0.0, -2e-5)))
s.step(8, every=2)
np.savez(sys.argv[2], h=s.h, sigma=s.sigma, P=s.P, series=np.array(s.series))
"""


def test_openmp_build_of_the_3d_oracle_is_bitwise_the_serial_one(tmp_path):
    import oracle.o3d as O3
    assert not O3._OPENMP
    path = str(tmp_path / "omp3d.npz")
    env = dict(os.environ, VLB_ORACLE_OPENMP="1", OMP_NUM_THREADS="4")
    subprocess.check_call([sys.executable, "-c", _CHILD3D, ROOT, path], env=env, cwd=ROOT)
    got = np.load(path)
    s = O3.Sim3.from_workload(W.make3d(10, 8, 6, seed=4, fext=(1e-5, 0.0, -2e-5)))
    s.step(8, every=2)
    for k, v in (("h", s.h), ("sigma", s.sigma), ("P", s.P), ("series", np.array(s.series))):
        assert np.array_equal(got[k], v), k

