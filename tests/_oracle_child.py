"""Runs a seeded workload on the FP64 oracle built with OpenMP, in a child process (test
infrastructure: the OpenMP build is chosen when the oracle package is imported, and its results
are bitwise the serial build's, see test_oracle_openmp.py).  The child is a fresh interpreter
started by exec, so it inherits no CUDA state from the test process."""
import json
import os
import subprocess
import sys
import tempfile

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import oracle as O
from paper_2209_14889_gb300 import workloads as W
assert O._OPENMP
w = getattr(W, sys.argv[2])(**json.loads(sys.argv[3]))
sim = O.Sim.from_workload(w)
sim.step(int(sys.argv[4]), every=int(sys.argv[5]))
out = {"f_" + k: v for k, v in sim.fields().items()}
out["X"] = sim.X
out["series"] = np.array(sim.series)
np.savez(sys.argv[6], **out)
"""


def run_openmp(recipe: str, kwargs: dict, steps: int, every: int) -> dict:
    """fields (dict), series and X of `recipe(**kwargs)` after `steps` oracle steps."""
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "out.npz")
        env = dict(os.environ, VLB_ORACLE_OPENMP="1", OMP_NUM_THREADS=str(os.cpu_count() or 1))
        subprocess.check_call([sys.executable, "-c", _CHILD, ROOT, recipe, json.dumps(kwargs), str(steps),
                               str(every), path], env=env, cwd=ROOT)
        z = np.load(path)
        return dict(fields={k[2:]: z[k] for k in z.files if k.startswith("f_")}, series=z["series"], X=z["X"])
