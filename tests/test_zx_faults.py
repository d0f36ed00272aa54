"""Failure detection without a GPU fault: a non-finite value written into the state from the
host is reported by lb_sync as LB_ENONFINITE after the next readout step, and the flags are
cleared once reported.  The value sits far from the ring (35 cells; one step carries it at most
4 cells), so the node positions stay finite."""
import numpy as np
import pytest

from paper_2209_14889_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_14889_gb300 import lb
    return lb


@pytest.mark.parametrize("value", [np.nan, np.inf])
def test_host_injected_non_finite_is_reported(value):
    lb = _gpu()
    w = W.make(64, 48, rings=[W.ring(20, 4.0, (15.3, 24.1), pull_force=1e-3)], seed=2)
    s = lb.Solver.from_workload(w)
    sxx = s.readout("sxx", device=False).copy()
    sxx[24, 50] = value
    s.write_field("sxx", sxx)
    s.step(1)                                   # t = 0 is a readout step
    with pytest.raises(lb.LBError) as e:
        s.sync()
    assert e.value.code == lb.LB_ENONFINITE
    assert np.isfinite(s.nodes()).all()
    s.sync()                                    # reported once, then cleared
    s.close()
