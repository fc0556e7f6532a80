"""The bounded device waits of the sweeps give up with a status instead of hanging.

The tensor-core sweep waits on an mbarrier for its MMAs and the cooperative sweep (every tick
of Algorithm 1 in one launch) on a grid barrier between ticks.  mdl_selftest_wait runs each wait
on a phase or a count that nothing completes; the test checks the reported status, that the
wait ended in bounded time, and that the device then still steps a simulation (the context is
not lost).  No fault is raised: the wait only runs out of polls.
"""
import numpy as np
import pytest

import workloads as W
from paper_2310_07607_gb300 import mdl

pytestmark = pytest.mark.gpu

MDL_E_TIMEOUT = -6


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_wait_gives_up_and_device_stays_usable(which):
    status, ms = mdl.selftest_wait(which)
    assert status == MDL_E_TIMEOUT
    assert 0.0 < ms < 30000.0
    # the device still runs the sweep (plain FP64 2D workload, a few barriers under the stimulus)
    sim = mdl.Sim(W.plain_2d_q1_32x32())
    sim.step_barriers(5)
    V = sim.read_V()
    assert np.all(np.isfinite(V)) and V.max() > 0.0


def test_selftest_rejects_unknown_wait():
    with pytest.raises(mdl.MdlError):
        mdl.selftest_wait(7)
