"""Failure detection without a GPU fault: a bounded device wait that runs out
reports PF_ETIMEOUT to the host and leaves the context usable.

pf_selftest_wait makes one thread wait on a shared-memory mbarrier that no
thread arrives on, with the poll loop the TMA-staged kernels use (their
waits give up after 2^22 polls and raise the same flag)."""
import time

import numpy as np
import pytest

from paper_2601_16522_gb300 import inputs as I

from test_gpu_parity import pf  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu

PF_EINVAL, PF_ETIMEOUT = 1, 4


def test_bounded_wait_times_out_and_context_survives(pf):
    import torch
    t0 = time.perf_counter()
    assert pf.selftest_wait(1 << 16) == PF_ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    assert pf.selftest_wait(1 << 10, stream=torch.cuda.Stream()) == PF_ETIMEOUT
    assert pf.selftest_wait(0) == PF_EINVAL and pf.selftest_wait(1 << 23) == PF_EINVAL
    # the context is intact: a normal run afterwards is well defined
    prob, u = I.circle(32, 9.0, W=2.5)
    with pf.Simulation(prob, precision=64) as sim:
        sim.set_state(u)
        st = sim.step(pf.FEULER, 10 * 0.9 * sim.dt_e(), dt_mult=0.9)
        ug, _ = sim.get_state()
    assert st["rhs_evals"] == 10 and np.isfinite(ug).all()
    assert np.abs(ug.sum(0) - 1.0).max() < 1e-12
