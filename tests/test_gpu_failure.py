"""Failure detection on the GPU without a fault: the bounded device waits.

A self-test kernel polls an mbarrier that nothing arrives at with the same
bounded wait the TMA row rings use.  The timeout must land in the context's
status word (LB_ERR_TIMEOUT from lb_diagnostics), the context must stay
usable, and lb_set_params clears the status.  The time per poll bounds how
long a stuck row wait can take before the step kernel gives up.
"""
import time

import numpy as np
import pytest

from paper_1806_10241_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_10241_gb300 import build
    build.build()


def test_bounded_wait_timeout_reaches_the_status_word_and_the_context_survives():
    from paper_1806_10241_gb300 import _abi
    from paper_1806_10241_gb300.solver import Solver
    c = W.swirling_cylinder(nr=70, nz=64, Re=200.0, Ra=1e4, amp=1e-3, seed=2)
    s = Solver(c.params, storage="fp32")
    s.init_fields(c.fields)
    s.step(10)
    assert s.diag()["status"] == _abi.LB_OK
    t = time.perf_counter()
    _abi.check(s.L.lb_selftest_timeout(s.ctx, 64))
    per_poll = (time.perf_counter() - t) / 64
    assert s.diag()["status"] == _abi.LB_ERR_TIMEOUT
    # 2^18 polls (the limit of the row waits) must end within seconds
    assert per_poll * (1 << 18) < 10.0, per_poll
    assert s.L.lb_selftest_timeout(s.ctx, 0) == _abi.LB_ERR_ARG
    # the context stays usable: a reset clears the status and steps run again
    s.reset()  # lb_set_params: rest state, status cleared
    assert s.diag()["status"] == _abi.LB_OK
    s.init_fields(c.fields)
    s.step(10)
    d = s.diag()
    assert d["status"] == _abi.LB_OK and np.isfinite(d["nu_avg"])
    ref = Solver(c.params, storage="fp32")
    ref.init_fields(c.fields)
    ref.step(10)
    assert np.array_equal(ref.get_dist(), s.get_dist())
