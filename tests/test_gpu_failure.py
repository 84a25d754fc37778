"""Failure detection without a GPU fault.

Every device-side wait of the library is bounded: the bulk-copy rings of the
structured matvec and apply poll their mbarriers for at most about a second,
then flag the handle and return, and the next synchronous call reports
STS_ERR_TIMEOUT.  Here a wait is made to run out on purpose (an mbarrier phase
that nothing completes, through the same bounded-wait code) and the device is
checked to be usable afterwards.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2403_09198_gb300.binding import StsJacobian, load
from tests._gpu import TOL64, dev, host, oracle_jac, rel_err, workload

pytestmark = pytest.mark.gpu

STS_ERR_TIMEOUT = 7


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def test_bounded_wait_gives_up_and_the_device_stays_usable():
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = load().sts_selftest_bounded_wait(None)
    dt = time.perf_counter() - t0
    assert st == STS_ERR_TIMEOUT, load().sts_last_error()
    assert 0.5 < dt < 30.0
    # the context still runs the library's kernels correctly
    w = workload("grid16_N10")
    jac = StsJacobian(w, dev(w.S), dev(w.U), dev(w.V))
    x = np.random.default_rng(3).standard_normal(w.n)
    y = host(jac.matvec(dev(x)))
    assert rel_err(y, oracle.matvec(oracle_jac(w), x)) <= TOL64
    jac.bjacobi_setup()        # reports a flagged handle; this one has none
    jac.close()
