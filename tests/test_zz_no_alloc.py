"""sts_jac_matvec_noalloc: the matvec for callers that must not allocate device
memory during the call (fixed memory budgets, or work that cannot take the
device-wide synchronisation cudaMalloc / cudaFree may cause).  Its first-pass
scratch lives in a library-owned static device buffer of 2^19 doubles, shared
by all calls; the result must equal sts_jac_matvec's, call after call.

This file is collected last so that a run that stops at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2403_09198_gb300 import inputs
from paper_2403_09198_gb300.binding import StsJacobian, check, load
from tests._gpu import TOL64, dev, host, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _noalloc(jac, x, y, trans):
    return load().sts_jac_matvec_noalloc(jac.h, ctypes.c_void_p(x.data_ptr()),
                                         ctypes.c_void_p(y.data_ptr()), int(trans))


@pytest.mark.parametrize("name,layout", [("grid16_N10", "cell"), ("grid128_N60", "component")])
def test_noalloc_matches_matvec_on_consecutive_calls(name, layout):
    import torch
    w = inputs.named_workload(name)
    jac = StsJacobian(w, dev(w.S), dev(w.U), dev(w.V), transpose=True, layout=layout)
    rng = np.random.default_rng(7)
    for trans in (False, True):
        for call in range(2):
            x = dev(rng.standard_normal(w.n))
            ref = host(jac.matvec(x, trans=trans))
            y = torch.full_like(x, float("nan"))
            check(_noalloc(jac, x, y, trans))
            torch.cuda.synchronize()
            assert rel_err(host(y), ref) <= TOL64, (name, trans, call)
    jac.close()


def test_noalloc_rejects_handles_beyond_the_static_buffer():
    import torch
    # 200 x 200 cells: 1250 tiles x 21 dot tasks x 32 = 840000 > 2^19 scratch values
    w = inputs.make_workload(200, 200, N=4, w=2, seed=3)
    jac = StsJacobian(w, dev(w.S), dev(w.U), dev(w.V))
    x = dev(np.ones(w.n))
    y = torch.empty_like(x)
    st = _noalloc(jac, x, y, False)
    assert st == 1 and "static buffer" in load().sts_last_error().decode()
    jac.close()
