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

import oracle
from paper_2403_09198_gb300 import inputs
from paper_2403_09198_gb300.binding import StsJacobian, check, load
from tests._gpu import TOL64, dev, host, oracle_jac, rel_err, workload

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
    J = oracle_jac(w)
    rng = np.random.default_rng(7)
    for trans in (False, True):
        for call in range(2):
            xh = rng.standard_normal(w.n)
            xv = xh if layout == "cell" else xh.reshape(w.n_cells, w.b).T.ravel()
            x = dev(np.ascontiguousarray(xv))
            ref = host(jac.matvec(x, trans=trans))
            y = torch.full_like(x, float("nan"))
            check(_noalloc(jac, x, y, trans))
            torch.cuda.synchronize()
            assert rel_err(host(y), ref) <= TOL64, (name, trans, call)
            got = host(y) if layout == "cell" else host(y).reshape(w.b, w.n_cells).T.ravel()
            assert rel_err(got, oracle.matvec(J, xh, trans=trans)) <= TOL64, (name, trans, call)
    jac.close()


def test_noalloc_allocates_nothing_and_keeps_handles_apart():
    """After a first call (which looks up the buffer's address) further calls
    leave the device's free memory unchanged; calls on two handles with
    different numbers of dot tasks, interleaved on one stream, each equal
    sts_jac_matvec, so no call reads scratch entries another call left."""
    import torch
    ws = [workload("grid16_N10"), workload("pairs9_2")]
    jacs = [StsJacobian(w, dev(w.S), dev(w.U), dev(w.V), transpose=True) for w in ws]
    rng = np.random.default_rng(9)
    xs = [dev(rng.standard_normal(w.n)) for w in ws]
    ys = [torch.empty_like(x) for x in xs]
    refs = [[host(j.matvec(x, trans=t)) for t in (False, True)] for j, x in zip(jacs, xs)]
    for j, x, y in zip(jacs, xs, ys):
        check(_noalloc(j, x, y, False))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for rep in range(3):
        for trans in (False, True):
            outs = []
            for j, x in zip(jacs, xs):
                y = torch.full_like(x, float("nan"))
                outs.append(y)
            free_before = torch.cuda.mem_get_info()[0]
            for j, x, y in zip(jacs, xs, outs):
                check(_noalloc(j, x, y, trans))
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info()[0] == free_before
            for k, y in enumerate(outs):
                assert rel_err(host(y), refs[k][int(trans)]) <= TOL64, (k, rep, trans)
    assert torch.cuda.mem_get_info()[0] >= free0 - 64 * 2 ** 20
    for j in jacs:
        j.close()


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
