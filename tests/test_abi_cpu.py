"""C ABI checks that need no GPU: the library loads, exports every entry point
declared in include/sts.h, and rejects malformed problem statements before it
makes any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2403_09198_gb300 import binding, build, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "sts.h")).read()
    return sorted(set(re.findall(r"^\s*(?:sts_status|const char \*)\s*(sts_\w+)\s*\(", text, re.M)))


def test_header_lists_the_binding_functions():
    assert _declared() == sorted(binding.ABI_FUNCTIONS)


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    assert lib.sts_version().startswith(b"sts-gb300")
    assert lib.sts_last_error() is not None


def test_struct_layouts_match_header(lib):
    # int fields then pointers: a mismatch would shift the pointers
    assert ctypes.sizeof(binding.sts_jac_desc) == 6 * 4 + 6 * 8 + 2 * 4 + 8 + 3 * 8 + 2 * 4 + 8
    # three ints, the double (8-aligned), then the two operator counts
    assert ctypes.sizeof(binding.sts_gmres_info) == 4 * 4 + 8 + 2 * 4
    assert binding.sts_gmres_info.true_rel_residual.offset == 16
    assert binding.sts_gmres_info.matvecs.offset == 24 and binding.sts_gmres_info.applies.offset == 28


def _desc(w, **kw):
    idx = [np.ascontiguousarray(a, dtype=np.int32) for a in
           (w.block_indptr, w.block_indices, w.d_indptr, w.d_indices, w.o_indptr, w.o_indices)]
    d = binding.sts_jac_desc()
    d.n_cells = w.n_cells
    d.block_size = w.b
    (d.block_indptr, d.block_indices, d.d_indptr, d.d_indices, d.o_indptr,
     d.o_indices) = [a.ctypes.data for a in idx]
    d.r_diag, d.r_off = w.r_diag, w.r_off
    d.S, d.U, d.V = w.S.ctypes.data, w.U.ctypes.data, w.V.ctypes.data
    d.values_on_host = 1
    for k, v in kw.items():
        setattr(d, k, v)
    return d, idx


def _create(lib, d):
    h = ctypes.c_void_p()
    st = lib.sts_jac_create(ctypes.byref(d) if d is not None else None, ctypes.byref(h))
    return st, h, lib.sts_last_error().decode()


def test_create_rejects_malformed_input_on_the_host(lib):
    w = inputs.make_workload(3, 2, N=2, w=1, seed=0)
    st, h, msg = _create(lib, None)
    assert st == 1 and not h.value and "desc" in msg
    d, keep = _desc(w, n_cells=0)
    assert _create(lib, d)[0] == 1
    d, keep = _desc(w, dtype=7)
    assert _create(lib, d)[0] == 1
    # unsorted block row
    bi = w.block_indices.copy()
    bi[0], bi[1] = bi[1], bi[0]
    w2 = inputs.make_workload(3, 2, N=2, w=1, seed=0)
    w2.block_indices = bi
    d, keep = _desc(w2)
    st, h, msg = _create(lib, d)
    assert st == 1 and "ascending" in msg
    # diagonal entry missing from the diagonal-block pattern
    w3 = inputs.make_workload(3, 2, N=2, w=1, seed=0)
    dp, di = w3.d_indptr.copy(), w3.d_indices.copy()
    keep_rows = [e for e in range(di.shape[0]) if not (e < dp[1] and di[e] == 0)]
    w3.d_indices = di[keep_rows]
    w3.d_indptr = dp - np.array([0] + [1] * (dp.shape[0] - 1))
    d, keep = _desc(w3)
    st, h, msg = _create(lib, d)
    assert st == 1 and "diagonal" in msg
    # column out of range in the off-diagonal pattern
    w4 = inputs.make_workload(3, 2, N=2, w=1, seed=0)
    w4.o_indices = w4.o_indices.copy()
    w4.o_indices[-1] = w4.b + 3
    d, keep = _desc(w4)
    st, h, msg = _create(lib, d)
    assert st == 1 and "out of range" in msg


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.sts_jac_bjacobi_setup(None) == 1
    assert lib.sts_jac_destroy(None) == 0
    n = ctypes.c_size_t()
    assert lib.sts_jac_memory(None, ctypes.byref(n)) == 1


def test_flow_create_rejects_malformed_input_on_the_host(lib):
    c = inputs.make_flow_case(3, 2, N=4, w=1, seed=0)
    keep = [np.ascontiguousarray(a, dtype=np.float64) for a in (c.r, c.cv, c.e0, c.beta, c.ws, c.K)]

    def desc(**kw):
        d = binding.sts_flow_desc()
        d.Lx, d.Ly, d.n_species, d.band = c.Lx, c.Ly, c.N, c.w
        d.r, d.cv, d.e0, d.beta, d.ws, d.K = [a.ctypes.data for a in keep]
        d.A, d.theta, d.dt = c.A, c.theta, c.dt
        for k, v in kw.items():
            setattr(d, k, v)
        return d

    def create(d):
        h = ctypes.c_void_p()
        st = lib.sts_flow_create(ctypes.byref(d) if d is not None else None, ctypes.byref(h))
        return st, h, lib.sts_last_error().decode()

    assert ctypes.sizeof(binding.sts_flow_desc) == 4 * 4 + 6 * 8 + 3 * 8 + 8
    assert ctypes.sizeof(binding.sts_flow_sizes) == 6 * 4 + 8
    st, h, msg = create(None)
    assert st == 1 and not h.value and "desc" in msg
    for kw, what in ((dict(Lx=0), ">= 1"), (dict(n_species=0), ">= 1"), (dict(band=-1), "band"),
                     (dict(n_species=254), "256"), (dict(cv=None), "NULL"), (dict(dt=float("nan")), "dt")):
        st, h, msg = create(desc(**kw))
        assert st == 1 and not h.value and what in msg, (kw, msg)
    bad = keep[1].copy()
    bad[2] = 0.0
    st, h, msg = create(desc(cv=bad.ctypes.data))
    assert st == 1 and "cv[2]" in msg
    for fn, args in (("sts_flow_residual", (None, None, None, None)),
                     ("sts_flow_jacobian", (None, None, None, None, None)),
                     ("sts_flow_get_sizes", (None, None))):
        assert getattr(lib, fn)(*args) == 1
    assert lib.sts_flow_destroy(None) == 0
