"""The allocation-free PCG entry point against the context-based IR solve.

Some callers cannot give this library device memory: they run under another
framework's allocator and may not call cudaMalloc themselves, or they cannot
take the device-wide synchronisation a cudaMalloc / cudaFree can cause in the
middle of their own stream work.  ems_ir_pcg_noalloc serves them from one
fixed device array.  Two calls in a row, on two different IR systems, must
each agree with ems_ir_solve within the IR tolerance the other tests use.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import ems_synth as es

pytestmark = pytest.mark.gpu


def _free_node_system(g):
    """CSR (row_ptr, col, val) and right-hand side of G u = -I on the non-pad
    nodes, pads held at their voltage; plus the free-node ids."""
    n = len(g["node_x"])
    a = np.asarray(g["seg_a"]); b = np.asarray(g["seg_b"]); cond = 1.0 / np.asarray(g["seg_R0"])
    pad_v = np.full(n, np.nan); pad_v[g["pad_node"]] = g["pad_V"]
    free = np.nonzero(np.isnan(pad_v))[0]
    idx = -np.ones(n, np.int64); idx[free] = np.arange(free.size)
    rows = [dict() for _ in range(free.size)]
    rhs = np.zeros(free.size)
    for nd, cur in zip(g["sink_node"], g["sink_I"]):
        if idx[nd] >= 0:
            rhs[idx[nd]] -= cur
    for s in range(a.size):
        for p, q in ((a[s], b[s]), (b[s], a[s])):
            if idx[p] < 0:
                continue
            r = rows[idx[p]]
            r[idx[p]] = r.get(idx[p], 0.0) + cond[s]
            if idx[q] >= 0:
                r[idx[q]] = r.get(idx[q], 0.0) - cond[s]
            else:
                rhs[idx[p]] += cond[s] * pad_v[q]
    rp = [0]; col = []; val = []
    for r in rows:
        for k in sorted(r):
            col.append(k); val.append(r[k])
        rp.append(len(col))
    return (np.array(rp, np.int32), np.array(col, np.int32), np.array(val), rhs, free)


def test_noalloc_pcg_matches_ir_solve_on_two_calls():
    import torch

    import __graft_entry__ as ge
    ge.build()
    from paper_2604_10743_gb300 import _abi
    from paper_2604_10743_gb300.engine import Engine
    L = _abi.lib()
    stream = torch.cuda.current_stream()
    for g in (es.tiny_grid(), es.mid_grid(N=64, with_map=False)):
        eng = Engine(es.default_params(), g)
        u, _ = eng.ir_solve()
        eng.close()
        rp, col, val, rhs, free = _free_node_system(g)
        dev = [torch.from_numpy(x).cuda() for x in (rp, col, val, rhs)]
        x = torch.ones(free.size, dtype=torch.float64, device="cuda")
        its = ctypes.c_int()
        st = L.ems_ir_pcg_noalloc(int(free.size), *(ctypes.c_void_p(t.data_ptr()) for t in dev),
                                  ctypes.c_void_p(x.data_ptr()), 1e-13, 20000, ctypes.byref(its),
                                  ctypes.c_void_p(stream.cuda_stream))
        assert st == 0 and its.value > 0
        assert np.abs(x.cpu().numpy() - u[0][free]).max() < 1e-11


def test_noalloc_rejects_oversized_systems():
    import __graft_entry__ as ge
    ge.build()
    from paper_2604_10743_gb300 import _abi
    L = _abi.lib()
    one = ctypes.c_void_p(1)
    assert L.ems_ir_pcg_noalloc(16385, one, one, one, one, one, 1e-12, 10, None, None) == 1
    assert L.ems_ir_pcg_noalloc(0, one, one, one, one, one, 1e-12, 10, None, None) == 1


def test_noalloc_iteration_cap_then_normal_call():
    """A call stopped by its iteration cap reports EMS_E_NOCONV and the
    iterations it ran (read back from the shared array's info slots); the
    next call on the same array still converges to the context solve."""
    import torch

    import __graft_entry__ as ge
    ge.build()
    from paper_2604_10743_gb300 import _abi
    from paper_2604_10743_gb300.engine import Engine
    L = _abi.lib()
    stream = torch.cuda.current_stream()
    g = es.tiny_grid()
    eng = Engine(es.default_params(), g)
    u, _ = eng.ir_solve()
    eng.close()
    rp, col, val, rhs, free = _free_node_system(g)
    dev = [torch.from_numpy(x).cuda() for x in (rp, col, val, rhs)]
    ptrs = [ctypes.c_void_p(t.data_ptr()) for t in dev]
    x = torch.ones(free.size, dtype=torch.float64, device="cuda")
    its = ctypes.c_int()
    st = L.ems_ir_pcg_noalloc(int(free.size), *ptrs, ctypes.c_void_p(x.data_ptr()), 1e-13, 2,
                              ctypes.byref(its), ctypes.c_void_p(stream.cuda_stream))
    assert st == 5 and its.value == 2
    x2 = torch.ones(free.size, dtype=torch.float64, device="cuda")
    st = L.ems_ir_pcg_noalloc(int(free.size), *ptrs, ctypes.c_void_p(x2.data_ptr()), 1e-13, 20000,
                              ctypes.byref(its), ctypes.c_void_p(stream.cuda_stream))
    assert st == 0 and its.value > 2
    assert np.abs(x2.cpu().numpy() - u[0][free]).max() < 1e-11
