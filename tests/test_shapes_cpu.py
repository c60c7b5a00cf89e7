"""Host logic of the chain shapes the autotuner picks from (no GPU): every
candidate holds the whole chain in whole warps within its kernel's thread
limit, the built-in choice comes first, and shape rules change the packed
layout (and so the workspace) only where they fit the chains."""
import ctypes

import pytest

import ems_synth as es


@pytest.fixture(scope="module")
def A():
    from paper_2604_10743_gb300 import build as B
    from paper_2604_10743_gb300 import _abi as A
    B.build()
    A.lib()
    return A


def _check_candidate(r, n, prec):
    M, CL, T = r["M"], r["CL"], r["T"]
    assert M in (4, 8, 16, 32, 64)
    assert T * M >= n                              # every node has a slot
    assert T % (32 * CL) == 0                       # whole warps in every CTA
    tc = T // CL
    if r["kernel"] == "cluster":
        assert 2 <= CL <= 8 and tc <= 320
        assert M == (16 if prec == 1 else 8)
        assert (CL - 1) * tc * M < n                # no CTA without nodes
    elif r["kernel"] == "cluster_shared":
        assert prec == 1 and M == 16 and CL in (2, 4, 5, 6, 8)
        assert tc <= (256 if CL in (5, 6) else 320)
        assert (CL - 1) * tc * M < n
        assert 2 * (20 * tc * M + 9 * 1024) <= 228 * 1024   # two CTAs' shared memory on one SM
    else:
        assert CL == 1
        assert T - 32 < -(-n // M)                  # the smallest team in whole warps
    if r["kernel"] == "register":
        assert prec == 1 and T <= {4: 896, 8: 576, 16: 320}[M]
    if r["kernel"] == "shared":
        assert prec == 1 and 5 * 4 * T * M <= 200 * 1024


@pytest.mark.parametrize("n,prec", [(281, 0), (281, 1), (5101, 1), (5101, 0), (20471, 1), (20471, 0), (1, 1),
                                    (64, 0), (16385, 0)])
def test_candidates_hold_the_chain(A, n, prec):
    c = A.chain_candidates(n, prec)
    assert c, n
    for r in c:
        _check_candidate(r, n, prec)
    keys = [(r["kind"], r["M"], r["CL"]) for r in c]
    assert len(keys) == len(set(keys))


def test_builtin_choice_first(A):
    # full-chip stripes: a 4-CTA cluster in FP32 (coefficients in shared memory), 8 CTAs in FP64
    c32 = A.chain_candidates(20471, 1)
    assert (c32[0]["kernel"], c32[0]["M"], c32[0]["CL"], c32[0]["T"]) == ("cluster_shared", 16, 4, 1280)
    assert {(r["kernel"], r["M"], r["CL"]) for r in c32} >= {("cluster", 16, 4), ("cluster", 16, 5), ("cluster", 16, 6),
                                                          ("cluster", 16, 8), ("global", 32, 1), ("global", 64, 1)}
    assert all(r["T"] // r["CL"] <= 256 for r in c32 if r["kernel"] == "cluster" and r["CL"] in (5, 6))
    # the same clusters with the coefficients in shared memory
    assert {(r["CL"], r["T"]) for r in c32 if r["kernel"] == "cluster_shared"} == {(4, 1280), (5, 1280), (6, 1344),
                                                                                  (8, 1280)}
    assert not any(r["kernel"] == "cluster_shared" for r in A.chain_candidates(20471, 0))
    c64 = A.chain_candidates(20471, 0)
    assert (c64[0]["kernel"], c64[0]["CL"]) == ("cluster", 8)
    # mid-grid stripes: 16 nodes per thread in registers, 320 threads
    m = A.chain_candidates(5101, 1)
    assert (m[0]["kernel"], m[0]["M"], m[0]["T"]) == ("register", 16, 320)
    assert any(r["kernel"] == "cluster" and r["CL"] == 2 for r in m)


def _ws(A, g, rules, **kw):
    prm = A.make_params(es.default_params(), **kw)
    gd = A.GridDesc(g)
    arr = A.rules_array(rules)
    return A.lib().ems_workspace_bytes_rules(ctypes.byref(prm), ctypes.byref(gd.desc), arr, len(rules))


def test_rules_change_the_layout_only_where_they_fit(A):
    g = es.tiny_grid()                              # 16 stripes of 281 stress nodes
    base = _ws(A, g, [])
    assert base > 0
    # 64 nodes per thread: a 32-thread team of 2,048 slots per chain instead of 288
    wide = _ws(A, g, [dict(n_lo=1, n_hi=10**6, kind=1, M=64, CL=1)], precision=A.EMS_F64)
    assert wide > base
    # a rule outside the chains' lengths, or a shape they cannot take, changes nothing
    assert _ws(A, g, [dict(n_lo=300, n_hi=400, kind=1, M=64, CL=1)]) == base
    assert _ws(A, g, [dict(n_lo=1, n_hi=10**6, kind=3, M=16, CL=1)], precision=A.EMS_F64) == base
    # malformed rules are rejected
    assert _ws(A, g, [dict(n_lo=1, n_hi=10**6, kind=1, M=12, CL=1)]) == 0
    assert _ws(A, g, [dict(n_lo=1, n_hi=10**6, kind=4, M=8, CL=9)]) == 0
    assert _ws(A, g, [dict(n_lo=1, n_hi=10**6, kind=5, M=16, CL=1)]) == 0
    assert _ws(A, g, [dict(n_lo=1, n_hi=10**6, kind=6, M=16, CL=2)]) == 0
    assert _ws(A, g, [dict(n_lo=5, n_hi=4, kind=1, M=8, CL=1)]) == 0


def test_tuning_cache_key():
    """The tuned-shape cache is keyed by what the chain lengths and launch
    sizes depend on: the same grid gives the same key, a changed
    discretisation, sample count, window or precision another."""
    import numpy as np
    from paper_2604_10743_gb300 import tune
    g = es.mc_grid(n_samples=4)
    k = tune.grid_key(g, 1)
    assert k == tune.grid_key(dict(g), 1)
    g2 = dict(g)
    g2["seg_cells"] = np.array(g["seg_cells"]) + 1
    assert tune.grid_key(g2, 1) != k
    assert tune.grid_key(es.mc_grid(n_samples=5), 1) != k
    assert tune.grid_key(g, 1, window=2) != k
    assert tune.grid_key(g, 0) != k
