"""Loading a grid: the plan ems_workspace_bytes makes is kept for the
following ems_load_grid of the same inputs (one planning per load).  A load
that reuses it must give the same context, bit for bit, as one that plans
again; and an input array changed in place between the size query and the
load must not reuse it."""
import ctypes

import numpy as np
import pytest

import ems_synth as es
from oracle import flow as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as ge
    ge.build()


def _query(g):
    from paper_2604_10743_gb300 import _abi as A
    prm = A.make_params(es.default_params())
    gd = A.GridDesc(g)
    return A.lib().ems_workspace_bytes(ctypes.byref(prm), ctypes.byref(gd.desc))


class _Replan:
    """Engine whose load plans again: a size query for another grid runs
    between its own size query and its load (the cache holds one plan)."""
    def __new__(cls, p, g, other):
        from paper_2604_10743_gb300 import _abi as A
        from paper_2604_10743_gb300.engine import Engine
        L = A.lib()
        orig = L.ems_load_grid

        def load(ctx, desc):
            assert _query(other) > 0
            return orig(ctx, desc)
        L.ems_load_grid = load
        try:
            return Engine(p, g)
        finally:
            L.ems_load_grid = orig


def test_cached_plan_equals_fresh_plan():
    from paper_2604_10743_gb300.engine import Engine
    g = es.mc_grid(n_samples=4)
    p = es.default_params(n_outer=8)
    a = Engine(p, g)                                   # size query, then a load that reuses its plan
    b = _Replan(p, g, es.tiny_grid())
    ra, rb = a.ttf(), b.ttf()
    assert np.array_equal(a.sigma(), b.sigma())
    assert np.array_equal(ra["drops"], rb["drops"]) and np.array_equal(ra["ttf"], rb["ttf"])
    va, vb = a.voids(), b.voids()
    assert np.array_equal(va["node"], vb["node"]) and np.array_equal(va["volume"], vb["volume"])
    a.close(); b.close()


def test_changed_input_misses_the_cache():
    """The segment lengths change in place after the size query (sizes stay,
    the faces' spacing changes): the load plans again, and the stress run
    matches the oracle's with the new lengths, not the old ones."""
    from paper_2604_10743_gb300 import _abi as A
    from paper_2604_10743_gb300.engine import Engine
    g = dict(es.mid_grid(N=32, with_map=False))
    g["seg_L"] = np.array(g["seg_L"], dtype=np.float64)
    L = A.lib()
    orig = L.ems_load_grid
    L_new = g["seg_L"] * 1.25

    def load(ctx, desc):
        g["seg_L"][:] = L_new                          # same array, new values, after the size query
        return orig(ctx, desc)
    L.ems_load_grid = load
    p = es.default_params(n_outer=4)
    try:
        e = Engine(p, g)
    finally:
        L.ems_load_grid = orig
    e.ttf()
    ref = F.run_ttf(g, p, keep_state=True)          # g holds the new lengths
    assert np.abs(e.sigma()[0] - ref["state"].sigma).max() < 1e-9 * np.abs(ref["state"].sigma).max()
    e.close()
