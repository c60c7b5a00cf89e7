"""Chain shapes and the autotuner on the GPU (the batching form: the shape of
every size group's eliminations picked by measurement).  Every shape a
chain can take solves the same backward-Euler system, so each one must give
the oracle's result at the parity bar; ems_autotune must leave the context
exactly as it found it; and a table it returns, applied by loading again,
changes nothing but the time."""
import math

import numpy as np
import pytest

import ems_synth as es
from oracle import flow as F

pytestmark = pytest.mark.gpu

TOL64 = 1e-9
TOL32 = 1e-4
TTF_TOL = 5e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as ge
    ge.build()


def _relerr(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300)


def _voids(eng, sample=0):
    v = eng.voids()
    m = v["sample"] == sample
    return sorted(zip(v["node"][m].tolist(), v["seg"][m].tolist()))


@pytest.mark.parametrize("prec", [0, 1])
def test_every_shape_matches_the_oracle(prec):
    """The 16 stripes of 281 stress nodes of the 8 x 8 grid, the whole TTF
    run, once per valid shape (streaming with 4-64 nodes per thread, FP32
    register and shared-memory variants, a 2-CTA cluster)."""
    from paper_2604_10743_gb300 import _abi as A
    from paper_2604_10743_gb300.engine import Engine
    g = es.tiny_grid()
    p = es.default_params()
    ref = F.run_ttf(g, p, keep_state=True)
    n = int(np.diff(ref["trees"]["off"]).max())
    assert n == int(np.diff(ref["trees"]["off"]).min()) == 281
    cands = A.chain_candidates(n, prec)
    kinds = {r["kernel"] for r in cands}
    assert kinds >= ({"global", "cluster"} if prec == 0 else {"global", "shared", "register"})
    ora = sorted(zip(ref["void_nodes"].tolist(), ref["void_seg"].tolist()))
    assert len(ora) >= 10
    checked = 0
    for r in cands:
        rule = dict(r, n_lo=1, n_hi=10 ** 9)
        eng = Engine(p, g, precision=prec, chain_rules=[rule])
        res = eng.ttf()
        err = _relerr(eng.sigma()[0], ref["state"].sigma)
        tag = "%s M=%d CL=%d" % (r["kernel"], r["M"], r["CL"])
        if prec == 0:
            assert err < TOL64, tag
            assert _voids(eng) == ora, tag
            assert abs(res["ttf"][0] - ref["ttf"]) <= 1e-6 * ref["ttf"], tag
        else:
            assert err < TOL32, tag
            assert abs(len(_voids(eng)) - len(ora)) <= 2, tag
            metric = "ttf" if math.isfinite(ref["ttf"]) else "final_drop"
            assert abs(res[metric][0] - ref[metric]) <= TTF_TOL * ref[metric], tag
        checked += 1
        eng.close()
    assert checked == len(cands) >= 5


def _state(eng):
    v = eng.voids()
    return eng.sigma(), eng.resistance(), v["node"].copy(), v["volume"].copy(), v["t_nuc"].copy()


@pytest.mark.parametrize("window", [0, 2])
def test_autotune_leaves_the_context_unchanged(window):
    """Uneven stripes (32-1,024 cells), 4 Monte Carlo samples, after two
    aging steps with voids: the tuner times every shape of every group on
    scratch copies; the state before and after is bit-identical, and the run
    continues exactly as an untuned twin's."""
    from paper_2604_10743_gb300.engine import Engine
    g = es.mc_grid(n_samples=4)
    p = es.default_params(n_outer=8)
    eng = Engine(p, g, window=window)
    twin = Engine(p, g, window=window)
    eng.ttf(n_outer=3)
    twin.ttf(n_outer=3)
    before = _state(eng)
    assert before[2].size > 0
    table = eng.autotune(n_steps=16, max_samples=2)
    after = _state(eng)
    for x, y in zip(before, after):
        assert np.array_equal(x, y)
    assert len(table) >= 3                          # groups of different chain lengths
    for r in table:
        assert 1 <= r["n_lo"] <= r["n_hi"] and r["T"] * r["M"] >= r["n_hi"]
        assert 0.0 < r["ms"] <= r["ms_default"]
    # the log holds every shape timed; each group's rule is its fastest, or
    # the built-in shape when nothing beat it by 3 %
    log = eng.autotune_log()
    assert len(log) > len(table)
    for k, r in enumerate(table):
        times = [e["ms"] for e in log if e["group"] == k and e["ms"] > 0]
        assert r["ms"] == min(times) or (r["ms"] == r["ms_default"] and min(times) > 0.97 * r["ms_default"])
    ra = eng.ttf()
    rb = twin.ttf()
    assert _relerr(eng.sigma(), twin.sigma()) < 1e-12
    assert np.array_equal(ra["n_voids"], rb["n_voids"])
    eng.close(); twin.close()


def test_tuned_engine_cache_and_parity(tmp_path):
    """tuned_engine measures once, stores the table under the grid's key and
    reads it back; the tuned context matches the oracle like the default one."""
    from paper_2604_10743_gb300 import tune
    g = es.mc_grid(n_samples=0)
    p = es.default_params()
    cache = str(tmp_path / "shapes.json")
    e1 = tune.tuned_engine(p, g, cache=cache, n_steps=16, max_samples=1)
    assert e1.tune_measured and len(e1.tune_table) >= 3
    e2 = tune.tuned_engine(p, g, cache=cache, n_steps=16, max_samples=1)
    assert not e2.tune_measured and e2.tune_table == e1.tune_table
    r = e2.ttf()
    ref = F.run_ttf(g, p, keep_state=True)
    assert _relerr(e2.sigma()[0], ref["state"].sigma) < TOL64
    assert _voids(e2) == sorted(zip(ref["void_nodes"].tolist(), ref["void_seg"].tolist()))
    metric = "ttf" if math.isfinite(ref["ttf"]) else "final_drop"
    assert abs(r[metric][0] - ref[metric]) <= 1e-6 * ref[metric]
    e1.close(); e2.close()



def test_cluster_shapes_on_full_chip_length_stripes():
    """FP32 stripes of the full chip's length (20,469 stress nodes) on every
    cluster shape the autotuner may pick -- coefficients in registers (one
    CTA per SM) or in shared memory (two per SM), 4 to 8 CTAs a chain --
    against one oracle run: stress at the FP32 bar, every tree's voids
    within two nodes of the oracle's, TTF / final drop at 0.05 %.  A
    shared-memory kernel does the register kernel's arithmetic in the same
    order; the two compiled forms may contract a product into an addition
    differently, so on the same cluster they agree at the FP32 bar (measured
    on 8 CTAs: 7.2e-6)."""
    from paper_2604_10743_gb300 import _abi as A
    from paper_2604_10743_gb300.engine import Engine
    g = es.stripe_mesh(8, 20e-6)
    g["seg_cells"][:] = 2924
    t = es.tiny_grid()
    g["pad_node"], g["pad_V"], g["sink_node"], g["sink_I"] = t["pad_node"], t["pad_V"], t["sink_node"], t["sink_I"]
    g["thermal"] = es.hotspot_raster(np.random.default_rng(2924), 140e-6, 2, 360.0, 20.0, 40.0, 0.2, nx=33, ny=33)
    p = es.default_params(n_outer=3, n_inner=64, sigma_crit=250e6)
    ref = F.run_ttf(g, p, keep_state=True, n_threads=8)
    assert ref["n_voids"] >= 16
    off = ref["trees"]["off"]
    n = int(np.diff(off).max())
    assert n == 20469
    cands = [r for r in A.chain_candidates(n, 1) if r["kernel"] in ("cluster", "cluster_shared")]
    assert {(r["kernel"], r["CL"]) for r in cands} >= {("cluster", 4), ("cluster_shared", 4), ("cluster_shared", 5),
                                                        ("cluster_shared", 8)}
    metric = "ttf" if math.isfinite(ref["ttf"]) else "final_drop"
    sig = {}
    for r in cands:
        rule = dict(r, n_lo=1, n_hi=10 ** 9)
        eng = Engine(p, g, precision=1, max_voids=64, chain_rules=[rule])
        res = eng.ttf()
        tag = "%s CL=%d" % (r["kernel"], r["CL"])
        s = eng.sigma()[0]
        assert _relerr(s, ref["state"].sigma) < TOL32, tag
        v = eng.voids()
        for k in range(len(off) - 1):
            gv = sorted(x for x in v["node"].tolist() if off[k] <= x < off[k + 1])
            ov = sorted(x for x in ref["void_nodes"].tolist() if off[k] <= x < off[k + 1])
            assert len(gv) == len(ov), (tag, k)
            assert all(abs(a - b) <= 2 for a, b in zip(gv, ov)), (tag, k)
        assert abs(res[metric][0] - ref[metric]) <= TTF_TOL * ref[metric], tag
        sig[(r["kernel"], r["CL"])] = s
        eng.close()
    for (kind, cl), s in sig.items():
        if kind == "cluster_shared" and ("cluster", cl) in sig:
            assert _relerr(s, sig[("cluster", cl)]) < TOL32, cl
