"""Monte Carlo windows (ems_params.window_samples): the per-sample state of
every sample stays resident while the per-node coefficients and IR work
vectors exist for W samples at a time.  The results must be the full
layout's bit for bit -- the same kernels run on the same numbers, window by
window -- and the oracle's per sample."""
import math

import numpy as np
import pytest

import ems_synth as es
from oracle import flow as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as ge
    ge.build()


def _engine(p, g, **kw):
    from paper_2604_10743_gb300.engine import Engine
    return Engine(p, g, **kw)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_windows_equal_full_layout(prec):
    """10 samples of the uneven 8 x 8 grid in windows of 3 (the last holds
    one): every output equals the full layout's exactly."""
    from paper_2604_10743_gb300 import EMS_F32, EMS_F64
    pr = EMS_F32 if prec == "f32" else EMS_F64
    g = es.mc_grid(n_samples=10)
    p = es.default_params(n_outer=24)
    full = _engine(p, g, precision=pr)
    win = _engine(p, g, precision=pr, window=3)
    assert win.ws_bytes < full.ws_bytes
    rf = full.ttf()
    rw = win.ttf()
    assert rf["graph"] and rw["graph"]
    for k in ("ttf", "final_drop", "drops", "n_voids"):
        assert np.array_equal(rf[k], rw[k]), k
    assert np.array_equal(full.sigma(), win.sigma())
    assert np.array_equal(full.resistance(), win.resistance())
    assert np.array_equal(full.currents(), win.currents())
    vf, vw = full.voids(), win.voids()
    for k in vf:
        assert np.array_equal(vf[k], vw[k]), k
    mf, sf, ssf = full.immortality_check(want_sigma=True)
    mw, sw, ssw = win.immortality_check(want_sigma=True)
    assert np.array_equal(mf, mw) and np.array_equal(sf, sw) and np.array_equal(ssf, ssw)
    assert rw["node_steps"] == rf["node_steps"]
    full.close(); win.close()


def test_windows_host_loop_and_checkpoint():
    """The host-driven loop and a checkpoint taken half way give the same
    bits as the graph run; the resumed half matches too."""
    g = es.mc_grid(n_samples=5)
    p = es.default_params(n_outer=16)
    a = _engine(p, g, window=2)
    b = _engine(p, g, window=2)
    ra = a.ttf(graph=True)
    rb = b.ttf(graph=False)
    assert ra["graph"] and not rb["graph"]
    assert np.array_equal(a.sigma(), b.sigma())
    assert np.array_equal(ra["drops"], rb["drops"])
    c = _engine(p, g, window=2)
    c.ttf(n_outer=8)
    ck = c.state_export()
    rc = c.ttf(n_outer=8)
    d = _engine(p, g, window=2)
    d.state_import(ck)
    rd = d.ttf(n_outer=8)
    assert np.array_equal(c.sigma(), d.sigma())
    assert np.array_equal(rc["drops"], rd["drops"])
    for e in (a, b, c, d):
        e.close()


def test_windows_match_oracle_per_sample():
    """Windows of 2 over 5 samples against the oracle's run of each sample."""
    g = es.mc_grid(n_samples=5)
    p = es.default_params(n_outer=32)
    eng = _engine(p, g, window=2)
    r = eng.ttf()
    sig = eng.sigma()
    g["trees"] = F.build_trees(g)
    v = eng.voids()
    for s in range(5):
        ref = F.run_ttf(g, p, sample=s, keep_state=True)
        assert np.abs(sig[s] - ref["state"].sigma).max() / np.abs(ref["state"].sigma).max() < 1e-9
        m = v["sample"] == s
        assert sorted(zip(v["node"][m].tolist(), v["seg"][m].tolist())) == \
            sorted(zip(ref["void_nodes"].tolist(), ref["void_seg"].tolist()))
        assert abs(r["final_drop"][s] - ref["final_drop"]) <= 5e-4 * ref["final_drop"]
        if math.isfinite(ref["ttf"]):
            assert abs(r["ttf"][s] - ref["ttf"]) <= 5e-4 * ref["ttf"]
        else:
            assert math.isinf(r["ttf"][s])
    eng.close()


def test_windows_reject_reduced_models():
    from paper_2604_10743_gb300 import EMS_KRYLOV, EmsError
    with pytest.raises(EmsError) as e:
        _engine(es.default_params(krylov_q=10), es.mc_grid(n_samples=4), method=EMS_KRYLOV, window=2)
    assert e.value.status == 1
