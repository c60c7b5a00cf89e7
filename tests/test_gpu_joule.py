"""Joule-heating branch profiles (Sec. III-A) on the GPU against the oracle:
the temperature of every stress node, and a coupled aging run whose kappa
and thermomigration term come from that profile."""
import numpy as np
import pytest

import ems_synth as es
from oracle import flow as F
from oracle import joule as J

pytestmark = pytest.mark.gpu

K_CU, K_ILD, T_ILD = 400.0, 1.4, 0.2e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as ge
    ge.build()


def _engine(p, g, **kw):
    from paper_2604_10743_gb300.engine import Engine
    return Engine(p, g, **kw)


@pytest.mark.parametrize("case", ["mesh_map", "mesh_no_map", "T", "comb", "star"])
def test_profile_matches_oracle(case):
    if case.startswith("mesh"):
        g = es.mid_grid(N=32, raster=64)
        g["sink_I"] = g["sink_I"] * 40.0             # a visible Joule rise
        if case == "mesh_no_map":
            g["thermal"] = None
    else:
        g = es.tree_grid(case, cells=9, seed=4, I_sink=20e-3)
    p = es.default_params(T0=345.0)
    eng = _engine(p, g)
    eng.ir_solve()
    eng.joule_profile(K_CU, K_ILD, T_ILD)
    T = eng.node_temperature()
    j = eng.currents()[0]
    tr = F.build_trees(g)
    ref = J.stress_node_temperature(tr, g, p, j, K_CU, K_ILD, T_ILD, g.get("thermal"))
    base = F.node_temperature(tr, g.get("thermal"), p["T0"])
    assert np.abs(ref - base).max() > 0.05              # the profile differs from the map / T0
    assert np.abs(T - ref).max() < 1e-9 * ref.max()
    eng.close()


def test_aging_run_with_joule_profile():
    """One T-shaped tree, 8 aging steps: stress, voids and drops against the
    oracle's run with the same node temperatures."""
    g = es.tree_grid("T", cells=12, seed=5, I_sink=6e-3)
    p = es.default_params(n_outer=8, n_inner=64, sigma_crit=150e6)
    eng = _engine(p, g)
    eng.ir_solve()
    eng.joule_profile(K_CU, K_ILD, T_ILD)
    Tn = eng.node_temperature()
    r = eng.ttf()
    tr = F.build_trees(g)
    ref = F.run_ttf(g, p, keep_state=True, Tn=J.stress_node_temperature(
        tr, g, p, F.current_density(g, F.ir_solve(g, g["seg_R0"]), g["seg_R0"]), K_CU, K_ILD, T_ILD))
    assert Tn.max() > p["T0"] + 0.05                  # heated above ambient
    s = eng.sigma()[0]
    assert np.abs(s - ref["state"].sigma).max() / np.abs(ref["state"].sigma).max() < 1e-9
    v = eng.voids()
    assert sorted(zip(v["node"].tolist(), v["seg"].tolist())) == \
        sorted(zip(ref["void_nodes"].tolist(), ref["void_seg"].tolist()))
    assert np.abs(r["drops"][0] - ref["drops"]).max() < 1e-9
    eng.close()


@pytest.mark.parametrize("window", [0, 2])
def test_per_sample_thermal_perturbation(window):
    """Monte Carlo samples with their own temperature-map perturbation (a
    coarse random raster per sample, +-15 K) on top of the hotspot map and
    the kappa / sigma_crit factors: every sample against the oracle run with
    that sample's node temperatures (base map + its perturbation)."""
    g = es.mc_grid(n_samples=4)
    g["thermal"] = es.hotspot_raster(np.random.default_rng(8), 140e-6, 2, 360.0, 20.0, 40.0, 0.2, nx=33, ny=33)
    th = g["thermal"]
    rng = np.random.default_rng(9)
    dT = rng.uniform(-15.0, 15.0, size=(4, 6, 7))
    p = es.default_params(n_outer=24)
    eng = _engine(p, g, window=window)
    eng.set_thermal_perturbation(dT)
    r = eng.ttf()
    sig = eng.sigma()
    v = eng.voids()
    tr = F.build_trees(g)
    g["trees"] = tr
    base = F.node_temperature(tr, th, p["T0"])
    spread = []
    for s in range(4):
        Tn = base + F.bilinear(dict(T=dT[s], x0=th["x0"], y0=th["y0"], x1=th["x1"], y1=th["y1"]), tr["x"], tr["y"])
        ref = F.run_ttf(g, p, sample=s, keep_state=True, Tn=Tn)
        assert np.abs(sig[s] - ref["state"].sigma).max() / np.abs(ref["state"].sigma).max() < 1e-9
        m = v["sample"] == s
        assert sorted(zip(v["node"][m].tolist(), v["seg"][m].tolist())) == \
            sorted(zip(ref["void_nodes"].tolist(), ref["void_seg"].tolist()))
        assert abs(r["final_drop"][s] - ref["final_drop"]) <= 5e-4 * ref["final_drop"]
        spread.append(ref["n_voids"])
    eng.close()
