"""Pins of the oracle's event logic: which segment a void degrades, the Monte
Carlo factor mapping, the cadence of the coupled aging loop, and Adam beyond
its first step.

Each case is checked against values fixed by hand from the grid's definition
(stripe numbering, the canonical node order) or by a closed form, not by
re-running the oracle's own rule.
"""
import math

import numpy as np
import pytest

import ems_synth as es
from oracle import flow as F
from oracle import mlp

P = es.default_params()


# ---------------------------------------------------------------------------
# Void segment (reading of Sec. III-D.3 / IV-C: a void at an IR node degrades
# the incident tree segment with the larger |j| at nucleation, lower id on ties)
# ---------------------------------------------------------------------------

def _chain_trees(cells=4):
    # straight chain 0-1-2-3-4, segments 0:(0,1) 1:(1,2) 2:(2,3) 3:(3,4);
    # canonical order from root IR node 0: IR node k sits at local k*cells
    g = es.tree_grid("chain", cells=cells)
    return g, F.build_trees(g)


def test_void_segment_larger_current_wins():
    g, tr = _chain_trees(cells=4)
    st = F.StressState(tr, P)
    j = np.array([3.0, -5.0, 1.0, 1.0])
    # IR node 1 (local 4) touches segments 0 and 1: |j1| = 5 > |j0| = 3
    # IR node 3 (local 12) touches segments 2 and 3: equal |j| -> lower id 2
    # local 9 is interior to segment 2; local 16 is the far leaf (segment 3)
    F.assign_void_segments(tr, st, j, [4, 12, 9, 16])
    assert st.vseg[4] == 1
    assert st.vseg[12] == 2
    assert st.vseg[9] == 2
    assert st.vseg[16] == 3
    j2 = np.array([-7.0, 2.0, -1.0, 0.5])
    F.assign_void_segments(tr, st, j2, [4, 12])
    assert st.vseg[4] == 0 and st.vseg[12] == 2


def test_void_segment_tie_goes_to_lower_id():
    g, tr = _chain_trees(cells=4)
    st = F.StressState(tr, P)
    F.assign_void_segments(tr, st, np.array([4.0, -4.0, 4.0, 4.0]), [4, 8])
    assert st.vseg[4] == 0 and st.vseg[8] == 1


# ---------------------------------------------------------------------------
# Monte Carlo factor mapping (Sec. IV-F): kappa factor of a face = its
# segment's; sigma_crit factor of a node = its segment's, a crossing node the
# lowest-id incident segment of the same tree
# ---------------------------------------------------------------------------

def test_mc_factor_mapping_by_hand():
    g = es.tiny_grid()                       # 8 x 8, 40 cells per 20 um segment
    ns = g["seg_a"].size                     # 56 horizontal (row-major) + 56 vertical
    kf = 1.0 + 0.01 * np.arange(ns)
    sf = 2.0 + 0.001 * np.arange(ns)
    tr = F.build_trees(g)
    T = 378.0
    phys0 = F.tree_physics(tr, P, np.full(tr["n_nodes"], T))
    phys = F.tree_physics(tr, P, np.full(tr["n_nodes"], T), kf, sf)
    a = 0.5e-6 * 0.2e-6
    kap = P["D0"] * math.exp(-P["Ea"] / (P["k_B"] * T)) * P["B_modulus"] * P["Omega"] / (P["k_B"] * T)
    # tree 0 = horizontal stripe 0 (segments 0..6), root IR node 0.
    # local 40 = IR node 1: face to its parent lies on segment 0; the node
    # touches tree segments {0, 1} -> sigma_crit factor of segment 0.
    # local 41: first interior node of segment 1.
    o = tr["off"][0]
    assert tr["ir"][o + 40] == 1 and tr["ir"][o + 41] == -1
    assert abs(phys["kap_a"][o + 40] - a * kap * kf[0]) <= 1e-14 * a * kap
    assert abs(phys["kap_a"][o + 41] - a * kap * kf[1]) <= 1e-14 * a * kap
    assert phys["sig_crit"][o + 40] == P["sigma_crit"] * sf[0]
    assert phys["sig_crit"][o + 41] == P["sigma_crit"] * sf[1]
    assert phys["sig_crit"][o] == P["sigma_crit"] * sf[0]             # root IR node 0: segment 0
    # tree 8 = vertical stripe 0 (segments 56..62), nodes 0, 8, 16, ..., 56.
    # local 40 = IR node 8; it also touches horizontal segment 7 (row 1), which
    # belongs to another tree: the factor is segment 56's, not 7's.
    o8 = tr["off"][8]
    assert tr["layer"][8] == 1 and tr["ir"][o8 + 40] == 8
    assert phys["sig_crit"][o8 + 40] == P["sigma_crit"] * sf[56]
    assert phys["sig_crit"][o8 + 80] == P["sigma_crit"] * sf[56 + 1]  # IR node 16: {57, 58} -> 57
    assert abs(phys["kap_a"][o8 + 80] - a * kap * kf[57]) <= 1e-14 * a * kap
    # the leak sums the faces at a node: both incident faces of IR node 1
    assert abs(phys["leak"][o + 40] - a * kap * (kf[0] + kf[1]) / P["delta"]) <= 1e-13 * phys["leak"][o + 40]
    # unperturbed reference is the plain Arrhenius value
    assert abs(phys0["kap_a"][o + 41] - a * kap) <= 1e-14 * a * kap


# ---------------------------------------------------------------------------
# Aging-loop cadence (Sec. IV-A; TTF per Sec. V): scripted drops and
# resistances, so that only the loop's own bookkeeping is under test
# ---------------------------------------------------------------------------

class _Script:
    """Scripted IR solves: the k-th solve returns voltages whose max drop is
    drops[k] and whose currents are the constant j_k = k + 1 on every
    segment; void_resistance returns R0 + bumps[step]."""

    def __init__(self, g, drops, bumps):
        self.g, self.drops, self.bumps = g, list(drops), list(bumps)
        self.solves = 0
        self.step = 0
        self.seen_j = []

    def ir_solve(self, grid, R):
        d = self.drops[self.solves]
        u = np.full(len(grid["node_x"]), 1.0)
        u[-1] = 1.0 - d
        self.solves += 1
        return u

    def current_density(self, grid, u, R):
        return np.full(len(grid["seg_a"]), float(self.solves))

    def void_resistance(self, grid, p, st, tr=None):
        R = np.array(grid["seg_R0"], float) + self.bumps[self.step]
        self.step += 1
        return R

    def stepper(self, tr, p, phys, f, st, t0, dt, n, margin=None):
        k = int(round(t0 / (p["horizon"] / p["n_outer"])))
        if k == 0:                          # one void at IR node 1 of tree 0 in step 0
            st.void[tr["off"][0] + 40] = 1
        if margin is not None:
            margin[:] = 1.0
        return 0

    def assign(self, tr, st, j, new):
        self.seen_j.append((self.step, float(j[0]), list(new)))


def _scripted(monkeypatch, drops, bumps, n_outer):
    g = es.tiny_grid()
    s = _Script(g, drops, bumps)
    monkeypatch.setattr(F, "ir_solve", s.ir_solve)
    monkeypatch.setattr(F, "current_density", s.current_density)
    monkeypatch.setattr(F, "void_resistance", s.void_resistance)
    monkeypatch.setattr(F, "assign_void_segments", s.assign)
    p = dict(P, n_outer=n_outer)
    r = F.run_ttf(g, p, stepper=s.stepper)
    return r, s, p["horizon"] / n_outer


def test_cadence_resolve_only_on_change_and_first_crossing(monkeypatch):
    # R changes after steps 0, 2, 3, 4 (not 1): solves at t = 0 and after
    # those four steps; drops are read after the write-back of each step
    drops = [0.08, 0.09, 0.12, 0.09, 0.13]
    bumps = [1.0, 1.0, 2.0, 3.0, 4.0]
    r, s, dto = _scripted(monkeypatch, drops, bumps, n_outer=5)
    assert s.solves == 5
    assert np.allclose(r["drops"], [0.08, 0.09, 0.09, 0.12, 0.09, 0.13], rtol=0, atol=1e-15)
    # first crossing between the ends of steps 1 and 2 (t = 2 dto and 3 dto)
    assert r["ttf"] == pytest.approx(2 * dto + (0.10 - 0.09) / (0.12 - 0.09) * dto, rel=1e-12)
    # the void found in step 0 is assigned with the currents in force during
    # that step (the t = 0 solve, j = 1), before the end-of-step re-solve
    assert s.seen_j[0] == (0, 1.0, [40])


def test_cadence_initial_drop_above_threshold_is_zero(monkeypatch):
    r, s, _ = _scripted(monkeypatch, [0.11, 0.05, 0.2], [1.0, 2.0], n_outer=2)
    assert r["ttf"] == 0.0
    assert np.allclose(r["drops"], [0.11, 0.05, 0.2], rtol=0, atol=1e-15)


def test_cadence_never_crossed_is_censored(monkeypatch):
    r, s, _ = _scripted(monkeypatch, [0.01, 0.02, 0.03, 0.04], [1.0, 2.0, 3.0], n_outer=3)
    assert math.isinf(r["ttf"]) and r["ttf"] > 0
    assert r["final_drop"] == pytest.approx(0.04, abs=1e-15)


def test_cadence_no_resistance_change_no_resolve(monkeypatch):
    r, s, _ = _scripted(monkeypatch, [0.05], [0.0, 0.0, 0.0, 0.0], n_outer=4)
    assert s.solves == 1
    assert np.allclose(r["drops"], [0.05] * 5, rtol=0, atol=1e-15)


# ---------------------------------------------------------------------------
# Adam beyond the first step: closed forms of the bias-corrected moments
# after one non-zero gradient followed by zero gradients (geometric sums)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("b1,b2", [(0.9, 0.999), (0.5, 0.8)])
def test_adam_steps_two_and_three_closed_form(b1, b2):
    g1, lr, eps = 0.37, 1e-2, 1e-8
    W = np.zeros((1, 1)); b = np.zeros(1)
    opt = mlp.Adam([(W, b)], lr=lr, b1=b1, b2=b2, eps=eps)
    p1 = opt.step([(W, b)], [(np.full((1, 1), g1), np.full(1, -g1))])
    zero = [(np.zeros((1, 1)), np.zeros(1))]
    p2 = opt.step(p1, zero)
    p3 = opt.step(p2, zero)
    for t, (prev, cur) in ((2, (p1, p2)), (3, (p2, p3))):
        # m_t = b1^(t-1) (1 - b1) g1, v_t = b2^(t-1) (1 - b2) g1^2; corrections 1 - b^t
        mhat = b1 ** (t - 1) * (1 - b1) * g1 / (1 - b1 ** t)
        vhat = b2 ** (t - 1) * (1 - b2) * g1 * g1 / (1 - b2 ** t)
        step = lr * mhat / (math.sqrt(vhat) + eps)
        assert cur[0][0][0, 0] - prev[0][0][0, 0] == pytest.approx(-step, rel=1e-12)
        assert cur[0][1][0] - prev[0][1][0] == pytest.approx(step, rel=1e-12)
    # step 2 with b1 = 0.9, b2 = 0.999: m_hat = 0.9/1.9 g1, v_hat = 0.999/1.999 g1^2
    if b1 == 0.9:
        lit = lr * (0.9 / 1.9) / math.sqrt(0.999 / 1.999)
        assert p2[0][0][0, 0] - p1[0][0][0, 0] == pytest.approx(-lit, rel=1e-7)
