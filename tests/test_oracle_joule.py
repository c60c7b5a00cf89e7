"""Pins of the oracle's Joule-heating profile (Sec. III-A) against the
differential equation itself: the closed form solves the stationary thermal
equation with its end values, and the per-tree profile with solved
unconstrained nodes agrees with a brute-force finite-difference solution of
the same equation over the whole tree."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import ems_synth as es
from oracle import flow as F
from oracle import joule as J

P = es.default_params()
K_CU, K_ILD, T_ILD = 400.0, 1.4, 0.2e-6


def test_closed_form_solves_the_thermal_equation():
    L, G, T0, Tm, T1, T2 = 12e-6, 3.4e-6, 340.0, 6.5, 352.0, 331.0
    x = np.linspace(-L / 2, L / 2, 20001)
    T = J.wire_profile(x, L, G, T0, Tm, T1, T2)
    assert abs(T[0] - T1) < 1e-12 * T1 and abs(T[-1] - T2) < 1e-12 * T2
    h = x[1] - x[0]
    d2 = (T[2:] - 2 * T[1:-1] + T[:-2]) / (h * h)
    # k T'' + j^2 rho - k (T - T0) / G^2 = 0 with j^2 rho / k = Tm / G^2
    res = d2 + Tm / G ** 2 - (T[1:-1] - T0) / G ** 2
    assert np.abs(res).max() * G ** 2 < 1e-5 * Tm
    # the heat flow at the a end is -k A T'(-L/2)
    A = 0.1e-12
    q = J.end_heat_flow(L, G, A, K_CU, T0, Tm, T1, T2)
    dT = (-3 * T[0] + 4 * T[1] - T[2]) / (2 * h)
    assert abs(q - (-K_CU * A * dT)) < 1e-6 * abs(q)


def test_no_current_and_equal_ends_is_ambient_and_long_wire_plateau():
    x = np.linspace(-5e-6, 5e-6, 101)
    assert np.abs(J.wire_profile(x, 10e-6, 2e-6, 350.0, 0.0, 350.0, 350.0) - 350.0).max() < 1e-12
    # a wire 40 Gamma long: the middle sits at T0 + Tm (cosh(20) ~ 2.4e8)
    G = 1e-6
    Tmid = J.wire_profile(np.array([0.0]), 40 * G, G, 330.0, 9.0, 360.0, 350.0)[0]
    assert abs(Tmid - 339.0) < 1e-6


def _fd_tree(grid, p, j, cells=400):
    """Brute force: the whole single-layer tree discretised in `cells` cells
    per segment; k T'' - k (T - T0)/G^2 + j^2 rho = 0 on each wire, heat flow
    continuity at every IR node, the pad held at T0, zero flow at free leaves."""
    a = np.asarray(grid["seg_a"]); b = np.asarray(grid["seg_b"])
    n_ir = len(grid["node_x"])
    L = np.asarray(grid["seg_L"]); A = np.asarray(grid["seg_W"]) * np.asarray(grid["seg_H"])
    G = J.gamma(grid["seg_H"], K_CU, K_ILD, T_ILD)
    T0 = p["T0"]
    # unknowns: IR nodes, then interior points of each segment
    nint = cells - 1
    N = n_ir + a.size * nint
    rows, cols, vals = [], [], []
    rhs = np.zeros(N)

    def add(r, c, v):
        rows.append(r); cols.append(c); vals.append(v)
    for s in range(a.size):
        dx = L[s] / cells
        ids = [a[s]] + [n_ir + s * nint + k for k in range(nint)] + [b[s]]
        src = j[s] ** 2 * p["rho_Cu"] / K_CU
        # control volumes: interior points full dx, IR ends half dx (finite volume)
        for k in range(cells + 1):
            vol = dx if 0 < k < cells else dx / 2
            i = ids[k]
            w = A[s]
            add(i, i, w * vol / G[s] ** 2)
            rhs[i] += w * vol * (src + T0 / G[s] ** 2)
            for nb in (k - 1, k + 1):
                if 0 <= nb <= cells:
                    add(i, i, w / dx)
                    add(i, ids[nb], -w / dx)
    M = sp.csr_matrix((vals, (rows, cols)), shape=(N, N)).tolil()
    for pn in grid["pad_node"]:
        M.rows[pn] = [pn]; M.data[pn] = [1.0]; rhs[pn] = T0
    return spla.spsolve(M.tocsc(), rhs), n_ir, nint


@pytest.mark.parametrize("kind", ["chain", "T", "comb"])
def test_tree_profile_matches_finite_differences(kind):
    g = es.tree_grid(kind, cells=8, seed=2, seg_len=8e-6)
    p = dict(P, T0=345.0)
    rng = np.random.default_rng(1)
    j = rng.uniform(0.5e11, 1.5e11, size=g["seg_a"].size) * rng.choice([-1, 1], size=g["seg_a"].size)
    Tir, Tm, G = J.node_temperatures(g, p, j, K_CU, K_ILD, T_ILD)
    ref, n_ir, nint = _fd_tree(g, p, j)
    rise = (Tir - p["T0"]).max()
    assert rise > 1.0                                   # the test heats the tree visibly
    assert np.abs(Tir - ref[:n_ir]).max() < 2e-4 * rise
    tr = F.build_trees(g)
    Tn = J.stress_node_temperature(tr, g, p, j, K_CU, K_ILD, T_ILD)
    # the FD interior points at the stress nodes' positions (8 cells = every 50th point)
    for i in range(tr["n_nodes"]):
        if tr["ir"][i] >= 0:
            continue
        s = tr["face_seg"][i]
        fr = math.hypot(tr["x"][i] - g["node_x"][g["seg_a"][s]], tr["y"][i] - g["node_y"][g["seg_a"][s]]) / g["seg_L"][s]
        k = int(round(fr * 400))
        assert abs(Tn[i] - ref[n_ir + s * nint + k - 1]) < 2e-4 * rise
    # zero net heat flow at every unconstrained IR node
    A = np.asarray(g["seg_W"]) * np.asarray(g["seg_H"])
    flows = {}
    for s in range(g["seg_a"].size):
        for u, v in ((g["seg_a"][s], g["seg_b"][s]), (g["seg_b"][s], g["seg_a"][s])):
            flows.setdefault(int(u), []).append(
                J.end_heat_flow(g["seg_L"][s], G[s], A[s], K_CU, p["T0"], Tm[s], Tir[u], Tir[v]))
    scale = max(abs(q) for qs in flows.values() for q in qs)
    pads = set(g["pad_node"].tolist())
    for nd, qs in flows.items():
        if nd not in pads:
            assert abs(sum(qs)) <= 1e-9 * scale, nd


def test_mesh_nodes_take_the_map():
    """Two-layer mesh: every crossing is a via, so every IR node takes the
    map's value and the interior of each segment adds the Joule rise."""
    g = es.mid_grid(N=16, raster=32)
    u = F.ir_solve(g, g["seg_R0"])
    j = F.current_density(g, u, g["seg_R0"]) * 50.0       # strong enough for a visible rise
    Tir, Tm, G = J.node_temperatures(g, P, j, K_CU, K_ILD, T_ILD, g["thermal"])
    ref = F.bilinear(g["thermal"], g["node_x"], g["node_y"])
    assert np.array_equal(Tir, ref)
    tr = F.build_trees(g)
    Tn = J.stress_node_temperature(tr, g, P, j, K_CU, K_ILD, T_ILD, g["thermal"])
    assert Tn.max() > ref.max()
