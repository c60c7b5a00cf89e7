"""Oracle for the Joule-heating temperature profile along every branch (Sec. III-A).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Stationary thermal equation of a wire with Joule heating j^2 rho and heat
loss to the surroundings k (T - T0) / Gamma^2, Gamma^2 = t_cu t_ILD k_cu / k_ILD
(Eq. stationary_thermal_equation and the thermal characteristic length):

    k T'' + j^2 rho - k (T - T0) / Gamma^2 = 0.

Reading (the printed solution is garbled: it uses cos / sin, which solve the
equation with the opposite sign of the loss term, and it returns T0 at the
right end whatever T2 is): the solution on x in [-L/2, L/2] with T(-L/2) = T1
and T(L/2) = T2 is

    T(x) = T0 + Tm + (Tbar - T0 - Tm) cosh(x/G) / cosh(L/(2G))
                   - Tn sinh(x/G) / sinh(L/(2G)),

Tm = j^2 rho G^2 / k_cu (the symmetric Joule rise, as printed), Tbar =
(T1 + T2)/2 and Tn = (T1 - T2)/2 (the antisymmetric part, as printed).

Branch endpoints (per the paper: via-node temperatures from the map,
unconstrained endpoints from tridiagonal thermal blocks, T0 without a map):
an IR node touched by segments of more than one metal layer (a via in the
two-layer mesh) or a pad is constrained, its temperature the map's value at
the node (T0 without a map).  Every other IR node is unconstrained: the heat
flows into its incident segments sum to zero, which with the closed form
gives one linear equation per node (symmetric, diagonally dominant; a
tridiagonal system along a chain), solved here with a direct sparse solver.
An unconstrained leaf has zero heat flow.  The profile uses the current
density of each segment as given.
"""
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import flow as F


def gamma(H, k_cu, k_ild, t_ild):
    """Thermal characteristic length, Gamma^2 = t_cu t_ILD k_cu / k_ILD."""
    return np.sqrt(np.asarray(H, np.float64) * t_ild * k_cu / k_ild)


def wire_profile(x, L, G, T0, Tm, T1, T2):
    """Closed-form temperature at positions x in [-L/2, L/2] of one wire."""
    h = L / (2.0 * G)
    Tbar, Tn = 0.5 * (T1 + T2), 0.5 * (T1 - T2)
    return (T0 + Tm + (Tbar - T0 - Tm) * np.cosh(x / G) / math.cosh(h)
            - Tn * np.sinh(x / G) / math.sinh(h))


def end_heat_flow(L, G, A, k_cu, T0, Tm, Ta, Tb):
    """Heat flowing from the wire's a end (x = -L/2) into the wire:
    -k_cu A T'(-L/2) for the closed form above."""
    h = L / (2.0 * G)
    Tbar, Tn = 0.5 * (Ta + Tb), 0.5 * (Ta - Tb)
    dT = -(Tbar - T0 - Tm) * math.tanh(h) / G - Tn / (G * math.tanh(h))
    return -k_cu * A * dT


def node_temperatures(grid, p, j_seg, k_cu, k_ild, t_ild, thermal=None):
    """Temperature of every IR node: constrained nodes (multi-layer or pad)
    from the map or T0, the rest from the zero-net-heat-flow equations."""
    a = np.asarray(grid["seg_a"]); b = np.asarray(grid["seg_b"])
    layer = np.asarray(grid["seg_layer"])
    n = len(grid["node_x"])
    T0 = float(p["T0"])
    L = np.asarray(grid["seg_L"], np.float64)
    A = np.asarray(grid["seg_W"]) * np.asarray(grid["seg_H"])
    G = gamma(grid["seg_H"], k_cu, k_ild, t_ild)
    Tm = np.asarray(j_seg, np.float64) ** 2 * p["rho_Cu"] * G * G / k_cu
    layers = [set() for _ in range(n)]
    for s in range(a.size):
        layers[a[s]].add(int(layer[s])); layers[b[s]].add(int(layer[s]))
    fixed = np.array([len(ls) > 1 for ls in layers])
    fixed[np.asarray(grid["pad_node"])] = True
    T = np.full(n, T0)
    if thermal is not None:
        T[fixed] = F.bilinear(thermal, np.asarray(grid["node_x"])[fixed], np.asarray(grid["node_y"])[fixed])
    free = np.nonzero(~fixed)[0]
    if free.size:
        idx = -np.ones(n, np.int64); idx[free] = np.arange(free.size)
        rows, cols, vals = [], [], []
        rhs = np.zeros(free.size)
        for s in range(a.size):
            h = L[s] / (2.0 * G[s])
            w = k_cu * A[s] / G[s]
            cth, csh, th = 1.0 / math.tanh(2 * h), 1.0 / math.sinh(2 * h), math.tanh(h)
            # heat flow into segment s at end u: w [T_u coth 2h - T_v csch 2h - (T0 + Tm) tanh h]
            for u, v in ((a[s], b[s]), (b[s], a[s])):
                if idx[u] < 0:
                    continue
                rows.append(idx[u]); cols.append(idx[u]); vals.append(w * cth)
                if idx[v] >= 0:
                    rows.append(idx[u]); cols.append(idx[v]); vals.append(-w * csh)
                else:
                    rhs[idx[u]] += w * csh * T[v]
                rhs[idx[u]] += w * (T0 + Tm[s]) * th
        Mx = sp.csc_matrix((vals, (rows, cols)), shape=(free.size, free.size))
        T[free] = spla.spsolve(Mx, rhs)
    return T, Tm, G


def stress_node_temperature(tr, grid, p, j_seg, k_cu, k_ild, t_ild, thermal=None):
    """Per stress node (canonical order): an IR node's temperature, or the
    closed-form profile of its segment at its position along the segment."""
    Tir, Tm, G = node_temperatures(grid, p, j_seg, k_cu, k_ild, t_ild, thermal)
    a = np.asarray(grid["seg_a"]); b = np.asarray(grid["seg_b"])
    xn = np.asarray(grid["node_x"]); yn = np.asarray(grid["node_y"])
    L = np.asarray(grid["seg_L"], np.float64)
    out = np.empty(tr["n_nodes"])
    for i in range(tr["n_nodes"]):
        irn = tr["ir"][i]
        if irn >= 0:
            out[i] = Tir[irn]
            continue
        s = tr["face_seg"][i]
        # fraction along a -> b from the coordinates, then centred on the segment
        frac = math.hypot(tr["x"][i] - xn[a[s]], tr["y"][i] - yn[a[s]]) / \
            math.hypot(xn[b[s]] - xn[a[s]], yn[b[s]] - yn[a[s]])
        x = (frac - 0.5) * L[s]
        out[i] = wire_profile(x, L[s], G[s], float(p["T0"]), Tm[s], Tir[a[s]], Tir[b[s]])
    return out
