"""Pins of the oracle's via-aware failure (Sec. IV-C): via resistors join
layers but belong to no stress tree; a void at a node with a via up to a
strictly higher layer opens that via (open-circuit sentinel) once it passes
the critical volume, while late failure alone applies elsewhere."""
import numpy as np

import ems_synth as es
from oracle import flow as F

P = es.default_params()


def test_via_mesh_trees_and_up_vias():
    g = es.via_mesh(N=4)
    tr = F.build_trees(g)
    # 4 lower horizontal + 4 upper vertical stripes; vias in no tree
    assert tr["n_trees"] == 8
    assert all(not g["seg_via"][s] for segs in tr["tree_segs"] for s in segs)
    up = F.up_vias(g)
    # every lower crossing i*4 + j has its via (segment 24 + i*4 + j) up; upper nodes have none
    ns = 2 * 4 * 3
    assert np.array_equal(up[:16], ns + np.arange(16))
    assert np.all(up[16:] == -1)
    # the merged mesh has no via information: no node has an up via
    assert np.all(F.up_vias(es.tiny_grid()) == -1)


def _state_with_void(tr, node, vol):
    st = F.StressState(tr, P)
    st.void[node] = 1
    st.vol[node] = vol
    return st


def test_early_failure_opens_the_via_past_the_critical_volume():
    g = es.via_mesh(N=4, cells=10)
    tr = F.build_trees(g)
    # tree 0: lower stripe 0; its IR node 1 (crossing (0, 1)) sits at local 10
    o = tr["off"][0]
    v = o + 10
    assert tr["ir"][v] == 1
    seg = 0                                        # the larger-|j| choice is not under test here
    W, H = g["seg_W"][seg], g["seg_H"][seg]
    Vc = W * W * H
    via = F.up_vias(g)[1]
    for vol, opened in ((0.5 * Vc, False), (2.0 * Vc, True)):
        st = _state_with_void(tr, v, vol)
        st.vseg[v] = seg
        R = F.void_resistance(g, P, st, tr)
        assert (R[via] == F.R_OPEN) == opened
        # the wire segment still takes its late-failure increment
        coef = P["rho_Ta"] / (P["h_Ta"] * (2 * H + W)) - P["rho_Cu"] / (H * W)
        assert R[seg] == g["seg_R0"][seg] + max(0.0, (vol - Vc) / (W * H) * coef)
        others = np.ones(R.size, bool); others[[via, seg]] = False
        assert np.array_equal(R[others], g["seg_R0"][others])
    # a void inside a segment, or at a node without an up via, opens nothing
    st = _state_with_void(tr, o + 5, 3.0 * Vc); st.vseg[o + 5] = 0
    assert np.sum(F.void_resistance(g, P, st, tr) == F.R_OPEN) == 0
    o4 = tr["off"][4]                              # first upper stripe: upper nodes have no up via
    st = _state_with_void(tr, o4 + 10, 3.0 * Vc); st.vseg[o4 + 10] = tr["face_seg"][o4 + 10]
    assert np.sum(F.void_resistance(g, P, st, tr) == F.R_OPEN) == 0
