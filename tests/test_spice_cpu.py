"""The SPICE netlist reader (ems_spice_parse, host code of libems.so): a
synthetic junction-heavy netlist parses into exactly the grid its generator
describes, and malformed lines are rejected with the line number."""
import numpy as np
import pytest

import ems_synth as es


@pytest.fixture(scope="module")
def sp():
    from paper_2604_10743_gb300 import build as B
    B.build()
    from paper_2604_10743_gb300 import spice
    return spice


def test_parse_matches_generator(sp):
    text, g = es.spice_netlist()
    p = sp.parse_spice(text, W=[0.5e-6, 0.8e-6], H=[0.2e-6, 0.3e-6])
    for k in ("node_x", "node_y", "seg_a", "seg_b", "seg_layer", "seg_cells", "seg_R0", "seg_W", "seg_H",
              "seg_L", "seg_via", "pad_node", "pad_V", "sink_node", "sink_I"):
        assert p[k].shape == np.asarray(g[k]).shape, k
        assert np.array_equal(p[k], np.asarray(g[k]).astype(p[k].dtype)), k
    # junction-heavy: many layer-1 nodes have three or more segments
    deg = np.bincount(np.concatenate([g["seg_a"], g["seg_b"]]), minlength=len(g["node_x"]))
    assert np.sum(deg >= 3) >= 8
    from oracle import flow as F
    tr = F.build_trees(g)
    assert tr["n_trees"] == 8                     # 4 trees on layer 1, 4 straps on layer 2


@pytest.mark.parametrize("bad,why", [
    ("R1 n1_0_0 0 1.0\nV1 n1_0_0 0 1\n", "resistor to ground"),
    ("R1 n1_0_0 n1_10_0 1.0\nV1 n1_0_0 n1_10_0 1\n", "source must join"),
    ("R1 foo n1_10_0 1.0\nV1 n1_10_0 0 1\n", "node name"),
    ("R1 n1_0_0 n1_10_0 abc\nV1 n1_0_0 0 1\n", "bad value"),
    ("C1 n1_0_0 n1_10_0 1e-12\nV1 n1_0_0 0 1\n", "unsupported"),
    ("R1 n1_0_0 n1_10_0 1.0\n", "voltage source"),
    ("R1 n3_0_0 n3_10_0 1.0\nV1 n3_0_0 0 1\n", "node name"),
])
def test_rejects_malformed(sp, bad, why):
    from paper_2604_10743_gb300 import EmsError
    with pytest.raises(EmsError) as e:
        sp.parse_spice(bad, W=[0.5e-6, 0.8e-6], H=[0.2e-6, 0.3e-6])
    assert why in str(e.value)
