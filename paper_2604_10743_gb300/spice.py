"""Python face of the SPICE netlist reader of include/ems.h (marshalling only).

parse_spice(text, W, H, ...) runs ems_spice_parse in libems.so and returns
the grid as a dict of NumPy arrays (copied out of the library's netlist), in
the form Engine takes.
"""
import ctypes

import numpy as np

from . import _abi as A


def parse_spice(text, W, H, via_W=0.2e-6, via_H=0.2e-6, coord_unit=1e-9, dx=0.5e-6):
    """Parse a SPICE power-grid netlist; W, H: per-layer wire width and
    thickness (layers 1..len(W)).  Raises EmsError on a malformed netlist."""
    L = A.lib()
    raw = text.encode() if isinstance(text, str) else bytes(text)
    Wa = np.ascontiguousarray(W, np.float64); Ha = np.ascontiguousarray(H, np.float64)
    o = A.EmsSpiceOpts(int(Wa.size), Wa.ctypes.data_as(A.c_double_p), Ha.ctypes.data_as(A.c_double_p),
                       float(via_W), float(via_H), float(coord_unit), float(dx))
    nl = ctypes.c_void_p()
    st = L.ems_spice_parse(raw, len(raw), ctypes.byref(o), ctypes.byref(nl))
    try:
        if st != A.EMS_OK:
            msg = L.ems_netlist_error(nl) if nl.value else b"bad arguments"
            raise A.EmsError(st, msg.decode())
        d = A.EmsGridDesc()
        st = L.ems_netlist_desc(nl, ctypes.byref(d))
        if st != A.EMS_OK:
            raise A.EmsError(st, "ems_netlist_desc")

        def arr(ptr, n, dt):
            return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dt, copy=True) if n else np.zeros(0, dt)
        g = dict(
            node_x=arr(d.node_x, d.n_nodes, np.float64), node_y=arr(d.node_y, d.n_nodes, np.float64),
            seg_a=arr(d.seg_a, d.n_seg, np.int32), seg_b=arr(d.seg_b, d.n_seg, np.int32),
            seg_layer=arr(d.seg_layer, d.n_seg, np.int32), seg_cells=arr(d.seg_cells, d.n_seg, np.int32),
            seg_R0=arr(d.seg_R0, d.n_seg, np.float64), seg_W=arr(d.seg_W, d.n_seg, np.float64),
            seg_H=arr(d.seg_H, d.n_seg, np.float64), seg_L=arr(d.seg_L, d.n_seg, np.float64),
            seg_via=arr(d.seg_via, d.n_seg, np.int8),
            pad_node=arr(d.pad_node, d.n_pads, np.int32), pad_V=arr(d.pad_V, d.n_pads, np.float64),
            sink_node=arr(d.sink_node, d.n_sinks, np.int32), sink_I=arr(d.sink_I, d.n_sinks, np.float64),
            thermal=None, kappa_factor=None, sigc_factor=None)
    finally:
        if nl.value:
            L.ems_netlist_free(nl)
    return g
