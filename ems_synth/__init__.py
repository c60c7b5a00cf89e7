"""Seeded synthetic inputs (netlists, thermal maps, MC factors, parameters).

Shared by the CPU oracle and the CUDA library's tests and benchmark; holds no
part of the EM/TM method's arithmetic.
"""
from .params import default_params, EV, YEAR
from .grid import (stripe_mesh, via_mesh, spice_netlist, tiny_grid, mid_grid, mc_grid, large_grid, tree_grid,
                   hotspot_raster, mc_factors, config)

__all__ = ["default_params", "EV", "YEAR", "stripe_mesh", "via_mesh", "spice_netlist", "tiny_grid", "mid_grid",
           "mc_grid", "large_grid", "tree_grid", "hotspot_raster", "mc_factors", "config"]
