"""Convenience: build the tables and grid handles from a workload description
(any object with the attributes of workloads.Workload)."""
from __future__ import annotations

from .binding import Grid, Tables


def setup(wl, knots=None):
    """(tables, grid) for a workload: nao_tabulate (nao_tabulate_knots when the
    radials are given by their knot values [sum n_rad][n_log]) then grid_partition."""
    t = Tables(wl.n_rad_per_species, wl.rad_l, None if knots is not None else wl.rad_alpha, wl.r_c, wl.r_on,
               wl.r_min, wl.n_log, knots=knots)
    g = Grid(t, wl.xyz, wl.species_of_atom, wl.n_rad, wl.R, wl.n_theta, wl.n_phi, wl.r_nb, wl.batch_max,
             getattr(wl, "lattice", None), getattr(wl, "n_shell", 0), getattr(wl, "mol_atom_ptr", None),
             getattr(wl, "partition", "becke"))
    return t, g
