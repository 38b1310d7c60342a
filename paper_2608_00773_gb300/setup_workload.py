"""Convenience: build the tables and grid handles from a workload description
(any object with the attributes of workloads.Workload)."""
from __future__ import annotations

from .binding import Grid, Tables


def setup(wl):
    """(tables, grid) for a workload: nao_tabulate then grid_partition."""
    t = Tables(wl.n_rad_per_species, wl.rad_l, wl.rad_alpha, wl.r_c, wl.r_on, wl.r_min, wl.n_log)
    g = Grid(t, wl.xyz, wl.species_of_atom, wl.n_rad, wl.R, wl.n_theta, wl.n_phi, wl.r_nb, wl.batch_max,
             getattr(wl, "lattice", None), getattr(wl, "n_shell", 0), getattr(wl, "mol_atom_ptr", None),
             getattr(wl, "partition", "becke"))
    return t, g
