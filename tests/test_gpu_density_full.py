"""GPU parity of the density with gradient terms (q4c_density_full):
n_p = sum_M sum_ij P^M_ij f^M_ij(p) over the V, W0 and SO slots, against the
oracle on a molecule, a cluster and a periodic cell; with only the V slot it
equals q4c_density."""
import numpy as np
import pytest

import oracle as O
import paper_2608_00773_gb300 as q
from gpu_helpers import LibCase, OracleCase, point_map, rel_fro
from workloads import periodic_cell, small_cluster, water

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-12, "split": 1e-9}


@pytest.fixture(scope="module")
def cases():
    from paper_2608_00773_gb300 import _build
    _build.build()
    O.build()
    return {name: (LibCase(wl), OracleCase(wl))
            for name, wl in (("water", water()), ("cluster", small_cluster(8, seed=7)), ("cell", periodic_cell()))}


@pytest.mark.parametrize("prec", ["fp64", "split"])
@pytest.mark.parametrize("name", ["water", "cluster", "cell"])
def test_density_full_matches_oracle(name, prec, cases):
    lib, orc = cases[name]
    n = q.q4c_density_full(lib.tables, lib.grid, lib.G(81), prec).cpu().numpy()
    lib.grid.status()
    nref = orc.ob.density_full(orc.xyz, orc.G(81), orc.pat)
    li, oi = point_map(lib.ex["point_id"], orc.ids)
    assert rel_fro(n[li], nref[oi]) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_v_slot_only_is_the_density(prec, cases):
    lib, _ = cases["cluster"]
    P = lib.random(82, "P")
    a = q.q4c_density(lib.tables, lib.grid, P, prec).cpu().numpy()
    b = q.q4c_density_full(lib.tables, lib.grid, [P, None, None, None, None], prec).cpu().numpy()
    assert rel_fro(b, a) <= TOL[prec]
