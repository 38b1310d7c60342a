"""GPU parity of the small-component integrals: tables built from the values
of the Q(r) radials at the knots (nao_tabulate_knots; phi^S = Q/r Y_(l~ m~),
Eq. 12b, with the synthetic atomic-ZORA Q of Eq. 8b) and the SS block of
Eq. 19 in the scalar form, F^S_ij = sum_p w phi^S_i (eps_j - V_j + v) phi^S_j
(the i of phi^S cancels against its conjugate), against the oracle within
1e-12 relative Frobenius on a molecule, a cluster and a periodic cell; the
split path on the same tables within 1e-9 of FP64; knot-value tables of the
large-component radials against the (l, alpha) tables; and l~ = 4 (from f
shells) refused."""
import dataclasses

import numpy as np
import pytest

import oracle as O
import paper_2608_00773_gb300 as q
from gpu_helpers import LibCase, OracleCase, rel_fro
from workloads import Species, column_operator, periodic_cell, small_cluster, small_component, water

pytestmark = pytest.mark.gpu


def up_to_d(wl):
    """The workload with its f shells dropped (their small components need l~ = 4)."""
    sp = [Species(s.name, s.Z, [l for l in s.l if l <= 2], [a for l, a in zip(s.l, s.alpha) if l <= 2])
          for s in wl.species]
    return dataclasses.replace(wl, species=sp)


@pytest.fixture(scope="module", params=["water", "cluster", "cell"])
def case(request):
    from paper_2608_00773_gb300 import _build
    _build.build()
    O.build()
    wl = {"water": water, "cluster": lambda: up_to_d(small_cluster(8, seed=7)),
          "cell": lambda: up_to_d(periodic_cell())}[request.param]()
    eps, Vk = column_operator(wl, 41)
    ws, Q, parent, _ = small_component(wl, Vk)
    return LibCase(ws, Q), OracleCase(ws, Q), eps[parent], Vk[parent]


def test_small_integrals_match_oracle(case):
    lib, orc, _, _ = case
    got = lib.integrate("fp64")
    lib.grid.status()
    for g, r in zip(got[:5], orc.mats):
        assert rel_fro(g, r) <= 1e-12


def test_small_columns_match_oracle(case):
    lib, orc, eps, Vk = case
    q.q4c_tables_set_columns(lib.tables, eps, Vk)
    F = q.q4c_integrate_columns(lib.tables, lib.grid, lib.v).cpu().numpy()
    lib.grid.status()
    ref = orc.ob.matrix_columns(orc.xyz, orc.w, orc.v, eps, Vk, orc.pat)
    assert rel_fro(F, ref) <= 1e-12


def test_small_split_matches_fp64(case):
    lib, _, _, _ = case
    ref = lib.integrate("fp64")
    got = lib.integrate("split")
    for g, r in zip(got[:5], ref[:5]):
        assert rel_fro(g, r) <= 1e-9


def test_knot_tables_match_analytic_tables():
    from paper_2608_00773_gb300 import _build
    _build.build()
    wl = water()
    ob = O.OracleBasis(wl)
    ta = q.Tables(wl.n_rad_per_species, wl.rad_l, wl.rad_alpha, wl.r_c, wl.r_on, wl.r_min, wl.n_log)
    tk = q.nao_tabulate_knots(wl.n_rad_per_species, wl.rad_l, ob.tab_u, wl.r_c, wl.r_on, wl.r_min, wl.n_log)
    for k in range(len(wl.rad_l)):
        a, b = ta.coefficients(k), tk.coefficients(k)
        assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()


def test_l_tilde_4_is_refused():
    from paper_2608_00773_gb300 import _build
    _build.build()
    wl = small_cluster(8, seed=7)
    _, Vk = column_operator(wl, 3)
    ws, Q, _, _ = small_component(wl, Vk)
    assert ws.rad_l.max() == 4
    with pytest.raises(q.Q4CError):
        q.nao_tabulate_knots(ws.n_rad_per_species, ws.rad_l, Q, ws.r_c, ws.r_on, ws.r_min, ws.n_log)
