"""GPU parity of the small-component integrals: tables built from the values
of the Q(r) radials at the knots (nao_tabulate_knots; phi^S = Q/r Y_(l~ m~),
Eq. 12b, with the synthetic atomic-ZORA Q of Eq. 8b) and the SS block of
Eq. 19 in the scalar form, F^S_ij = sum_p w phi^S_i (eps_j - V_j + v) phi^S_j
(the i of phi^S cancels against its conjugate), against the oracle within
1e-12 relative Frobenius on a molecule, a cluster and a periodic cell; the
split path on the same tables within 1e-9 of FP64; knot-value tables of the
large-component radials against the (l, alpha) tables; l = 4 (g shells, and
the l~ = 4 small components of f shells) on both paths; l = 5 refused."""
import numpy as np
import pytest

import oracle as O
import paper_2608_00773_gb300 as q
from gpu_helpers import LibCase, OracleCase, rel_fro
from workloads import column_operator, periodic_cell, single_atom, small_cluster, small_component, water

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["water", "cluster", "cell"])
def case(request):
    from paper_2608_00773_gb300 import _build
    _build.build()
    O.build()
    # the cluster's f shells give small components with l~ = 4
    wl = {"water": water, "cluster": lambda: small_cluster(8, seed=7), "cell": periodic_cell}[request.param]()
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
    lib, _, eps, Vk = case
    ref = lib.integrate("fp64")
    got = lib.integrate("split")
    for g, r in zip(got[:5], ref[:5]):
        assert rel_fro(g, r) <= 1e-9
    q.q4c_tables_set_columns(lib.tables, eps, Vk)
    Fs = q.q4c_integrate_columns(lib.tables, lib.grid, lib.v, "split").cpu().numpy()
    F64 = q.q4c_integrate_columns(lib.tables, lib.grid, lib.v, "fp64").cpu().numpy()
    lib.grid.status()
    assert rel_fro(Fs, F64) <= 1e-9


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


def test_small_component_of_the_64_atom_cluster():
    """The bench's workload in the small-component basis (f shells give l~ = 4;
    ~2x the large component's functions per batch): split within 1e-9 of FP64
    for V, W0, SO and the per-column operator, and the spinor functions line up
    with the large component's."""
    from paper_2608_00773_gb300 import _build
    from workloads import cluster64
    _build.build()
    wl = cluster64()
    eps, Vk = column_operator(wl, 61)
    ws, Q, parent, kappa = small_component(wl, Vk)
    lib = LibCase(ws, Q)
    assert lib.grid.info.max_nb > 175
    ref = lib.integrate("fp64")
    got = lib.integrate("split")
    lib.grid.status()
    for g, r in zip(got[:5], ref[:5]):
        assert rel_fro(g, r) <= 1e-9
    q.q4c_tables_set_columns(lib.tables, eps[parent], Vk[parent])
    Fs = q.q4c_integrate_columns(lib.tables, lib.grid, lib.v, "split").cpu().numpy()
    F64 = q.q4c_integrate_columns(lib.tables, lib.grid, lib.v, "fp64").cpu().numpy()
    lib.grid.status()
    assert rel_fro(Fs, F64) <= 1e-9
    q.q4c_tables_set_kappa(lib.tables, -kappa)
    for s, sp in enumerate(wl.species):
        assert len(q.q4c_spinor_basis(lib.tables, s)[0]) == 2 * sp.n_fn


def test_g_shells_of_the_large_component():
    """l = 4 as a large-component radial (the basis evaluation has no
    small-component special case): FP64 against the oracle, split against FP64."""
    from paper_2608_00773_gb300 import _build
    _build.build()
    O.build()
    wl = single_atom([0, 2, 4, 4], [1.3, 0.9, 2.1, 0.6], Z=6.0, n_rad=40)
    lib, orc = LibCase(wl), OracleCase(wl)
    got = lib.integrate("fp64")
    for g, r in zip(got[:5], orc.mats):
        assert rel_fro(g, r) <= 1e-12
    for g, r in zip(lib.integrate("split")[:5], got[:5]):
        assert rel_fro(g, r) <= 1e-9


def test_l_5_is_refused():
    from paper_2608_00773_gb300 import _build
    _build.build()
    with pytest.raises(q.Q4CError):
        q.nao_tabulate([1], [5], [1.0])
