"""GPU parity of the small-component spinor path (Eqs. 11, 14, 19, 21):
tables of the Q radials with kappa~ = -kappa per radial (q4c_tables_set_kappa)
give the spinor basis of the large component, bit-exact against the oracle;
their forward map of the per-column operator F^S is the SS block of Eq. 19,
and with the large component's block the whole H+ (and S+), within 1e-12 of
the oracle; the reverse map and the small-component density of Eq. 21 on
seeded spinor density matrices within 1e-12; on a molecule, a cluster with f
shells (l~ = 4) and a periodic cell."""
import numpy as np
import pytest

import oracle as O
import paper_2608_00773_gb300 as q
from gpu_helpers import LibCase, OracleCase, point_map, rel_fro
from oracle import spinor as S
from workloads import column_operator, periodic_cell, small_cluster, small_component, water

pytestmark = pytest.mark.gpu


class Case:
    def __init__(self, wl):
        self.wl = wl
        self.eps, self.Vk = column_operator(wl, 51)
        self.ws, self.Q, self.parent, kappa = small_component(wl, self.Vk)
        self.kS = -kappa
        self.libL, self.orcL = LibCase(wl), OracleCase(wl)
        self.libS, self.orcS = LibCase(self.ws, self.Q), OracleCase(self.ws, self.Q)
        q.q4c_tables_set_kappa(self.libS.tables, self.kS)
        self.GL = S.atom_matrices(wl)
        self.GS = S.atom_matrices(self.ws, kappas=self.kS)


@pytest.fixture(scope="module", params=["water", "cluster", "cell"])
def case(request):
    from paper_2608_00773_gb300 import _build
    _build.build()
    O.build()
    # the cluster's f shells carry small components with l~ = 4
    return Case({"water": water, "cluster": lambda: small_cluster(8, seed=7), "cell": periodic_cell}[request.param]())


def _flat(blocks, pat):
    """Spinor blocks laid out consecutively in pattern order."""
    return np.concatenate([b.reshape(-1) for b in blocks]) if blocks else np.zeros(0, complex)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_small_spinor_basis_lines_up_with_the_large_one(case):
    r0 = 0
    for s, (sl, ss) in enumerate(zip(case.wl.species, case.ws.species)):
        rad, kap, mj = q.q4c_spinor_basis(case.libS.tables, s)
        ref = S.spinor_functions(ss.l, list(case.kS[r0:r0 + len(ss.l)]))
        assert [(int(a), int(b), int(c)) for a, b, c in zip(rad, kap, mj)] == [(r[0], r[4], r[3]) for r in ref]
        _, kapL, mjL = q.q4c_spinor_basis(case.libL.tables, s)
        assert np.array_equal(kap, -kapL) and np.array_equal(mj, mjL)
        r0 += len(ss.l)
    assert q.q4c_spinor_nnz(case.libS.tables, case.libS.grid) == 4 * case.libL.grid.nnz


def test_eq19_hamiltonian_and_overlap(case):
    lib, orc = case.libS, case.orcS
    nfL, nfS = case.wl.nf_of_atom, case.ws.nf_of_atom
    q.q4c_tables_set_columns(lib.tables, case.eps[case.parent], case.Vk[case.parent])
    q.q4c_tables_set_columns(case.libL.tables, case.eps, case.Vk)
    FS = q.q4c_integrate_columns(lib.tables, lib.grid, lib.v)
    FL = q.q4c_integrate_columns(case.libL.tables, case.libL.grid, case.libL.v)
    HS, _ = q.q4c_spinor_transform(lib.tables, lib.grid, [FS, None, None, None, None], small=False)
    HL, _ = q.q4c_spinor_transform(case.libL.tables, case.libL.grid, [FL, None, None, None, None], small=False)
    lib.grid.status()
    FSo = orc.ob.matrix_columns(orc.xyz, orc.w, orc.v, case.eps[case.parent], case.Vk[case.parent], orc.pat)
    FLo = case.orcL.ob.matrix_columns(case.orcL.xyz, case.orcL.w, case.orcL.v, case.eps, case.Vk, case.orcL.pat)
    refS = _flat(S.transform_blocks([S.scalar_spin_large(b) for b in S.blocks_of(FSo, orc.pat, nfS)], orc.pat,
                                    case.GS, nfS), orc.pat)
    refL = _flat(S.transform_blocks([S.scalar_spin_large(b) for b in S.blocks_of(FLo, case.orcL.pat, nfL)],
                                    case.orcL.pat, case.GL, nfL), case.orcL.pat)
    hs, hl = HS.cpu().numpy(), HL.cpu().numpy()
    assert _rel(hs, refS) <= 1e-12
    assert _rel(hl + hs, refL + refS) <= 1e-12
    # the overlap S+ of the same two bases (v = 1: the V slots of q4c_integrate)
    one = lib.v * 0 + 1
    SS = q.q4c_integrate(lib.tables, lib.grid, one, "fp64")[0]
    SL = q.q4c_integrate(case.libL.tables, case.libL.grid, case.libL.v * 0 + 1, "fp64")[0]
    Sp = (q.q4c_spinor_transform(lib.tables, lib.grid, [SS] + [None] * 4, small=False)[0]
          + q.q4c_spinor_transform(case.libL.tables, case.libL.grid, [SL] + [None] * 4, small=False)[0])
    ones_o = np.ones(len(orc.w))
    SSo = orc.ob.matrix_blocks(orc.xyz, orc.w, ones_o, orc.pat)[0]
    SLo = case.orcL.ob.matrix_blocks(case.orcL.xyz, case.orcL.w, np.ones(len(case.orcL.w)), case.orcL.pat)[0]
    ref = (_flat(S.transform_blocks([S.scalar_spin_large(b) for b in S.blocks_of(SSo, orc.pat, nfS)], orc.pat,
                                    case.GS, nfS), orc.pat)
           + _flat(S.transform_blocks([S.scalar_spin_large(b) for b in S.blocks_of(SLo, case.orcL.pat, nfL)],
                                      case.orcL.pat, case.GL, nfL), case.orcL.pat))
    assert _rel(Sp.cpu().numpy(), ref) <= 1e-12


def test_small_reverse_map_and_density(case):
    import torch
    lib, orc = case.libS, case.orcS
    pat, nfS = orc.pat, case.ws.nf_of_atom
    ns = [G.shape[1] for G in case.GS]
    rng = np.random.default_rng(23)
    keys = {}
    for A in range(len(pat.blk_ptr) - 1):
        for qq in range(int(pat.blk_ptr[A]), int(pat.blk_ptr[A + 1])):
            keys[(A, int(pat.blk_col[qq]), tuple(int(t) for t in pat.blk_T[qq]))] = qq
    D = [None] * len(keys)
    for (A, B, T), qq in keys.items():
        if D[qq] is not None:
            continue
        X = rng.standard_normal((ns[A], ns[B])) + 1j * rng.standard_normal((ns[A], ns[B]))
        qt = keys[(B, A, tuple(-t for t in T))]
        if qt == qq:
            X = 0.5 * (X + X.conj().T)
        D[qq] = X
        D[qt] = X.conj().T if qt != qq else X
    P = q.q4c_spinor_density_matrices(lib.tables, lib.grid, torch.tensor(_flat(D, pat), device="cuda"))
    ref = S.scalar_density_matrices(D, pat, case.GS, nfS)
    assert rel_fro(P[0].cpu().numpy(), ref[0]) <= 1e-13
    n = q.q4c_density(lib.tables, lib.grid, P[0]).cpu().numpy()
    nref = orc.ob.density(orc.xyz, ref[0], pat)
    li, oi = point_map(lib.ex["point_id"], orc.ids)
    assert rel_fro(n[li], nref[oi]) <= 1e-12


def test_set_kappa_checks_and_resets():
    from paper_2608_00773_gb300 import _build
    _build.build()
    wl = water()
    t, g = q.setup(wl)
    bad = np.zeros(len(wl.rad_l), np.int32)
    bad[int(np.flatnonzero(wl.rad_l == 1)[0])] = 2  # kappa of l = 2 on a p radial
    with pytest.raises(q.Q4CError):
        q.q4c_tables_set_kappa(t, bad)
    sel = np.where(wl.rad_l > 0, wl.rad_l, -1).astype(np.int32)  # j = l - 1/2 where it exists
    q.q4c_tables_set_kappa(t, sel)
    assert q.q4c_spinor_nnz(t, g) < 4 * g.nnz
    q.q4c_tables_set_kappa(t, None)
    assert q.q4c_spinor_nnz(t, g) == 4 * g.nnz
    for s, sp in enumerate(wl.species):
        assert len(q.q4c_spinor_basis(t, s)[0]) == 2 * sp.n_fn
