"""GPU parity of the scalar -> spinor transformation (Eqs. 9-14, 33-34,
37-38, Algorithm 1) against the oracle: the spinor basis bit-exact, the
forward and reverse maps on identical seeded inputs within 1e-13 relative,
the forward map of the library's own integrals against the oracle's
integrals transformed by the oracle (1e-12), on a molecule and on a periodic
cell (blocks with shifts T)."""
import numpy as np
import pytest

import oracle as O
import paper_2608_00773_gb300 as q
from gpu_helpers import LibCase, OracleCase
from oracle import spinor as S
from workloads import periodic_cell, water

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["water", "cell"])
def case(request):
    from paper_2608_00773_gb300 import _build
    _build.build()
    O.build()
    wl = water() if request.param == "water" else periodic_cell()
    return LibCase(wl), OracleCase(wl)


def _flat(blocks, pat, nf):
    out = np.zeros(4 * int(pat.blk_off[-1]), complex)
    for qq, (A, B) in enumerate(_pairs(pat)):
        o = 4 * int(pat.blk_off[qq])
        out[o:o + blocks[qq].size] = blocks[qq].reshape(-1)
    return out


def _pairs(pat):
    return [(A, int(pat.blk_col[qq])) for A in range(len(pat.blk_ptr) - 1)
            for qq in range(int(pat.blk_ptr[A]), int(pat.blk_ptr[A + 1]))]


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def test_spinor_basis_matches_oracle(case):
    lib, orc = case
    for s, sp in enumerate(lib.wl.species):
        rad, kap, mj = q.q4c_spinor_basis(lib.tables, s)
        ref = S.spinor_functions(sp.l)
        assert len(rad) == len(ref) == 2 * sp.n_fn
        assert [(int(a), int(b), int(c)) for a, b, c in zip(rad, kap, mj)] == [(r[0], r[4], r[3]) for r in ref]


def test_forward_transform_on_seeded_blocks(case):
    import torch
    lib, orc = case
    kinds = [("GV", False), ("GW0", False), ("GSOx", True), ("GSOy", True), ("GSOz", True)]
    F = [lib.random(91, k, a) for k, a in kinds]
    HL, HS = q.q4c_spinor_transform(lib.tables, lib.grid, F)
    Fo = [orc.random(91, k, a) for k, a in kinds]
    nf = lib.wl.nf_of_atom
    Gs = S.atom_matrices(lib.wl)
    Fl = [S.scalar_spin_large(b) for b in S.blocks_of(Fo[0], orc.pat, nf)]
    Fs = [S.scalar_spin_small(*bs) for bs in zip(*[S.blocks_of(m, orc.pat, nf) for m in Fo[1:]])]
    refL = _flat(S.transform_blocks(Fl, orc.pat, Gs, nf), orc.pat, nf)
    refS = _flat(S.transform_blocks(Fs, orc.pat, Gs, nf), orc.pat, nf)
    assert _rel(HL.cpu().numpy(), refL) <= 1e-13
    assert _rel(HS.cpu().numpy(), refS) <= 1e-13
    # the small component alone, and NULL SO slots counting as zero
    _, HS2 = q.q4c_spinor_transform(lib.tables, lib.grid, [None, F[1], None, None, None], large=False)
    Fs2 = [S.scalar_spin_small(b, 0 * b, 0 * b, 0 * b) for b in S.blocks_of(Fo[1], orc.pat, nf)]
    assert _rel(HS2.cpu().numpy(), _flat(S.transform_blocks(Fs2, orc.pat, Gs, nf), orc.pat, nf)) <= 1e-13
    torch.cuda.synchronize()


def _hermitian_blocks(pat, nf, seed):
    rng = np.random.default_rng(seed)
    keys = {}
    for qq, (A, B) in enumerate(_pairs(pat)):
        keys[(A, B, tuple(int(t) for t in pat.blk_T[qq]))] = qq
    D = [None] * len(keys)
    for (A, B, T), qq in keys.items():
        if D[qq] is not None:
            continue
        X = rng.standard_normal((2 * nf[A], 2 * nf[B])) + 1j * rng.standard_normal((2 * nf[A], 2 * nf[B]))
        qt = keys[(B, A, tuple(-t for t in T))]
        if qt == qq:
            X = 0.5 * (X + X.conj().T)
        D[qq] = X
        D[qt] = X.conj().T if qt != qq else X
    return D


def test_reverse_map_on_seeded_density_matrix(case):
    import torch
    lib, orc = case
    nf = lib.wl.nf_of_atom
    D = _hermitian_blocks(orc.pat, nf, 17)
    Dd = torch.tensor(_flat(D, orc.pat, nf), device="cuda")
    P = q.q4c_spinor_density_matrices(lib.tables, lib.grid, Dd)
    ref = S.scalar_density_matrices(D, orc.pat, S.atom_matrices(lib.wl), nf)
    for k in range(5):
        assert _rel(P[k].cpu().numpy(), ref[k]) <= 1e-13, k
    # the large- and small-component densities of these matrices, on the GPU
    n = q.q4c_density(lib.tables, lib.grid, P[0]).cpu().numpy()
    nref = orc.ob.density(orc.xyz, ref[0], orc.pat)
    from gpu_helpers import point_map, rel_fro
    li, oi = point_map(lib.ex["point_id"], orc.ids)
    assert rel_fro(n[li], nref[oi]) <= 1e-12
    ns = q.q4c_density_full(lib.tables, lib.grid, [None] + P[1:]).cpu().numpy()
    nsref = orc.ob.density_full(orc.xyz, [None] + ref[1:], orc.pat)
    assert rel_fro(ns[li], nsref[oi]) <= 1e-12


def test_forward_transform_of_integrals(case):
    lib, orc = case
    outs = q.q4c_integrate(lib.tables, lib.grid, lib.v, "fp64")
    HL, HS = q.q4c_spinor_transform(lib.tables, lib.grid, outs[:5])
    nf = lib.wl.nf_of_atom
    Gs = S.atom_matrices(lib.wl)
    mats = orc.mats
    Fl = [S.scalar_spin_large(b) for b in S.blocks_of(mats[0], orc.pat, nf)]
    Fs = [S.scalar_spin_small(*bs) for bs in zip(*[S.blocks_of(m, orc.pat, nf) for m in mats[1:]])]
    refL = _flat(S.transform_blocks(Fl, orc.pat, Gs, nf), orc.pat, nf)
    refS = _flat(S.transform_blocks(Fs, orc.pat, Gs, nf), orc.pat, nf)
    assert np.linalg.norm(HL.cpu().numpy() - refL) <= 1e-12 * np.linalg.norm(refL)
    assert np.linalg.norm(HS.cpu().numpy() - refS) <= 1e-12 * np.linalg.norm(refS)


def test_batch_spinors_algorithm1(case):
    lib, _ = case
    ex = lib.ex
    info_nb = np.diff(ex["batch_fn_ptr"]) if "batch_fn_ptr" in ex else None
    for b in range(0, len(ex["batch_ptr"]) - 1, max(1, (len(ex["batch_ptr"]) - 1) // 7)):
        cen, mu = lib.grid.batch_spinors(b)
        act = ex["batch_atoms"][ex["batch_atom_ptr"][b]:ex["batch_atom_ptr"][b + 1]]
        # every active centre contributes all spinor functions of its atom, in order
        nA = lib.wl.n_atoms
        per = [2 * int(lib.wl.nf_of_atom[c % nA]) for c in act]
        assert len(cen) == sum(per)
        assert np.array_equal(cen, np.repeat(act, per))
        assert np.array_equal(mu, np.concatenate([np.arange(p) for p in per]))
        if info_nb is not None:
            assert len(cen) == 2 * int(info_nb[b])
