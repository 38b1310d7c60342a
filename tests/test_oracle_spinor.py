"""Pins of the oracle's scalar -> spinor transformation (Eqs. 9-14, 33-34,
37-38, Appendix A, Algorithm 1).  CPU only.

What fixes it from outside:
* textbook Clebsch-Gordan values and their orthonormality (and sympy's
  values where sympy is installed);
* unitarity of G;
* physics: for one atom in a spherical potential the small-component block
  G^dagger (W0 1 + i SO.sigma) G must be diagonal in (kappa, m_j) and equal
  for all m_j of one kappa (kappa, m_j are good quantum numbers), while the
  literal Eq. 13 phases break that (a planted variant);
* Eq. 33 both ways: G^dagger F G equals the quadrature of the spinor
  functions themselves, chi = sum G phi eta (and sigma.grad of it for the
  small component), at the grid points;
* Eq. 38 both ways: the scalar density matrices of the reverse map give the
  density that the spinor functions give point by point;
* forward and reverse maps are adjoint: Re sum D F~ = sum P F;
* Algorithm 1 on a set of local functions.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import spinor as S
from workloads import potential, single_atom, water


def test_clebsch_gordan_textbook_values():
    h = 1  # doubled 1/2
    assert abs(S.clebsch_gordan(0, 0, h, h, h, h) - 1.0) < 1e-15
    assert abs(S.clebsch_gordan(2, 0, h, h, h, h) + math.sqrt(1 / 3)) < 1e-15      # <1 0; 1/2 1/2 | 1/2 1/2>
    assert abs(S.clebsch_gordan(2, 2, h, -h, h, h) - math.sqrt(2 / 3)) < 1e-15     # <1 1; 1/2 -1/2 | 1/2 1/2>
    assert abs(S.clebsch_gordan(2, 0, h, h, 3, h) - math.sqrt(2 / 3)) < 1e-15      # <1 0; 1/2 1/2 | 3/2 1/2>
    assert abs(S.clebsch_gordan(2, 2, h, -h, 3, h) - math.sqrt(1 / 3)) < 1e-15     # <1 1; 1/2 -1/2 | 3/2 1/2>
    assert abs(S.clebsch_gordan(4, 4, h, h, 5, 5) - 1.0) < 1e-15                   # stretched state
    # orthonormality over (m1, m2) for fixed (J, M), and completeness over J
    for l in range(4):
        for Jx2 in ([2 * l - 1] if l else []) + [2 * l + 1]:
            for Mx2 in range(-Jx2, Jx2 + 1, 2):
                nrm = sum(S.clebsch_gordan(2 * l, Mx2 - ms, 1, ms, Jx2, Mx2) ** 2 for ms in (1, -1))
                assert abs(nrm - 1) < 1e-14


def test_clebsch_gordan_against_sympy():
    cg = pytest.importorskip("sympy.physics.quantum.cg")
    from sympy import Rational
    for l in range(4):
        for Jx2 in ([2 * l - 1] if l else []) + [2 * l + 1]:
            for Mx2 in range(-Jx2, Jx2 + 1, 2):
                for ms in (1, -1):
                    ml = Mx2 - ms
                    if abs(ml) > 2 * l:
                        continue
                    ref = float(cg.CG(l, Rational(ml, 2), Rational(1, 2), Rational(ms, 2), Rational(Jx2, 2),
                                      Rational(Mx2, 2)).doit())
                    assert abs(S.clebsch_gordan(2 * l, ml, 1, ms, Jx2, Mx2) - ref) < 1e-14


def test_spinor_counts_and_unitarity():
    for l_list in ([0], [1], [0, 1, 2, 3], [0, 0, 1, 1, 2]):
        fns = S.spinor_functions(l_list)
        n = sum(2 * l + 1 for l in l_list)
        assert len(fns) == 2 * n
        for (q, l, jx2, mjx2, kappa) in fns:
            assert kappa == (l if jx2 == 2 * l - 1 else -l - 1) and jx2 in (2 * l - 1, 2 * l + 1)
        G = S.transformation_matrix(l_list)
        assert np.abs(G.conj().T @ G - np.eye(2 * n)).max() < 1e-14
        assert np.abs(G @ G.conj().T - np.eye(2 * n)).max() < 1e-14


def _one_atom_small_block(phase):
    wl = single_atom([0, 1, 1, 2, 3], [1.4, 1.6, 2.9, 1.9, 2.4], Z=5.0, n_rad=100)
    xyz, w, _ = O.grid(wl)
    ob = O.OracleBasis(wl, analytic=True)
    pat = ob.pattern()
    V, W0, SOx, SOy, SOz = [ob.dense(m, pat) for m in ob.matrix_blocks(xyz, w, potential(xyz, wl), pat)]
    G = S.transformation_matrix(wl.species[0].l, phase)
    return wl, G.conj().T @ S.scalar_spin_small(W0, SOx, SOy, SOz) @ G, G.conj().T @ S.scalar_spin_large(V) @ G


def test_one_atom_spinor_blocks_are_diagonal_in_kappa_mj():
    """Spherical potential: the spinor blocks couple only equal (kappa, m_j)
    (any radial pair), with one value per (radial pair, kappa); the small
    component's j = l +- 1/2 values differ (spin-orbit splitting)."""
    wl, Hs, Hl = _one_atom_small_block("cs")
    fns = S.spinor_functions(wl.species[0].l)
    scale = np.abs(Hs).max()
    for H in (Hs, Hl):
        sc = np.abs(H).max()
        for a, (qa, la, ja, ma, ka) in enumerate(fns):
            for b, (qb, lb, jb, mb, kb) in enumerate(fns):
                if (ka, ma) != (kb, mb):
                    assert abs(H[a, b]) < 1e-12 * sc, (a, b)
    # m_j independence: one value per (qa, qb, kappa)
    vals = {}
    for a, (qa, la, ja, ma, ka) in enumerate(fns):
        for b, (qb, lb, jb, mb, kb) in enumerate(fns):
            if (ka, ma) == (kb, mb):
                vals.setdefault((qa, qb, ka), []).append(Hs[a, b])
    for v in vals.values():
        assert max(abs(x - v[0]) for x in v) < 1e-11 * scale
    # the p shell splits: kappa = 1 (p1/2) and kappa = -2 (p3/2) differ
    assert abs(vals[(1, 1, 1)][0] - vals[(1, 1, -2)][0]) > 1e-3 * abs(vals[(1, 1, -2)][0])


def test_eq13_phases_as_printed_break_the_coupling():
    """A planted variant: with the phases printed in Eq. 13 applied to the real
    harmonics of Appendix B, the spin-orbit part mixes different m_j or kappa."""
    wl, Hs, _ = _one_atom_small_block("eq13")
    fns = S.spinor_functions(wl.species[0].l)
    off = max(abs(Hs[a, b]) for a, fa in enumerate(fns) for b, fb in enumerate(fns)
              if (fa[4], fa[3]) != (fb[4], fb[3]))
    assert off > 1e-3 * np.abs(Hs).max()


def _chi(G, phi, grad):
    """Spinor functions at points: chi[mu, p, s] (large) and sigma.grad chi (small)."""
    n = phi.shape[0]
    Gr = G.reshape(n, 2, -1)  # [t, s, mu]
    chiL = np.einsum("tsm,tp->mps", Gr, phi)
    chiS = np.zeros_like(chiL)
    for k, P in enumerate(S.PAULI):
        # (sigma_k eta_s) components: sum_s' (P)_{s' s}
        chiS += np.einsum("tsm,tp,us->mpu", Gr, grad[:, :, k], P)
    return chiL, chiS


def test_eq33_transform_equals_spinor_quadrature():
    """G^dagger (V 1) G and G^dagger (W0 1 + i SO.sigma) G equal the grid sums of
    w v chi_mu^dagger chi_nu and w v (sigma.grad chi_mu)^dagger (sigma.grad chi_nu)."""
    wl = water()
    xyz, w, _ = O.grid(wl)
    ob = O.OracleBasis(wl)
    pat = ob.pattern()
    v = potential(xyz, wl)
    V, W0, SOx, SOy, SOz = [ob.dense(m, pat) for m in ob.matrix_blocks(xyz, w, v, pat)]
    Gs = S.atom_matrices(wl)
    nf = wl.nf_of_atom
    from scipy.linalg import block_diag
    G = block_diag(*Gs)
    Hl = G.conj().T @ S.scalar_spin_large(V) @ G
    Hs = G.conj().T @ S.scalar_spin_small(W0, SOx, SOy, SOz) @ G
    phi, grad = ob.eval(xyz)
    chiL, chiS = _chi(G, phi, grad)
    wv = w * v
    refL = np.einsum("mps,p,nps->mn", chiL.conj(), wv, chiL)
    refS = np.einsum("mps,p,nps->mn", chiS.conj(), wv, chiS)
    assert np.abs(Hl - refL).max() <= 1e-12 * np.abs(refL).max()
    assert np.abs(Hs - refS).max() <= 1e-12 * np.abs(refS).max()
    assert int(np.sum(nf)) * 2 == G.shape[1]


def _random_hermitian_blocks(pat, nf, seed):
    """Random spinor density blocks with D(B, A, -T) = D(A, B, T)^dagger."""
    rng = np.random.default_rng(seed)
    keys = {}
    for A in range(len(pat.blk_ptr) - 1):
        for q in range(int(pat.blk_ptr[A]), int(pat.blk_ptr[A + 1])):
            keys[(A, int(pat.blk_col[q]), tuple(int(t) for t in pat.blk_T[q]))] = q
    D = [None] * len(keys)
    for (A, B, T), q in sorted(keys.items(), key=lambda kv: kv[1]):
        if D[q] is not None:
            continue
        X = rng.standard_normal((2 * nf[A], 2 * nf[B])) + 1j * rng.standard_normal((2 * nf[A], 2 * nf[B]))
        qt = keys[(B, A, tuple(-t for t in T))]
        if qt == q:
            X = 0.5 * (X + X.conj().T)
        D[q] = X
        D[qt] = X.conj().T if qt != q else X
    return D


def test_eq38_reverse_map_gives_the_spinor_density():
    """n^L(p) = Re sum D chi^dagger chi and n^S(p) with sigma.grad chi, point by
    point, equal the scalar densities of the reverse map's P matrices."""
    wl = water()
    xyz, w, _ = O.grid(wl)
    xyz = xyz[::7]
    ob = O.OracleBasis(wl)
    pat = ob.pattern()
    nf = wl.nf_of_atom
    Gs = S.atom_matrices(wl)
    D = _random_hermitian_blocks(pat, nf, 5)
    P = S.scalar_density_matrices(D, pat, Gs, nf)
    nL = ob.density(xyz, P[0], pat)
    nS = ob.density_full(xyz, [None, P[1], P[2], P[3], P[4]], pat)
    from scipy.linalg import block_diag
    G = block_diag(*Gs)
    Dd = np.zeros((G.shape[1], G.shape[1]), complex)
    first = np.concatenate([[0], np.cumsum(2 * nf)])
    q = 0
    for A in range(wl.n_atoms):
        for qq in range(int(pat.blk_ptr[A]), int(pat.blk_ptr[A + 1])):
            B = int(pat.blk_col[qq])
            Dd[first[A]:first[A + 1], first[B]:first[B + 1]] = D[q]
            q += 1
    phi, grad = ob.eval(xyz)
    chiL, chiS = _chi(G, phi, grad)
    refL = np.einsum("mn,mps,nps->p", Dd, chiL.conj(), chiL).real
    refS = np.einsum("mn,mps,nps->p", Dd, chiS.conj(), chiS).real
    assert np.abs(nL - refL).max() <= 1e-12 * np.abs(refL).max()
    assert np.abs(nS - refS).max() <= 1e-12 * np.abs(refS).max()


def test_forward_and_reverse_maps_are_adjoint():
    wl = water()
    xyz, w, _ = O.grid(wl)
    ob = O.OracleBasis(wl)
    pat = ob.pattern()
    nf = wl.nf_of_atom
    mats = ob.matrix_blocks(xyz, w, potential(xyz, wl), pat)
    Gs = S.atom_matrices(wl)
    Fl = [S.scalar_spin_large(b) for b in S.blocks_of(mats[0], pat, nf)]
    Fs = [S.scalar_spin_small(*bs) for bs in zip(*[S.blocks_of(m, pat, nf) for m in mats[1:]])]
    Hl, Hs = S.transform_blocks(Fl, pat, Gs, nf), S.transform_blocks(Fs, pat, Gs, nf)
    D = _random_hermitian_blocks(pat, nf, 9)
    P = S.scalar_density_matrices(D, pat, Gs, nf)
    lhs = sum(float(np.sum(d * (hl + hs)).real) for d, hl, hs in zip(D, Hl, Hs))
    rhs = sum(float(np.dot(p, m)) for p, m in zip(P, mats))
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs)


def test_algorithm1_local_spinor_index_map():
    """Spinor functions present for a set of local scalar functions: those of
    the radial shells that have a local function, in global order; a set of
    whole atoms gives twice its function count."""
    l_list = [0, 1, 2]
    per_atom = sum(2 * l + 1 for l in l_list)
    n_atoms = 3
    fn_shell, shell_spinors, g = [], {}, 0
    for a in range(n_atoms):
        for q, l in enumerate(l_list):
            fn_shell += [a * len(l_list) + q] * (2 * l + 1)
        for q, l in enumerate(l_list):
            sh = a * len(l_list) + q
            shell_spinors[sh] = list(range(g, g + 2 * (2 * l + 1)))
            g += 2 * (2 * l + 1)
    local = list(range(per_atom, 2 * per_atom))  # atom 1 whole
    got = S.batch_spinors(local, fn_shell, shell_spinors)
    assert got == list(range(2 * per_atom, 4 * per_atom))
    got = S.batch_spinors([0, per_atom + 1], fn_shell, shell_spinors)  # an s function of atom 0, a p of atom 1
    assert got == [0, 1] + list(range(2 * per_atom + 2, 2 * per_atom + 8))
