"""Pins of the small-component spinor functions of the oracle (Eqs. 7-8b, 11,
12b, 14, 19, 21): Q radials with kappa~ = -kappa per radial (the G^S of
Eq. 14).  CPU only.

What fixes it from outside:
* Eq. 7 point by point: with V = 0 the balance is K = sigma.p / 2c, so the
  small components sum_t G^S_(t s),mu Q_t/r Y_t (the i of Eq. 12b taken out)
  must equal -(1/2c) sigma.grad chi^L_mu at any point, for every spinor
  function: this fixes l~, the sign and kappa term of Q, the pairing
  kappa~ = -kappa and the coupling phases of the small component (a Q with
  the kappa term's sign flipped, planted here, fails);
* the same identity integrated: (2c)^2 G^S^dagger (S^S x 1) G^S equals the
  kinetic-balance block G^dagger (W0 1 + i SO.sigma) G of the gradients with
  v = 1, for a molecule (all blocks, cross-atom ones included);
* Eq. 21 point by point: the scalar density matrix of the reverse map with
  G^S gives the density Re sum D chi^S^dagger chi^S of the spinor functions.

Exponents below 1 are raised to 1 here: for diffuse functions the Q radial
(which contains the derivative of the cutoff) varies on the scale of the knot
spacing between r_on and r_c, where the 200-knot spline of Q, and of P's
derivative, are off by percents."""
import dataclasses

import numpy as np
import pytest
from scipy.linalg import block_diag

import oracle as O
from oracle import spinor as S
from workloads import C_LIGHT, Species, column_operator, small_component, small_radial, water


def compact(wl):
    sp = [Species(s.name, s.Z, s.l, [max(a, 1.0) for a in s.alpha]) for s in wl.species]
    return dataclasses.replace(wl, species=sp)


@pytest.fixture(scope="module")
def mol():
    wl = compact(water())
    _, Vk = column_operator(wl, 5)
    ws, Q, parent, kappa = small_component(wl, 0 * Vk)
    return wl, ws, Q, kappa, parent


def _sigma_grad(G, grad):
    n = grad.shape[0]
    Gr = G.reshape(n, 2, -1)
    out = np.zeros((G.shape[1], grad.shape[1], 2), complex)
    for k, P in enumerate(S.PAULI):
        out += np.einsum("tsm,tp,us->mpu", Gr, grad[:, :, k], P)
    return out


def _values(G, phi):
    return np.einsum("tsm,tp->mps", G.reshape(phi.shape[0], 2, -1), phi)


def test_spinor_counts_line_up(mol):
    wl, ws, Q, kappa, parent = mol
    for sl, ss, ks in zip(wl.species, ws.species, np.split(-kappa, np.cumsum([len(s.l) for s in ws.species])[:-1])):
        fl = S.spinor_functions(sl.l)
        fs = S.spinor_functions(ss.l, list(ks))
        assert len(fl) == len(fs) == 2 * sl.n_fn
        # the same (j, m_j) in the same order, with kappa~ = -kappa
        assert [(f[2], f[3], -f[4]) for f in fl] == [(f[2], f[3], f[4]) for f in fs]


def test_small_spinors_are_the_balance_of_the_large_ones(mol):
    wl, ws, Q, kappa, parent = mol
    oL, oS = O.OracleBasis(wl), O.OracleBasis(ws, knots=Q)
    GL = block_diag(*S.atom_matrices(wl))
    GS = block_diag(*S.atom_matrices(ws, kappas=-kappa))
    rng = np.random.default_rng(11)
    pts = wl.xyz[rng.integers(0, wl.n_atoms, 300)] + rng.normal(0, 1.2, (300, 3))
    phL, grL = oL.eval(pts)
    phS, _ = oS.eval(pts)
    X = _values(GS, phS)
    Y = -_sigma_grad(GL, grL) / (2 * C_LIGHT)
    scale = np.abs(Y).max()
    # spline derivatives of P against spline values of Q: ~2e-5 apart
    assert np.abs(X - Y).max() <= 1e-4 * scale
    # a planted mistake: the kappa term of Q with the wrong sign
    r = wl.r_min * (wl.r_c / wl.r_min) ** (np.arange(wl.n_log) / (wl.n_log - 1))
    r[-1] = wl.r_c
    Qw = np.array([small_radial(r, wl.rad_l[parent[k]], wl.rad_alpha[parent[k]], -kappa[k], 0.0, wl.r_on, wl.r_c)
                   for k in range(len(kappa))])
    phW, _ = O.OracleBasis(ws, knots=Qw).eval(pts)
    assert np.abs(_values(GS, phW) - Y).max() > 0.1 * scale


def test_small_overlap_is_the_kinetic_balance_block(mol):
    wl, ws, Q, kappa, parent = mol
    xyz, w, _ = O.grid(wl)
    oL, oS = O.OracleBasis(wl), O.OracleBasis(ws, knots=Q)
    pL, pS = oL.pattern(), oS.pattern()
    one = np.ones(len(w))
    SS = oS.dense(oS.matrix_blocks(xyz, w, one, pS)[0], pS)
    _, W0, SOx, SOy, SOz = [oL.dense(m, pL) for m in oL.matrix_blocks(xyz, w, one, pL)]
    GL = block_diag(*S.atom_matrices(wl))
    GS = block_diag(*S.atom_matrices(ws, kappas=-kappa))
    lhs = (2 * C_LIGHT) ** 2 * (GS.conj().T @ np.kron(SS, np.eye(2)) @ GS)
    rhs = GL.conj().T @ S.scalar_spin_small(W0, SOx, SOy, SOz) @ GL
    assert np.abs(lhs - rhs).max() <= 1e-4 * np.abs(rhs).max()
    # off-atom blocks are present and agree too
    nA = 2 * wl.nf_of_atom[0]
    assert np.abs(rhs[:nA, nA:]).max() > 1e-2 * np.abs(rhs).max()


def test_reverse_map_gives_the_small_component_density(mol):
    wl, ws, Q, kappa, parent = mol
    oS = O.OracleBasis(ws, knots=Q)
    pat = oS.pattern()
    nfS = ws.nf_of_atom
    Gs = S.atom_matrices(ws, kappas=-kappa)
    ns = np.array([G.shape[1] for G in Gs])
    rng = np.random.default_rng(4)
    keys = {}
    for A in range(wl.n_atoms):
        for q in range(int(pat.blk_ptr[A]), int(pat.blk_ptr[A + 1])):
            keys[(A, int(pat.blk_col[q]))] = q
    D = [None] * len(keys)
    for (A, B), q in keys.items():
        if D[q] is None:
            X = rng.standard_normal((ns[A], ns[B])) + 1j * rng.standard_normal((ns[A], ns[B]))
            qt = keys[(B, A)]
            if qt == q:
                X = 0.5 * (X + X.conj().T)
            D[q] = X
            D[qt] = X.conj().T if qt != q else X
    P = S.scalar_density_matrices(D, pat, Gs, nfS)
    xyz, _, _ = O.grid(ws)
    xyz = xyz[::9]
    n = oS.density(xyz, P[0], pat)
    G = block_diag(*Gs)
    first = np.concatenate([[0], np.cumsum(ns)])
    Dd = np.zeros((G.shape[1], G.shape[1]), complex)
    for (A, B), q in keys.items():
        Dd[first[A]:first[A + 1], first[B]:first[B + 1]] = D[q]
    phi, _ = oS.eval(xyz)
    chi = _values(G, phi)
    ref = np.einsum("mn,mps,nps->p", Dd, chi.conj(), chi).real
    assert np.abs(n - ref).max() <= 1e-12 * np.abs(ref).max()
