"""Pins of the oracle's periodic path (real-space H(T) blocks, Eqs. 24-25).

The periodic sums are checked against things other than themselves: a
closed form (Gaussian overlap and kinetic integrals between a centre and the
images of another, which fixes the sign convention of T), the molecular
result (a huge cell), a 2x1x1 supercell that must fold onto the primitive
cell's blocks, rigid translation, the transpose symmetry of H(T), and the
trace and linearity identities of the density and the adjoint.  CPU only.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle as O
from workloads import ADJOINT_KINDS, Species, Workload, fill_pattern, periodic_cell, potential, water


def _blocks(pat):
    """(A, B, T) -> block index"""
    out = {}
    for A in range(len(pat.blk_ptr) - 1):
        for q in range(int(pat.blk_ptr[A]), int(pat.blk_ptr[A + 1])):
            out[(A, int(pat.blk_col[q]), tuple(int(t) for t in pat.blk_T[q]))] = q
    return out


def _block(vals, pat, q, nfA, nfB):
    o = int(pat.blk_off[q])
    return np.asarray(vals[o:o + nfA * nfB]).reshape(nfA, nfB)


def test_huge_cell_equals_molecule():
    """With images 1000 Bohr away the periodic path is the molecular one, bit for bit."""
    wl = water()
    wlp = dataclasses.replace(wl, lattice=1000.0 * np.eye(3), n_shell=1)
    xyz, w, ids = O.grid(wl)
    xyzp, wp, idsp = O.grid(wlp)
    assert np.array_equal(ids, idsp) and np.array_equal(xyz, xyzp) and np.array_equal(w, wp)
    ob, obp = O.OracleBasis(wl), O.OracleBasis(wlp)
    pat, patp = ob.pattern(), obp.pattern()
    assert np.array_equal(pat.blk_col, patp.blk_col) and np.array_equal(pat.blk_off, patp.blk_off)
    assert not patp.blk_T.any()
    v = potential(xyz, wl)
    for a, b in zip(ob.matrix_blocks(xyz, w, v, pat), obp.matrix_blocks(xyz, w, v, patp)):
        assert np.array_equal(a, b)


def test_image_gaussian_overlap_and_kinetic_closed_form():
    """Two s-Gaussian centres in a cell 3.5 Bohr long in x: every block (A, B, T)
    is the overlap of phi_A at R_A with phi_B at R_B + T.L,
    S = (pi/p)^(3/2) exp(-mu d^2)/(4 pi), d = |R_A - R_B - T.L|, and
    W0(v = 1) = 2 mu (3 - 2 mu d^2) S."""
    a, b = 1.3, 1.7
    sp = [Species("A", 1.0, [0], [a]), Species("B", 1.0, [0], [b])]
    L = np.diag([3.5, 30.0, 30.0])
    wl = Workload("pair-cell", np.array([[0.2, 0.0, 0.0], [0.5, 0.5, 1.4]]), np.array([0, 1], np.int32), sp,
                  n_rad=90, n_theta=20, n_phi=40, r_nb=7.0, lattice=L, n_shell=4)
    xyz, w, _ = O.grid(wl)
    ob = O.OracleBasis(wl, analytic=True)
    pat = ob.pattern()
    V, W0, *_ = ob.matrix_blocks(xyz, w, np.ones(len(w)), pat)
    al = (a, b)
    checked = 0
    for (A, B, T), q in _blocks(pat).items():
        d = wl.xyz[A] - wl.xyz[B] - np.asarray(T, float) @ L
        d2 = float(d @ d)
        p, mu = al[A] + al[B], al[A] * al[B] / (al[A] + al[B])
        S = (math.pi / p) ** 1.5 * math.exp(-mu * d2) / (4 * math.pi)
        if S < 1e-6:
            continue
        Wk = 2 * mu * (3 - 2 * mu * d2) * S
        # quadrature error at 90 x 800 points: ~1e-7 relative (1e-5 at 60 x 392);
        # a flipped sign of T would change the image overlaps by percents
        assert abs(V[int(pat.blk_off[q])] / S - 1) < 1e-6, (A, B, T)
        assert abs(W0[int(pat.blk_off[q])] / Wk - 1) < 1e-6, (A, B, T)
        checked += 1
    # blocks with T != 0 (the images along x) are among those checked
    assert checked >= 8 and any(T != (0, 0, 0) for (_, _, T) in _blocks(pat))


@pytest.fixture(scope="module")
def cell_case():
    wl = periodic_cell()
    xyz, w, ids = O.grid(wl)
    ob = O.OracleBasis(wl)
    pat = ob.pattern()
    v = potential(xyz, wl)
    mats = ob.matrix_blocks(xyz, w, v, pat)
    return wl, xyz, w, ids, ob, pat, v, mats


def test_transpose_symmetry(cell_case):
    """H(T)_AB = H(-T)_BA^T for V and W0, and = -H(-T)_BA^T for the spin-orbit parts."""
    wl, xyz, w, ids, ob, pat, v, mats = cell_case
    nf = wl.nf_of_atom
    blk = _blocks(pat)
    for (A, B, T), q in blk.items():
        qt = blk[(B, A, tuple(-t for t in T))]
        for k, m in enumerate(mats):
            X = _block(m, pat, q, nf[A], nf[B])
            Y = _block(m, pat, qt, nf[B], nf[A]).T
            sign = 1.0 if k < 2 else -1.0
            assert np.abs(X - sign * Y).max() <= 1e-15 * max(np.abs(m).max(), 1e-300)


def test_supercell_folds_onto_the_primitive_cell(cell_case):
    """A 2x1x1 supercell's block ((A, sa), (B, sb), T') equals the primitive
    cell's block (A, B, (sb - sa + 2 T'_1, T'_2, T'_3))."""
    wl, xyz, w, ids, ob, pat, v, mats = cell_case
    L = np.asarray(wl.lattice)
    n = wl.n_atoms
    wls = dataclasses.replace(wl, xyz=np.vstack([wl.xyz, wl.xyz + L[0]]),
                              species_of_atom=np.concatenate([wl.species_of_atom, wl.species_of_atom]),
                              lattice=np.vstack([2 * L[0], L[1], L[2]]))
    xyzs, ws, _ = O.grid(wls)
    obs = O.OracleBasis(wls)
    pats = obs.pattern()
    mats_s = obs.matrix_blocks(xyzs, ws, potential(xyzs, wls), pats)
    blk = _blocks(pat)
    nf = wl.nf_of_atom
    err = ref = 0.0
    for (As, Bs, Ts), qs in _blocks(pats).items():
        A, sa, B, sb = As % n, As // n, Bs % n, Bs // n
        T = (sb - sa + 2 * Ts[0], Ts[1], Ts[2])
        q = blk[(A, B, T)]
        for m, ms in zip(mats, mats_s):
            X = _block(m, pat, q, nf[A], nf[B])
            Y = _block(ms, pats, qs, nf[A], nf[B])
            err = max(err, float(np.abs(X - Y).max()))
            ref = max(ref, float(np.abs(X).max()))
    assert err <= 1e-12 * ref


def test_rigid_translation(cell_case):
    wl, xyz, w, ids, ob, pat, v, mats = cell_case
    wl2 = wl.translated([0.37, -1.2, 2.05])
    xyz2, w2, ids2 = O.grid(wl2)
    ob2 = O.OracleBasis(wl2)
    pat2 = ob2.pattern()
    assert np.array_equal(pat.blk_T, pat2.blk_T)
    mats2 = ob2.matrix_blocks(xyz2, w2, potential(xyz2, wl2), pat2)
    for a, b in zip(mats, mats2):
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(a)


def test_density_trace_and_adjoint_linearity(cell_case):
    """sum_p w_p n_p = sum over stored elements of P S with S = V(v = 1); and
    sum_p v_p dL/dv_p = L = sum_M <G^M, M(v)>, on the periodic pattern."""
    wl, xyz, w, ids, ob, pat, v, mats = cell_case
    nf = wl.nf_of_atom
    P = fill_pattern(pat.blk_ptr, pat.blk_col, pat.blk_off, nf, 21, "P", blk_T=pat.blk_T)
    S = ob.matrix_blocks(xyz, w, np.ones(len(w)), pat)[0]
    n = ob.density(xyz, P, pat)
    lhs, rhs = float((w * n).sum()), float((P * S).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs)
    G = [fill_pattern(pat.blk_ptr, pat.blk_col, pat.blk_off, nf, 22, k, a, blk_T=pat.blk_T)
         for k, a in ADJOINT_KINDS]
    g = ob.adjoint(xyz, w, G, pat)
    L = sum(float((Gm * M).sum()) for Gm, M in zip(G, mats))
    assert abs(float((v * g).sum()) - L) <= 1e-11 * abs(L)


def test_periodic_inputs():
    """v is lattice-periodic and the random blocks pair (A, B, T) with (B, A, -T)."""
    wl = periodic_cell()
    L = np.asarray(wl.lattice)
    rng = np.random.default_rng(3)
    pts = rng.uniform(0, 9, (20, 3))
    assert np.allclose(potential(pts, wl), potential(pts + L[1], wl), rtol=1e-13, atol=1e-13)
    ob = O.OracleBasis(wl)
    pat = ob.pattern()
    nf = wl.nf_of_atom
    blk = _blocks(pat)
    for anti in (False, True):
        G = fill_pattern(pat.blk_ptr, pat.blk_col, pat.blk_off, nf, 5, "GV", anti, blk_T=pat.blk_T)
        for (A, B, T), q in blk.items():
            qt = blk[(B, A, tuple(-t for t in T))]
            X, Y = _block(G, pat, q, nf[A], nf[B]), _block(G, pat, qt, nf[B], nf[A]).T
            assert np.array_equal(X, -Y if anti else Y)


def test_kfold_equals_bloch_sum_matrix_elements(cell_case):
    """H(k)_ij = sum_T exp(2 pi i k.T) H(T)_ij must equal the matrix element
    between Bloch sums, sum_p w_p v_p conj(chi_i(p)) chi_j(p) with
    chi_i(p) = sum_T exp(2 pi i k.T) phi_i(p - T.L), evaluated directly from
    the basis at the grid points (Eqs. 24-26); this fixes the sign of the
    phase and of T."""
    wl, xyz, w, ids, ob, pat, v, mats = cell_case
    L = np.asarray(wl.lattice)
    ks = np.array([[0.0, 0.0, 0.0], [0.25, 0.1, -0.3], [0.5, 0.5, 0.5]])
    s = wl.n_shell
    Ts = np.array([(a, b, c) for a in range(-s, s + 1) for b in range(-s, s + 1) for c in range(-s, s + 1)])
    phi_T = [ob.eval(xyz - T @ L)[0] for T in Ts]  # (n_fn, n_pts) per shift
    kptr, kcol, koff = ob.kpattern(pat)
    nf = wl.nf_of_atom
    first = np.concatenate([[0], np.cumsum(nf)])
    Hk = ob.kfold(mats[0], ks, pat)
    for ik, k in enumerate(ks):
        ph = np.exp(2j * np.pi * (Ts @ k))
        chi = sum(p * f for p, f in zip(ph, phi_T))
        direct = (np.conj(chi) * (w * v)) @ chi.T
        dense = np.zeros_like(direct)
        for A in range(wl.n_atoms):
            for r in range(int(kptr[A]), int(kptr[A + 1])):
                B = int(kcol[r])
                o = int(koff[r])
                dense[first[A]:first[A + 1], first[B]:first[B + 1]] = Hk[ik, o:o + nf[A] * nf[B]].reshape(nf[A], nf[B])
        assert np.abs(dense - direct).max() <= 1e-12 * np.abs(direct).max(), ik
        assert np.abs(dense - dense.conj().T).max() <= 1e-13 * np.abs(dense).max()  # Hermitian
