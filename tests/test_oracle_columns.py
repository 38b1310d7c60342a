"""Pins of the oracle's per-column operator (Eq. 19, large component in the
scalar form: F_ij = sum_p w phi_i (eps_j - V_j + v) phi_j), by reduction to
the already pinned integrals: with eps = V = 0 it is V(v); with v = V = 0 it is
eps_j S_ij, eps taken from the COLUMN's radial function (a transposed index
fails); a constant V_j = c_j shifts it by -c_j S_ij (the sign of V); and for
one atom with the potential -Z erf(a r)/r it equals -V(v = that potential at
the points) to the accuracy of the potential's spline.  CPU only."""
import math

import numpy as np
import pytest
from scipy.special import erf

import oracle as O
from workloads import column_operator, potential, single_atom, water


@pytest.fixture(scope="module")
def wcase():
    wl = water()
    xyz, w, _ = O.grid(wl)
    ob = O.OracleBasis(wl)
    pat = ob.pattern()
    v = potential(xyz, wl)
    V = ob.matrix_blocks(xyz, w, v, pat)[0]
    S = ob.matrix_blocks(xyz, w, np.ones(len(w)), pat)[0]
    eps, knots = column_operator(wl, 5)
    return wl, xyz, w, ob, pat, v, V, S, eps, knots


def test_reduces_to_the_potential_matrix(wcase):
    wl, xyz, w, ob, pat, v, V, S, eps, knots = wcase
    F = ob.matrix_columns(xyz, w, v, 0 * eps, 0 * knots, pat)
    assert np.abs(F - V).max() <= 1e-14 * np.abs(V).max()


def test_eigenvalue_multiplies_the_overlap_by_column(wcase):
    wl, xyz, w, ob, pat, v, V, S, eps, knots = wcase
    F = ob.dense(ob.matrix_columns(xyz, w, 0 * v, eps, 0 * knots, pat), pat)
    Sd = ob.dense(S, pat)
    ref = Sd * eps[ob.fn_rad][None, :]
    assert np.abs(F - ref).max() <= 1e-14 * np.abs(ref).max()
    wrong = Sd * eps[ob.fn_rad][:, None]  # the row's eigenvalue instead
    assert np.abs(F - wrong).max() > 1e-3 * np.abs(ref).max()


def test_constant_potential_shifts_by_minus_overlap(wcase):
    wl, xyz, w, ob, pat, v, V, S, eps, knots = wcase
    c = np.linspace(-2.0, 1.0, len(eps))
    F = ob.dense(ob.matrix_columns(xyz, w, v, eps, np.repeat(c[:, None], knots.shape[1], 1), pat), pat)
    ref = ob.dense(V, pat) + ob.dense(S, pat) * (eps - c)[ob.fn_rad][None, :]
    assert np.abs(F - ref).max() <= 1e-13 * np.abs(ref).max()


def test_one_atom_potential_against_points():
    Z, a = 3.0, 1.1
    wl = single_atom([0, 1, 2], [1.4, 1.6, 1.9], Z=Z, n_rad=80)
    xyz, w, _ = O.grid(wl)
    ob = O.OracleBasis(wl)
    pat = ob.pattern()
    r_k = wl.r_min * (wl.r_c / wl.r_min) ** (np.arange(wl.n_log) / (wl.n_log - 1))

    def pot(r):
        x = a * r
        return -Z * a * np.where(x > 1e-8, erf(x) / np.maximum(x, 1e-300), 2 / math.sqrt(math.pi))
    knots = np.repeat(pot(r_k)[None, :], 3, 0)
    F = ob.matrix_columns(xyz, w, np.zeros(len(w)), np.zeros(3), knots, pat)
    ref = -ob.matrix_blocks(xyz, w, pot(np.linalg.norm(xyz, axis=1)), pat)[0]
    # spline interpolation of the potential on 200 log knots: ~1e-8 relative
    assert np.abs(F - ref).max() <= 1e-6 * np.abs(ref).max()
    # same atom, same potential for every radial: symmetric
    Fd = ob.dense(F, pat)
    assert np.abs(Fd - Fd.T).max() <= 1e-13 * np.abs(Fd).max()
