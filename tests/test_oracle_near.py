"""Pins of the oracle's restricted routines, which the large workloads need
(a full grid or full matrices of the 3,383-atom cell are out of the
oracle's reach): grid_near must return exactly the points of the full grid
that lie within r_c of its targets, with bit-identical weights, and
matrix_entries must return exactly what the full block matrices hold at the
listed elements, images included (Eqs. 24-25, 29-30), also when it sums
over the near points alone.  CPU only.
"""
import numpy as np
import pytest

import oracle as O
from workloads import periodic_cell, potential, small_cluster, water

NAMES = ["V", "W0", "SOx", "SOy", "SOz"]


@pytest.fixture(scope="module", params=["cell", "cluster"])
def case(request):
    O.build()
    wl = periodic_cell() if request.param == "cell" else small_cluster(6, seed=3, n_rad=14, n_theta=6, n_phi=10)
    xyz, w, ids = O.grid(wl)
    ob = O.OracleBasis(wl)
    pat = ob.pattern()
    return wl, xyz, w, ids, ob, pat


def _near_mask(xyz, targets, r_c):
    d = np.sqrt(((xyz[:, None, :] - targets[None, :, :]) ** 2).sum(-1))
    return (d < r_c).any(axis=1)


def test_grid_near_is_the_full_grid_restricted(case):
    wl, xyz, w, ids, _, _ = case
    cen = O.centres(wl)
    rng = np.random.default_rng(5)
    for targets in (cen[[wl.n_atoms * (len(cen) // wl.n_atoms // 2)]],  # atom 0 in cell 0
                    cen[rng.choice(len(cen), 3, replace=False)],          # any three centres
                    cen[np.arange(0, len(cen), wl.n_atoms)]):              # every image of atom 0
        nx, nw, nid = O.grid_near(wl, targets)
        keep = _near_mask(xyz, targets, wl.r_c)
        assert len(nid) == keep.sum() and len(nid) > 0
        assert np.array_equal(nid, ids[keep])
        assert np.array_equal(nx, xyz[keep]) and np.array_equal(nw, w[keep])  # bit for bit


def test_grid_near_of_a_far_target_is_empty(case):
    wl = case[0]
    far = O.centres(wl).max(axis=0) + 10.0 * (wl.r_c + wl.r_nb)
    nx, nw, nid = O.grid_near(wl, far[None, :])
    assert len(nid) == 0


def _elements(pat, wl, n, rng):
    """n random elements (A, B, T, i, j) of the pattern and their value offsets"""
    nf = wl.nf_of_atom
    rows = np.repeat(np.arange(wl.n_atoms), np.diff(pat.blk_ptr))
    A, B, T, i, j, off = [], [], [], [], [], []
    for q in rng.choice(len(pat.blk_col), n):
        a, b = int(rows[q]), int(pat.blk_col[q])
        ii, jj = int(rng.integers(nf[a])), int(rng.integers(nf[b]))
        A.append(a); B.append(b); T.append(pat.blk_T[q]); i.append(ii); j.append(jj)
        off.append(int(pat.blk_off[q]) + ii * int(nf[b]) + jj)
    return np.array(A), np.array(B), np.array(T), np.array(i), np.array(j), np.array(off)


def test_matrix_entries_equal_the_full_blocks(case):
    wl, xyz, w, ids, ob, pat = case
    v = potential(xyz, wl)
    full = ob.matrix_blocks(xyz, w, v, pat)
    rng = np.random.default_rng(6)
    A, B, T, i, j, off = _elements(pat, wl, 300, rng)
    if wl.lattice is not None:
        assert (np.abs(T).sum(axis=1) > 0).sum() >= 50  # images across the cell faces among them
    got = ob.matrix_entries(xyz, w, v, A, B, T, i, j)
    for n, g, f in zip(NAMES, got, full):
        assert np.array_equal(g, f[off]), n


def test_matrix_entries_on_the_near_points(case):
    """Block (A, B, T) gathers only points within r_c of an image of A, so
    the elements of row A summed over grid_near(images of A) equal the full
    matrices' (the Neumaier sums see the same nonzero terms in the same order)."""
    wl, xyz, w, ids, ob, pat = case
    v = potential(xyz, wl)
    full = ob.matrix_blocks(xyz, w, v, pat)
    rng = np.random.default_rng(7)
    A, B, T, i, j, off = _elements(pat, wl, 400, rng)
    a0 = int(A[0])
    sel = A == a0
    cen = O.centres(wl)
    nx, nw, nid = O.grid_near(wl, cen[np.arange(a0, len(cen), wl.n_atoms)])
    got = ob.matrix_entries(nx, nw, potential(nx, wl), A[sel], B[sel], T[sel], i[sel], j[sel])
    for n, g, f in zip(NAMES, got, full):
        assert np.allclose(g, f[off[sel]], rtol=1e-15, atol=1e-15 * np.abs(f).max()), n
