"""GPU parity of the k-phase fold H(k)_AB = sum_T exp(2 pi i k.T) H(T)_AB
(Eqs. 24-26) against the oracle: the k-pattern bit-exact, H(k) within
1e-13 relative on seeded pattern values and on the integrated V, and
H(k) = H exactly for a molecule (only T = 0)."""
import numpy as np
import pytest

import oracle as O
import paper_2608_00773_gb300 as q
from gpu_helpers import LibCase, OracleCase, rel_fro
from workloads import periodic_cell, water

pytestmark = pytest.mark.gpu
KS = np.array([[0.0, 0.0, 0.0], [0.25, 0.1, -0.3], [0.5, 0.5, 0.5], [-0.5, 0.0, 0.125], [0.37, -0.41, 0.05]])


@pytest.fixture(scope="module")
def cell():
    from paper_2608_00773_gb300 import _build
    _build.build()
    O.build()
    wl = periodic_cell()
    return LibCase(wl), OracleCase(wl)


def test_kpattern_bit_exact(cell):
    lib, orc = cell
    ptr, col, off = lib.grid.kpattern()
    rptr, rcol, roff = orc.ob.kpattern(orc.pat)
    assert np.array_equal(ptr, rptr) and np.array_equal(col, rcol) and np.array_equal(off, roff)
    assert len(col) < len(lib.ex["blk_col"])  # several shifts fold onto one pair


def test_kfold_of_pattern_values(cell):
    lib, orc = cell
    H = lib.random(81, "P")
    got = q.q4c_kfold(lib.grid, H, KS).cpu().numpy()
    ref = orc.ob.kfold(orc.random(81, "P"), KS, orc.pat)
    assert got.shape == ref.shape
    for ik in range(len(KS)):
        assert np.linalg.norm(got[ik] - ref[ik]) <= 1e-13 * np.linalg.norm(ref[ik]), ik


def test_kfold_of_integrated_matrix(cell):
    lib, orc = cell
    V = lib.integrate("fp64")[0]
    import torch
    got = q.q4c_kfold(lib.grid, torch.as_tensor(V, device="cuda"), KS).cpu().numpy()
    ref = orc.ob.kfold(orc.mats[0], KS, orc.pat)
    assert rel_fro(got.view(np.float64), ref.view(np.float64)) <= 1e-12


def test_kfold_zero_kpoints(cell):
    lib, _ = cell
    out = q.q4c_kfold(lib.grid, lib.random(82, "P"), np.zeros((0, 3)))
    assert out.shape[0] == 0


def test_molecule_kfold_is_identity():
    lib = LibCase(water())
    ptr, col, off = lib.grid.kpattern()
    assert np.array_equal(ptr, lib.ex["blk_ptr"]) and np.array_equal(col, lib.ex["blk_col"])
    assert np.array_equal(off, lib.ex["blk_off"])
    H = lib.random(83, "P")
    got = q.q4c_kfold(lib.grid, H, KS[1:3]).cpu().numpy()
    for ik in range(2):
        assert np.array_equal(got[ik].real, H.cpu().numpy()) and not got[ik].imag.any()
