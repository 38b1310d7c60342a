"""GPU parity of batched molecules: many independent molecules in one grid
and one call.  Each molecule's rows of the pattern must hold exactly what
integrating that molecule alone gives; the oracle computes every checked
molecule on its own (its own grid, pattern and v)."""
import numpy as np
import pytest

import oracle as O
import paper_2608_00773_gb300 as q
from gpu_helpers import rel_fro
from workloads import molecule_batch, molecule_potential, potential

pytestmark = pytest.mark.gpu
NAMES = ["V", "W0", "SOx", "SOy", "SOz"]
TOL = {"fp64": 1e-12, "split": 1e-9}


def _lib(wl):
    import time
    import torch
    t0 = time.time()
    tables, grid = q.setup(wl)
    t1 = time.time()
    ex = grid.export()
    ppa = wl.n_rad * wl.n_theta * wl.n_phi
    v = torch.tensor(molecule_potential(ex["xyz"], ex["point_id"] // ppa, wl, device="cuda"), device="cuda")
    print(f"grid {t1 - t0:.1f} s, export + v {time.time() - t1:.1f} s")
    return tables, grid, ex, v


def _mol_slice(ex, wl, m):
    a0, a1 = int(wl.mol_atom_ptr[m]), int(wl.mol_atom_ptr[m + 1])
    q0, q1 = int(ex["blk_ptr"][a0]), int(ex["blk_ptr"][a1])
    return a0, a1, q0, q1, int(ex["blk_off"][q0]), int(ex["blk_off"][q1])


def _check_molecules(wl, ex, outs, mols, tol):
    for m in mols:
        a0, a1, q0, q1, o0, o1 = _mol_slice(ex, wl, m)
        wm = wl.molecule(m)
        xyz, w, _ = O.grid(wm)
        ob = O.OracleBasis(wm)
        pat = ob.pattern()
        # the molecule's pattern rows are its own pattern, shifted
        assert np.array_equal(ex["blk_col"][q0:q1] - a0, pat.blk_col)
        assert np.array_equal(ex["blk_off"][q0:q1 + 1] - o0, pat.blk_off)
        ref = ob.matrix_blocks(xyz, w, potential(xyz, wm), pat)
        errs = {n: rel_fro(o[o0:o1], r) for n, o, r in zip(NAMES, outs, ref)}
        assert max(errs.values()) <= tol, (m, errs)


@pytest.fixture(scope="module")
def small():
    from paper_2608_00773_gb300 import _build
    _build.build()
    O.build()
    wl = molecule_batch(12, seed=1003, n_max=12, n_rad=20, n_theta=6, n_phi=12, batch_max=64)
    return wl, _lib(wl)


def test_batches_hold_one_molecule(small):
    wl, (tables, grid, ex, v) = small
    ppa = wl.n_rad * wl.n_theta * wl.n_phi
    mol_of_atom = np.repeat(np.arange(wl.n_molecules), np.diff(wl.mol_atom_ptr))
    bp = ex["batch_ptr"]
    for b in range(len(bp) - 1):
        mols = np.unique(mol_of_atom[ex["point_id"][bp[b]:bp[b + 1]] // ppa])
        assert len(mols) == 1
        act = ex["batch_atoms"][ex["batch_atom_ptr"][b]:ex["batch_atom_ptr"][b + 1]]
        assert np.all(mol_of_atom[act] == mols[0])
    # no block couples two molecules
    rows = np.repeat(np.arange(wl.n_atoms), np.diff(ex["blk_ptr"]))
    assert np.array_equal(mol_of_atom[rows], mol_of_atom[ex["blk_col"]])


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_each_molecule_matches_its_own_oracle(prec, small):
    wl, (tables, grid, ex, v) = small
    outs = [o.cpu().numpy() for o in q.q4c_integrate(tables, grid, v, prec)[:5]]
    grid.status()
    _check_molecules(wl, ex, outs, range(wl.n_molecules), TOL[prec])


def test_two_thousand_molecules_sampled():
    """The batched-molecule configuration at full size (2,000 molecules of
    3-40 atoms, 40 x 200 points per atom, one grid, one split call): every
    molecule's blocks against the FP64 path (the largest relative error over
    the molecules, per matrix), and 20 molecules spread over the sizes, the
    three largest among them, each against its own oracle."""
    import time
    from concurrent.futures import ThreadPoolExecutor
    t0 = time.time()
    wl = molecule_batch()
    tables, grid, ex, v = _lib(wl)
    t1 = time.time()
    split = [o.cpu().numpy() for o in q.q4c_integrate(tables, grid, v, "split")[:5]]
    fp64 = [o.cpu().numpy() for o in q.q4c_integrate(tables, grid, v, "fp64")[:5]]
    grid.status()
    print(f"setup + v {t1 - t0:.1f} s, integrate (both paths) {time.time() - t1:.1f} s, points {grid.n_points}, "
          f"batches {grid.info.n_batches}, basis {grid.info.n_basis}")
    worst = {}
    for n, a, b in zip(NAMES, split, fp64):
        worst[n] = max(rel_fro(a[o0:o1], b[o0:o1])
                       for o0, o1 in ((_mol_slice(ex, wl, m)[4], _mol_slice(ex, wl, m)[5])
                                      for m in range(wl.n_molecules)))
    print("worst molecule, split vs FP64:", worst)
    assert max(worst.values()) <= 1e-12
    sizes = np.diff(wl.mol_atom_ptr)
    order = np.argsort(sizes, kind="stable")
    pick = list(order[np.linspace(0, len(order) - 4, 17).astype(int)]) + list(order[-3:])
    mols = sorted(set(int(m) for m in pick))
    assert len(mols) >= 20 and sizes[mols].max() == sizes.max() and sizes[mols].min() == sizes.min()
    with ThreadPoolExecutor(max_workers=8) as pool:  # the oracle's C calls release the GIL
        list(pool.map(lambda m: _check_molecules(wl, ex, split, [m], TOL["split"]), mols))
