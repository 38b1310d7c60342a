"""GPU parity of the periodic path (real-space H(T) blocks, Eqs. 24-25)
against the oracle on a small orthorhombic cell whose image shell covers
r_nb + r_c: pattern with shifts bit-exact, active centres exact, matrices,
density and adjoint within 1e-12 (FP64) and 1e-9 (split) relative."""
import numpy as np
import pytest

import oracle as O
import paper_2608_00773_gb300 as q
from gpu_helpers import LibCase, OracleCase, point_map, rel_fro
from workloads import periodic_cell

pytestmark = pytest.mark.gpu
NAMES = ["V", "W0", "SOx", "SOy", "SOz"]
TOL = {"fp64": 1e-12, "split": 1e-9}


@pytest.fixture(scope="module")
def cell():
    from paper_2608_00773_gb300 import _build
    _build.build()
    O.build()
    wl = periodic_cell()
    return LibCase(wl), OracleCase(wl)


def test_pattern_with_shifts_bit_exact(cell):
    lib, orc = cell
    for k in ("blk_ptr", "blk_col", "blk_off"):
        assert np.array_equal(lib.ex[k], getattr(orc.pat, k)), k
    assert np.array_equal(lib.ex["blk_T"], orc.pat.blk_T)
    assert (orc.pat.blk_T != 0).any(axis=1).sum() > 0


def test_grid_and_active_centres(cell):
    lib, orc = cell
    ex, wl = lib.ex, lib.wl
    li, oi = point_map(ex["point_id"], orc.ids)
    assert len(li) >= len(orc.ids) - 2 and len(li) >= len(ex["point_id"]) - 2
    assert np.abs(ex["xyz"][li] - orc.xyz[oi]).max() < 1e-13
    assert np.all(np.abs(ex["w"][li] - orc.w[oi]) <= 1e-12 * orc.w[oi] + 1e-15 * orc.w.max())
    # centres c = cell * n_atoms + A, cells lexicographic in T in [-s, s]^3
    s, n = wl.n_shell, wl.n_atoms
    side = 2 * s + 1
    T = np.array([(c // (side * side) - s, (c // side) % side - s, c % side - s) for c in range(side ** 3)])
    cen = (wl.xyz[None, :, :] + (T @ np.asarray(wl.lattice))[:, None, :]).reshape(-1, 3)
    bp = ex["batch_ptr"]
    for b in range(len(bp) - 1):
        P = ex["xyz"][bp[b]:bp[b + 1]]
        d = np.sqrt(((P[:, None, :] - cen[None]) ** 2).sum(-1))
        ref = np.where((d < wl.r_c).any(axis=0))[0]
        got = ex["batch_atoms"][ex["batch_atom_ptr"][b]:ex["batch_atom_ptr"][b + 1]]
        assert np.array_equal(got, ref)
    assert ex["batch_atoms"].max() >= n  # images take part


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_integrate_matches_oracle(prec, cell):
    lib, orc = cell
    got = lib.integrate(prec, spinor=True)
    lib.grid.status()
    errs = {nm: rel_fro(g, r) for nm, g, r in zip(NAMES, got[:5], orc.mats)}
    assert max(errs.values()) <= TOL[prec], errs
    ref = orc.ob.spinor_ss(*orc.mats[1:], orc.pat)
    assert np.linalg.norm(got[5].view(np.complex128) - ref) <= TOL[prec] * np.linalg.norm(ref)


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_density_and_adjoint_match_oracle(prec, cell):
    lib, orc = cell
    li, oi = point_map(lib.ex["point_id"], orc.ids)
    n = q.q4c_density(lib.tables, lib.grid, lib.random(71, "P"), prec).cpu().numpy()
    nref = orc.ob.density(orc.xyz, orc.random(71, "P"), orc.pat)
    assert rel_fro(n[li], nref[oi]) <= TOL[prec]
    g = q.q4c_integrate_backward(lib.tables, lib.grid, lib.G(72), prec).cpu().numpy()
    gref = orc.ob.adjoint(orc.xyz, orc.w, orc.G(72), orc.pat)
    lib.grid.status()
    assert rel_fro(g[li], gref[oi]) <= TOL[prec]
