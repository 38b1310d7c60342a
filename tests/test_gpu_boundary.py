"""Points within FP32 rounding of a cutoff sphere (|p - R_A| = r_c): the
tabulated radial functions vanish at r_c but their gradients do not, so the
split path must put such a point on the same side of the sphere as the FP64
path and the oracle, or W0 and SO (built from the gradients, Eq. 29) lose
that point's term.  The workload is a molecule of the batched set that has a
grid point at r_c (1 - 2e-8) from one of its atoms; the potential is kept only
at the points near some cutoff sphere, so every matrix is made of those
points alone, and a wrong decision shows at full size."""
import numpy as np
import pytest

import oracle as O
import paper_2608_00773_gb300 as q
from gpu_helpers import point_map, rel_fro
from workloads import molecule_batch, potential

pytestmark = pytest.mark.gpu
NAMES = ["V", "W0", "SOx", "SOy", "SOz"]


def _near_cutoff(xyz, centres, r_c, rel=1e-6):
    """Points whose squared distance to some centre is within rel of r_c^2."""
    d2 = ((xyz[:, None, :] - centres[None, :, :]) ** 2).sum(axis=2)
    return np.any(np.abs(d2 / (r_c * r_c) - 1.0) < rel, axis=1)


@pytest.fixture(scope="module")
def case():
    from paper_2608_00773_gb300 import _build
    _build.build()
    O.build()
    return molecule_batch(200).molecule(74)


def test_points_on_the_cutoff_sphere(case):
    import torch
    wl = case
    tables, grid = q.setup(wl)
    ex = grid.export()
    near = _near_cutoff(ex["xyz"], wl.xyz, wl.r_c)
    assert near.sum() >= 1  # the workload does hold such a point
    v = torch.tensor(potential(ex["xyz"], wl) * near, device="cuda")
    split = [o.cpu().numpy() for o in q.q4c_integrate(tables, grid, v, "split")[:5]]
    fp64 = [o.cpu().numpy() for o in q.q4c_integrate(tables, grid, v, "fp64")[:5]]
    grid.status()
    for n, a, b in zip(NAMES, split, fp64):
        assert np.linalg.norm(b) > 0, n
        assert rel_fro(a, b) <= 1e-9, (n, rel_fro(a, b))
    # the oracle on its own grid, v kept at the same raw points
    xyz, w, ids = O.grid(wl)
    ob = O.OracleBasis(wl)
    pat = ob.pattern()
    keep = np.isin(ids, ex["point_id"][near])
    assert keep.sum() == near.sum()
    ref = ob.matrix_blocks(xyz[keep], w[keep], potential(xyz[keep], wl), pat)
    for n, a, r in zip(NAMES, split, ref):
        assert rel_fro(a, r) <= 1e-9, (n, rel_fro(a, r))
    # the two grids differ only at points whose partition weight is rounding
    # (a cell function 1 - f with f within an ulp of 1): below 1e-15 of the largest
    li, oi = point_map(ex["point_id"], ids)
    lib_only = np.setdiff1d(np.arange(len(ex["w"])), li)
    orc_only = np.setdiff1d(np.arange(len(w)), oi)
    assert np.all(ex["w"][lib_only] <= 1e-15 * w.max()) and np.all(w[orc_only] <= 1e-15 * w.max())
