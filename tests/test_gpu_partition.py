"""GPU parity with the Stratmann partition (Stratmann, Scuseria and Frisch
1996): the library's grid weights against the oracle's point by point
(1e-12), and the integrals on that grid (FP64 within 1e-12, split within
1e-9 relative Frobenius per matrix)."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from gpu_helpers import LibCase, OracleCase, point_map, rel_fro
from workloads import small_cluster, water

pytestmark = pytest.mark.gpu
NAMES = ["V", "W0", "SOx", "SOy", "SOz"]


@pytest.fixture(scope="module", params=["water", "cluster"])
def case(request):
    from paper_2608_00773_gb300 import _build
    _build.build()
    O.build()
    wl = water() if request.param == "water" else small_cluster(8, seed=7)
    wl = dataclasses.replace(wl, partition="stratmann")
    return LibCase(wl), OracleCase(wl)


def test_stratmann_weights_match_oracle(case):
    lib, orc = case
    ex = lib.ex
    li, oi = point_map(ex["point_id"], orc.ids)
    assert len(li) >= len(orc.ids) - 2 and len(li) >= len(ex["point_id"]) - 2
    assert np.all(np.abs(ex["w"][li] - orc.w[oi]) <= 1e-12 * orc.w[oi] + 1e-15 * orc.w.max())
    # a different partition from Becke's on the same raw grid
    wb = O.grid(dataclasses.replace(lib.wl, partition="becke"))
    common, a, b = np.intersect1d(orc.ids, wb[2], return_indices=True)
    assert np.abs(orc.w[a] - wb[1][b]).max() > 1e-6 * orc.w.max()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("split", 1e-9)])
def test_integrals_on_stratmann_grid(case, prec, tol):
    lib, orc = case
    got = lib.integrate(prec)
    lib.grid.status()
    errs = {nm: rel_fro(g, r) for nm, g, r in zip(NAMES, got[:5], orc.mats)}
    assert max(errs.values()) <= tol, errs
