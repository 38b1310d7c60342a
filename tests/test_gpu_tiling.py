"""The split path's tile shapes (one or two 16-point K-steps per pipeline
stage, chosen per batch-size bucket) and the tuner that chooses them:
results must not depend on the shape (parity with the oracle and with the
other shape under every candidate), and the tuner must time every bucket
the grid uses and keep the faster shape."""
import numpy as np
import pytest

import oracle as O
import paper_2608_00773_gb300 as q
from gpu_helpers import LibCase, OracleCase, point_map, rel_fro
from workloads import cluster64, column_operator, periodic_cell, small_cluster, water

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cases():
    from paper_2608_00773_gb300 import _build
    _build.build()
    O.build()
    return {name: (LibCase(wl), OracleCase(wl))
            for name, wl in (("water", water()), ("cluster", small_cluster(12, seed=9)), ("cell", periodic_cell()))}


def _set_all(grid, ks):
    for k in range(q.binding.TILE_BUCKETS + 1):  # the products buckets and the density/adjoint kernel
        q.q4c_grid_set_tiling(grid, k, ks)


@pytest.mark.parametrize("name", ["water", "cluster", "cell"])
def test_every_shape_matches_oracle_and_each_other(name, cases):
    lib, orc = cases[name]
    outs = {}
    li, oi = point_map(lib.ex["point_id"], orc.ids)
    n_ref = orc.ob.density(orc.xyz, orc.random(61, "P"), orc.pat)
    g_ref = orc.ob.adjoint(orc.xyz, orc.w, orc.G(62), orc.pat)
    for ks in (1, 2):
        _set_all(lib.grid, ks)
        outs[ks] = lib.integrate("split", spinor=True)
        n = q.q4c_density(lib.tables, lib.grid, lib.random(61, "P"), "split").cpu().numpy()
        g = q.q4c_integrate_backward(lib.tables, lib.grid, lib.G(62), "split").cpu().numpy()
        lib.grid.status()
        for m, r in zip(outs[ks][:5], orc.mats):
            assert rel_fro(m, r) <= 1e-9
        assert rel_fro(n[li], n_ref[oi]) <= 1e-9
        assert rel_fro(g[li], g_ref[oi]) <= 1e-9
        outs[ks] = outs[ks] + [n, g]
    _set_all(lib.grid, 1)
    for a, b in zip(outs[1], outs[2]):
        assert rel_fro(b, a) <= 1e-13


def test_shapes_in_the_column_operator_and_the_one_pass_call(cases):
    import torch
    lib, orc = cases["cluster"]
    eps, knots = column_operator(lib.wl, 1201)
    q.q4c_tables_set_columns(lib.tables, eps, knots)
    F64 = q.q4c_integrate_columns(lib.tables, lib.grid, lib.v, "fp64").cpu().numpy()
    P, G = lib.G(71), lib.G(72)
    ref = None
    for ks in (1, 2):
        _set_all(lib.grid, ks)
        Fs = q.q4c_integrate_columns(lib.tables, lib.grid, lib.v, "split").cpu().numpy()
        H, n, g = q.q4c_scf_pass(lib.tables, lib.grid, lib.v, P, G, "split")
        torch.cuda.synchronize()
        lib.grid.status()
        assert rel_fro(Fs, F64) <= 1e-9
        for m, r in zip(H[:5], orc.mats):
            assert rel_fro(m.cpu().numpy(), r) <= 1e-9
        if ref is None:
            ref = (n.clone(), g.clone())
        else:
            assert float(torch.linalg.norm(n - ref[0]) / torch.linalg.norm(ref[0])) <= 1e-13
    _set_all(lib.grid, 1)


def test_set_tiling_rejects_bad_arguments(cases):
    lib, _ = cases["water"]
    for bucket, ks in ((-1, 1), (5, 1), (0, 3), (4, 0)):
        with pytest.raises(q.Q4CError) as e:
            q.q4c_grid_set_tiling(lib.grid, bucket, ks)
        assert e.value.status == 1


def test_autotune_times_every_used_bucket_and_keeps_the_faster():
    """The 64-atom workload has batches in every bucket; after tuning, each
    used bucket has both timings and its shape is the faster one, and the
    matrices equal those of the untuned grid."""
    import torch
    wl = cluster64()
    lib = LibCase(wl)
    before = q.q4c_integrate(lib.tables, lib.grid, lib.v, "split")
    tiling = q.q4c_autotune(lib.tables, lib.grid, lib.v)
    after = q.q4c_integrate(lib.tables, lib.grid, lib.v, "split")
    torch.cuda.synchronize()
    lib.grid.status()
    used = [t for t in tiling if t["batches"] > 0]
    assert len(used) >= 4 and tiling[-1]["batches"] == lib.grid.info.n_batches  # the last: density/adjoint
    for t in used:
        assert t["ms_one"] > 0 and t["ms_two"] > 0
        assert t["k_steps"] == (2 if t["ms_two"] < t["ms_one"] else 1)
    assert sum(t["batches"] for t in tiling[:-1]) == lib.grid.info.n_batches
    for a, b in zip(after[:5], before[:5]):
        assert float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) <= 1e-13
