"""GPU parity of the one-pass SCF call (q4c_scf_pass): the integration of v,
the density of P (with the gradient terms when P carries the W0/SO slots, the
plain density of Eq. 39 with the V slot alone) and the adjoint of G from one
basis evaluation per wave, against the oracle on a molecule, a heavy/light
cluster and a periodic cell, against the separate calls on the full-size
64-atom workload (where the oracle checks sampled points), and with one
basis-tile launch per wave instead of one per call."""
import numpy as np
import pytest

import oracle as O
import paper_2608_00773_gb300 as q
from gpu_helpers import LibCase, OracleCase, point_map, rel_fro
from workloads import cluster64, periodic_cell, small_cluster, water

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-12, "split": 1e-9}


@pytest.fixture(scope="module")
def cases():
    from paper_2608_00773_gb300 import _build
    _build.build()
    O.build()
    return {name: (LibCase(wl), OracleCase(wl))
            for name, wl in (("water", water()), ("cluster", small_cluster(8, seed=7)), ("cell", periodic_cell()))}


@pytest.mark.parametrize("prec", ["fp64", "split"])
@pytest.mark.parametrize("name", ["water", "cluster", "cell"])
def test_scf_pass_matches_oracle(name, prec, cases):
    lib, orc = cases[name]
    P, G = lib.G(91), lib.G(92)
    H, n, g = q.q4c_scf_pass(lib.tables, lib.grid, lib.v, P, G, prec)
    lib.grid.status()
    for m, r in zip(H[:5], orc.mats):
        assert rel_fro(m.cpu().numpy(), r) <= TOL[prec]
    li, oi = point_map(lib.ex["point_id"], orc.ids)
    n_ref = orc.ob.density_full(orc.xyz, orc.G(91), orc.pat)
    g_ref = orc.ob.adjoint(orc.xyz, orc.w, orc.G(92), orc.pat)
    assert rel_fro(n.cpu().numpy()[li], n_ref[oi]) <= TOL[prec]
    assert rel_fro(g.cpu().numpy()[li], g_ref[oi]) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_scf_pass_parts_and_plain_density(prec, cases):
    """Each part alone, and the V slot alone giving the density of Eq. 39."""
    lib, orc = cases["cluster"]
    Pv = lib.random(93, "P")
    _, n, _ = q.q4c_scf_pass(lib.tables, lib.grid, None, [Pv, None, None, None, None], None, prec)
    H, _, _ = q.q4c_scf_pass(lib.tables, lib.grid, lib.v, None, None, prec)
    _, _, g = q.q4c_scf_pass(lib.tables, lib.grid, None, None, lib.G(94), prec)
    lib.grid.status()
    li, oi = point_map(lib.ex["point_id"], orc.ids)
    n_ref = orc.ob.density(orc.xyz, orc.random(93, "P"), orc.pat)
    assert rel_fro(n.cpu().numpy()[li], n_ref[oi]) <= TOL[prec]
    for m, r in zip(H[:5], orc.mats):
        assert rel_fro(m.cpu().numpy(), r) <= TOL[prec]
    g_ref = orc.ob.adjoint(orc.xyz, orc.w, orc.G(94), orc.pat)
    assert rel_fro(g.cpu().numpy()[li], g_ref[oi]) <= TOL[prec]
    # all slots of G absent: the gradient is zero
    _, _, z = q.q4c_scf_pass(lib.tables, lib.grid, None, None, [None] * 5, prec)
    assert float(z.abs().max()) == 0.0


def test_scf_pass_full_size_equals_separate_calls_and_oracle_points():
    """The 64-atom workload (1.2M points): the fused pass against the separate
    calls on the split path, its density and adjoint against the oracle at
    200 points of the oracle's own grid, and one basis launch per wave."""
    import torch
    wl = cluster64()
    lib = LibCase(wl)
    P, G = lib.G(95), lib.G(96)
    q.profile(True)
    q.profile_read("")
    H, n, g = q.q4c_scf_pass(lib.tables, lib.grid, lib.v, P, G, "split")
    torch.cuda.synchronize()
    _, fused_basis = q.profile_read("basis_df")
    H_s = q.q4c_integrate(lib.tables, lib.grid, lib.v, "split")
    n_s = q.q4c_density_full(lib.tables, lib.grid, P, "split")
    g_s = q.q4c_integrate_backward(lib.tables, lib.grid, G, "split")
    torch.cuda.synchronize()
    _, sep_basis = q.profile_read("basis_df")
    q.profile(False)
    lib.grid.status()
    assert sep_basis == 3 * fused_basis and fused_basis >= 1
    for a, b in zip(H[:5], H_s[:5]):
        assert float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) <= 1e-13
    assert float(torch.linalg.norm(n - n_s) / torch.linalg.norm(n_s)) <= 1e-13
    assert float(torch.linalg.norm(g - g_s) / torch.linalg.norm(g_s)) <= 1e-13
    # sampled points of the oracle's own grid, matched by raw id
    xyz, w, ids = O.grid(wl, stride=7)
    ob = O.OracleBasis(wl)
    pat = ob.pattern()
    from workloads import ADJOINT_KINDS, fill_pattern
    Po = [fill_pattern(pat.blk_ptr, pat.blk_col, pat.blk_off, wl.nf_of_atom, 95, k, a) for k, a in ADJOINT_KINDS]
    Go = [fill_pattern(pat.blk_ptr, pat.blk_col, pat.blk_off, wl.nf_of_atom, 96, k, a) for k, a in ADJOINT_KINDS]
    pos = {int(p): k for k, p in enumerate(lib.ex["point_id"])}
    both = np.array([k for k, i in enumerate(ids) if int(i) in pos])
    sel = np.sort(np.random.default_rng(97).choice(both, 200, replace=False))
    li = np.array([pos[int(i)] for i in ids[sel]])
    n_ref = ob.density_full(xyz[sel], Po, pat)
    g_ref = ob.adjoint(xyz[sel], w[sel], Go, pat)
    assert rel_fro(n.cpu().numpy()[li], n_ref) <= 1e-9
    assert rel_fro(g.cpu().numpy()[li], g_ref) <= 1e-9
