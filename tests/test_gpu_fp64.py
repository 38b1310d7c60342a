"""GPU parity of the FP64 path against the CPU oracle (element by element).

Tolerance: 1e-12 relative Frobenius per matrix (FP64 path); indices, point
sets and the block pattern bit-exact.  Every input is seeded and synthetic.
"""
import math

import numpy as np
import pytest

import oracle as O
import paper_2608_00773_gb300 as q
from gpu_helpers import LibCase, OracleCase, point_map, rel_fro
from workloads import Species, Workload, potential, single_atom, small_cluster, water

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="session", autouse=True)
def _built():
    from paper_2608_00773_gb300 import _build
    _build.build()
    O.build()


@pytest.fixture(scope="module")
def water_pair():
    wl = water()
    return LibCase(wl), OracleCase(wl)


@pytest.fixture(scope="module")
def cluster_pair():
    wl = small_cluster(8, seed=7)
    return LibCase(wl), OracleCase(wl)


# ---------------------------------------------------------------- tables / basis


def test_tables_match_oracle_spline(water_pair):
    lib, orc = water_pair
    wl = lib.wl
    h = math.log(wl.r_c / wl.r_min) / (wl.n_log - 1)
    rng = np.random.default_rng(1)
    for k in range(len(wl.rad_l)):
        coef = lib.tables.coefficients(k)
        for r in np.exp(rng.uniform(math.log(wl.r_min), math.log(wl.r_c * 0.999), 40)):
            t = math.log(r / wl.r_min) / h
            j = min(int(t), wl.n_log - 2); s = t - j
            c = coef[j]
            u = c[0] + s * (c[1] + s * (c[2] + s * c[3]))
            ref, _ = O.spline_eval(int(wl.rad_l[k]), orc.ob.tab_u[k], orc.ob.tab_M[k], r, wl.r_min, wl.r_c)
            assert abs(u - ref) <= 1e-13 * np.abs(orc.ob.tab_u[k]).max()


@pytest.mark.parametrize("wlname", ["water", "cluster"])
def test_basis_values_match_oracle(wlname, water_pair, cluster_pair):
    import torch
    lib, orc = water_pair if wlname == "water" else cluster_pair
    wl = lib.wl
    rng = np.random.default_rng(2)
    pts = [wl.xyz[a] + rng.normal(scale=s, size=3) for a in range(wl.n_atoms) for s in (1e-6, 1e-4, 0.05, 0.7, 2.5)
           for _ in range(3)]
    pts += [wl.xyz[0].copy()]                                       # on a nucleus
    pts += [wl.xyz[0] + np.array([0, 0, wl.r_c * (1 - 1e-9)])]      # just inside r_c
    pts += [wl.xyz[0] + np.array([0, wl.r_c * 0.93, 0])]            # inside the cutoff ramp
    pts = np.array(pts)
    phi, grad = q.q4c_basis_eval(lib.tables, lib.grid, torch.tensor(pts, device="cuda"))
    rphi, rgrad = orc.ob.eval(pts)
    phi, grad = phi.cpu().numpy(), grad.cpu().numpy()
    scale_p = np.abs(rphi).max(axis=1, keepdims=True) + 1e-300
    # g'(r) = (u' - (l+1) u/r)/r^(l+1) cancels as r -> 0: two correct FP64
    # evaluation orders differ by ~eps |g|/r there, so the gradient bound
    # carries a 1/r term (r = distance to the function's own centre)
    fa = orc.ob.fn_atom
    r = np.linalg.norm(pts[None, :, :] - wl.xyz[fa][:, None, :], axis=2)[:, :, None]
    scale_g = np.abs(rgrad).max(axis=(1, 2), keepdims=True) + 1e-300
    bound_g = 1e-12 * scale_g + 1e-14 * np.abs(rphi)[:, :, None] / np.maximum(r, wl.r_min)
    ratio_p = (np.abs(phi - rphi) / scale_p).max()
    ratio_g = (np.abs(grad - rgrad) / bound_g).max()
    assert ratio_p <= 1e-12, ratio_p
    assert ratio_g <= 1.0, (ratio_g, np.unravel_index(np.argmax(np.abs(grad - rgrad) / bound_g), grad.shape))


# ---------------------------------------------------------------- grid


@pytest.mark.parametrize("wlname", ["water", "cluster"])
def test_grid_matches_oracle(wlname, water_pair, cluster_pair):
    lib, orc = water_pair if wlname == "water" else cluster_pair
    ex = lib.ex
    li, oi = point_map(ex["point_id"], orc.ids)
    only_lib = np.setdiff1d(ex["point_id"], orc.ids)
    only_orc = np.setdiff1d(orc.ids, ex["point_id"])
    # points kept by one side only carry negligible weight (w == 0 decided by rounding)
    wmax = orc.w.max()
    assert len(only_lib) + len(only_orc) <= 1e-4 * len(orc.ids) + 2
    if len(only_lib):
        assert ex["w"][np.isin(ex["point_id"], only_lib)].max() < 1e-13 * wmax
    if len(only_orc):
        assert orc.w[np.isin(orc.ids, only_orc)].max() < 1e-13 * wmax
    assert np.abs(ex["xyz"][li] - orc.xyz[oi]).max() < 1e-13
    assert np.all(np.abs(ex["w"][li] - orc.w[oi]) <= 1e-12 * orc.w[oi] + 1e-15 * wmax)


@pytest.mark.parametrize("wlname", ["water", "cluster"])
def test_pattern_bit_exact(wlname, water_pair, cluster_pair):
    lib, orc = water_pair if wlname == "water" else cluster_pair
    assert np.array_equal(lib.ex["blk_ptr"], orc.pat.blk_ptr)
    assert np.array_equal(lib.ex["blk_col"], orc.pat.blk_col)
    assert np.array_equal(lib.ex["blk_off"], orc.pat.blk_off)


@pytest.mark.parametrize("wlname", ["water", "cluster"])
def test_batch_invariants(wlname, water_pair, cluster_pair):
    """Batches partition the points (each point in exactly one batch), hold at
    most batch_max points, and list exactly the atoms with some point strictly
    inside r_c (the reduced index set nnz(B_v))."""
    lib, _ = water_pair if wlname == "water" else cluster_pair
    ex, wl = lib.ex, lib.wl
    bp = ex["batch_ptr"]
    assert bp[0] == 0 and bp[-1] == len(ex["w"]) and np.all(np.diff(bp) >= 1)
    assert np.diff(bp).max() <= wl.batch_max
    assert len(np.unique(ex["point_id"])) == len(ex["point_id"])
    for b in range(len(bp) - 1):
        P = ex["xyz"][bp[b]:bp[b + 1]]
        d = np.sqrt(((P[:, None, :] - wl.xyz[None]) ** 2).sum(-1))
        ref = np.where((d < wl.r_c).any(axis=0))[0]
        got = ex["batch_atoms"][ex["batch_atom_ptr"][b]:ex["batch_atom_ptr"][b + 1]]
        assert np.array_equal(got, ref)


# ---------------------------------------------------------------- integration


@pytest.mark.parametrize("wlname", ["water", "cluster"])
def test_integrate_fp64_matches_oracle(wlname, water_pair, cluster_pair):
    lib, orc = water_pair if wlname == "water" else cluster_pair
    got = lib.integrate("fp64", spinor=True)
    for name, g, r in zip(["V", "W0", "SOx", "SOy", "SOz"], got[:5], orc.mats):
        assert rel_fro(g, r) <= TOL, name
    # exact (anti)symmetry of the assembled matrices
    pat = orc.pat
    V, W0, SOx = (orc.ob.dense(m, pat) for m in (got[0], got[1], got[2]))
    assert np.array_equal(V, V.T) and np.array_equal(W0, W0.T) and np.array_equal(SOx, -SOx.T)
    # spinor SS blocks
    ref = orc.ob.spinor_ss(*orc.mats[1:], pat)
    ss = got[5].view(np.complex128)
    assert np.linalg.norm(ss - ref) <= TOL * np.linalg.norm(ref)


def test_integrate_fp64_edge_cases():
    # one atom with l = 0..3 (n_b = 16); two atoms beyond 2 r_c (diagonal blocks only);
    # batch_max = 1 (every point its own batch)
    wl1 = single_atom([0, 1, 2, 3], [0.8, 1.1, 1.6, 2.2], Z=6.0, n_rad=20, n_theta=6, n_phi=12)
    sp = [Species("A", 3.0, [0, 1], [0.9, 1.4]), Species("B", 1.0, [0, 2], [1.2, 0.7])]
    wl2 = Workload("far-pair", np.array([[0.0, 0, 0], [13.0, 0.5, -0.2]]), np.array([0, 1], np.int32), sp,
                   n_rad=16, n_theta=6, n_phi=12)
    wl3 = water(n_rad=8, n_theta=4, n_phi=8, batch_max=1)
    for wl in (wl1, wl2, wl3):
        lib, orc = LibCase(wl), OracleCase(wl)
        got = lib.integrate("fp64")
        for g, r in zip(got[:5], orc.mats):
            assert rel_fro(g, r) <= TOL
    assert lib.grid.info.max_np == 1


# ---------------------------------------------------------------- density / adjoint


@pytest.mark.parametrize("wlname", ["water", "cluster"])
def test_density_fp64_matches_oracle(wlname, water_pair, cluster_pair):
    lib, orc = water_pair if wlname == "water" else cluster_pair
    P = lib.random(55, "P")
    n = q.q4c_density(lib.tables, lib.grid, P, "fp64").cpu().numpy()
    nref = orc.ob.density(orc.xyz, orc.random(55, "P"), orc.pat)
    li, oi = point_map(lib.ex["point_id"], orc.ids)
    assert rel_fro(n[li], nref[oi]) <= TOL
    assert np.all(np.abs(n[li] - nref[oi]) <= 1e-11 * np.abs(nref).max())


@pytest.mark.parametrize("wlname", ["water", "cluster"])
def test_backward_fp64_matches_oracle(wlname, water_pair, cluster_pair):
    lib, orc = water_pair if wlname == "water" else cluster_pair
    g = q.q4c_integrate_backward(lib.tables, lib.grid, lib.G(66), "fp64").cpu().numpy()
    gref = orc.ob.adjoint(orc.xyz, orc.w, orc.G(66), orc.pat)
    li, oi = point_map(lib.ex["point_id"], orc.ids)
    assert rel_fro(g[li], gref[oi]) <= TOL
    # linearity: sum_p v_p dL/dv_p = L on the library's own outputs
    mats = lib.integrate("fp64")
    L = sum(float(np.dot(Gm.cpu().numpy(), M)) for Gm, M in zip(lib.G(66), mats[:5]))
    assert abs(np.dot(lib.v_host, g) - L) <= 1e-12 * abs(L) * 10


def test_autograd_matches_backward(water_pair):
    import torch
    lib, _ = water_pair
    v = lib.v.clone().requires_grad_(True)
    outs = q.integrate(v, lib.tables, lib.grid, "fp64")
    G = lib.G(3)
    L = sum((Gm * M).sum() for Gm, M in zip(G, outs))
    (gv,) = torch.autograd.grad(L, v)
    ref = q.q4c_integrate_backward(lib.tables, lib.grid, G, "fp64")
    assert torch.allclose(gv, ref, rtol=0, atol=0)
    # central finite difference (exact up to rounding for a linear map, step 1)
    idx = int(torch.argmax(ref.abs()))
    e = torch.zeros_like(lib.v); e[idx] = 1.0
    Lp = sum(float((Gm * M).sum()) for Gm, M in zip(G, q.integrate(lib.v + e, lib.tables, lib.grid, "fp64")))
    Lm = sum(float((Gm * M).sum()) for Gm, M in zip(G, q.integrate(lib.v - e, lib.tables, lib.grid, "fp64")))
    assert abs((Lp - Lm) / 2 - float(ref[idx])) <= 1e-9 * abs(float(ref[idx]))


def test_grid_handles_mismatch_rejected(water_pair):
    lib, _ = water_pair
    other = q.nao_tabulate([1], [0], [1.0])
    with pytest.raises(q.Q4CError) as e:
        q.q4c_integrate(other, lib.grid, lib.v, "fp64")
    assert e.value.status == 1
