"""GPU parity of the split-precision (BF16-slice tensor-core) path against
the CPU oracle, at the 1e-9 relative Frobenius bound per matrix, plus the
full-size workload that bench.py times (sampled entries the oracle computes
one by one, for both the FP64 and the split path)."""
import numpy as np
import pytest

import oracle as O
import paper_2608_00773_gb300 as q
from gpu_helpers import LibCase, OracleCase, rel_fro
from workloads import Species, Workload, cluster64, single_atom, small_cluster, water

pytestmark = pytest.mark.gpu
TOL_SPLIT = 1e-9
TOL_FP64 = 1e-12
NAMES = ["V", "W0", "SOx", "SOy", "SOz"]


@pytest.fixture(scope="session", autouse=True)
def _built():
    from paper_2608_00773_gb300 import _build
    _build.build()
    O.build()


@pytest.fixture(scope="module")
def pairs():
    return {name: (LibCase(wl), OracleCase(wl)) for name, wl in
            (("water", water()), ("cluster", small_cluster(8, seed=7)), ("cluster12", small_cluster(12, seed=9)))}


@pytest.mark.parametrize("name", ["water", "cluster", "cluster12"])
def test_integrate_split_matches_oracle(name, pairs):
    lib, orc = pairs[name]
    got = lib.integrate("split", spinor=True)
    lib.grid.status()
    errs = {n: rel_fro(g, r) for n, g, r in zip(NAMES, got[:5], orc.mats)}
    assert max(errs.values()) <= TOL_SPLIT, errs
    pat = orc.pat
    V, W0, SOx = (orc.ob.dense(m, pat) for m in got[:3])
    assert np.array_equal(V, V.T) and np.array_equal(W0, W0.T) and np.array_equal(SOx, -SOx.T)
    ref = orc.ob.spinor_ss(*orc.mats[1:], pat)
    assert np.linalg.norm(got[5].view(np.complex128) - ref) <= TOL_SPLIT * np.linalg.norm(ref)


def test_split_repeatable(pairs):
    lib, _ = pairs["cluster"]
    a = lib.integrate("split")
    b = lib.integrate("split")
    for x, y in zip(a[:5], b[:5]):
        assert rel_fro(x, y) <= 1e-14


EDGE = {
    "single-atom-l0123": lambda: single_atom([0, 1, 2, 3], [0.8, 1.1, 1.6, 2.2], Z=6.0, n_rad=20, n_theta=6,
                                             n_phi=12),
    "far-pair": lambda: Workload("far-pair", np.array([[0.0, 0, 0], [13.0, 0.5, -0.2]]), np.array([0, 1], np.int32),
                                 [Species("A", 3.0, [0, 1], [0.9, 1.4]), Species("B", 1.0, [0, 2], [1.2, 0.7])],
                                 n_rad=16, n_theta=6, n_phi=12),
    "one-point-batches": lambda: water(n_rad=8, n_theta=4, n_phi=8, batch_max=1),
    "341-point-batches": lambda: water(n_rad=40, n_theta=10, n_phi=20, batch_max=341),
}


@pytest.mark.parametrize("case", list(EDGE))
def test_integrate_split_edge_cases(case):
    wl = EDGE[case]()
    lib, orc = LibCase(wl), OracleCase(wl)
    got = lib.integrate("split")
    f64 = lib.integrate("fp64")
    lib.grid.status()
    errs = {n: rel_fro(g, r) for n, g, r in zip(NAMES, got[:5], orc.mats)}
    diag = {}
    for n, g, h, r in zip(NAMES, got[:5], f64[:5], orc.mats):
        k = int(np.argmax(np.abs(g - r)))
        diag[n] = dict(split_vs_fp64=rel_fro(g, h), fp64_vs_oracle=rel_fro(h, r), worst_index=k,
                       worst_abs=float(abs(g[k] - r[k])), ref_there=float(r[k]), max_ref=float(np.abs(r).max()))
    assert max(errs.values()) <= TOL_SPLIT, (case, errs, diag, int(lib.grid.info.max_np), int(lib.grid.info.max_nb))


def test_split_rejects_batches_beyond_exactness_bound():
    # ~18k kept points; median bisection down to <= 1000 points per batch
    # leaves batches of ~560 points, past the split path's 341-point bound
    wl = water(n_rad=40, n_theta=10, n_phi=20, batch_max=1000)
    lib = LibCase(wl)
    assert lib.grid.info.max_np > 341
    with pytest.raises(q.Q4CError) as e:
        lib.integrate("split")
    assert e.value.status == 5


def test_bounded_wait_timeout_is_reported_and_recovers():
    """A work-wait limit of 1 ns makes the tensor kernels' first unsatisfied
    wait give up: the call returns, q4c_grid_status reports Q4C_ETIMEOUT once
    and clears it, and with the default limit restored the same calls give
    the normal results on the same context."""
    wl = water()
    lib = LibCase(wl)
    G = lib.G(31)
    ref = lib.integrate("split")
    gref = q.q4c_integrate_backward(lib.tables, lib.grid, G, "split").cpu().numpy()
    lib.grid.status()
    try:
        q.q4c_set_wait_limit_ns(1)
        q.q4c_integrate(lib.tables, lib.grid, lib.v, "split")
        with pytest.raises(q.Q4CError) as e:
            lib.grid.status()
        assert e.value.status == 4
        lib.grid.status()  # the flag was cleared
        q.q4c_integrate_backward(lib.tables, lib.grid, G, "split")
        with pytest.raises(q.Q4CError) as e:
            lib.grid.status()
        assert e.value.status == 4
        # the autograd function raises instead of returning incomplete outputs
        import torch
        v = lib.v.clone().requires_grad_(True)
        with pytest.raises(q.Q4CError):
            q.integrate(v, lib.tables, lib.grid, "split")
    finally:
        q.q4c_set_wait_limit_ns(0)
    lib.grid.status()
    again = lib.integrate("split")
    gagain = q.q4c_integrate_backward(lib.tables, lib.grid, G, "split").cpu().numpy()
    lib.grid.status()
    for a, b in zip(again[:5], ref[:5]):
        assert rel_fro(a, b) <= 1e-13
    assert rel_fro(gagain, gref) <= 1e-13


# ----------------------------------------------------------------- full size


@pytest.fixture(scope="module")
def full():
    """The 64-atom, ~1.2M-point workload of bench.py; the oracle builds its
    own grid and evaluates sampled matrix entries over all of its points."""
    wl = cluster64()
    lib = LibCase(wl)
    xyz, w, ids = O.grid(wl)
    ob = O.OracleBasis(wl)
    from workloads import potential
    v = potential(xyz, wl)
    rng = np.random.default_rng(2024)
    nf = wl.nf_of_atom
    first = np.concatenate([[0], np.cumsum(nf)])
    pat = ob.pattern()
    pi, pj = [], []
    # diagonal blocks, near and far neighbour blocks, heavy and light atoms
    for A in rng.choice(wl.n_atoms, 12, replace=False):
        cols = pat.blk_col[pat.blk_ptr[A]:pat.blk_ptr[A + 1]]
        for B in (A, cols[len(cols) // 2], cols[-1]):
            i = first[A] + rng.integers(nf[A]); j = first[B] + rng.integers(nf[B])
            pi.append(i); pj.append(j)
    pi = np.array(pi, np.int32); pj = np.array(pj, np.int32)
    ref = ob.matrix_pairs(xyz, w, v, pi, pj)
    return lib, pat, pi, pj, ref, first


def _sampled(vals, pat, pi, pj, first, wl):
    out = np.zeros(len(pi))
    nf = wl.nf_of_atom
    atom_of = np.searchsorted(first, np.arange(first[-1]), side="right") - 1
    for k, (i, j) in enumerate(zip(pi, pj)):
        A, B = atom_of[i], atom_of[j]
        cols = pat.blk_col[pat.blk_ptr[A]:pat.blk_ptr[A + 1]]
        qb = pat.blk_ptr[A] + int(np.where(cols == B)[0][0])
        out[k] = vals[pat.blk_off[qb] + (i - first[A]) * nf[B] + (j - first[B])]
    return out


@pytest.mark.parametrize("prec,tol", [("fp64", TOL_FP64), ("split", TOL_SPLIT)])
def test_full_size_sampled_entries(prec, tol, full):
    lib, pat, pi, pj, ref, first = full
    got = lib.integrate(prec)
    lib.grid.status()
    # the library's pattern equals the oracle's (bit-exact), so offsets agree
    assert np.array_equal(lib.ex["blk_off"], pat.blk_off)
    for n, g, r in zip(NAMES, got[:5], ref):
        s = _sampled(g, pat, pi, pj, first, lib.wl)
        assert np.linalg.norm(s - r) <= tol * np.linalg.norm(r), (prec, n, np.linalg.norm(s - r) / np.linalg.norm(r))


# ----------------------------------------------------------------- density / adjoint


@pytest.mark.parametrize("name", ["water", "cluster", "cluster12"])
def test_density_split_matches_oracle(name, pairs):
    from gpu_helpers import point_map
    lib, orc = pairs[name]
    n = q.q4c_density(lib.tables, lib.grid, lib.random(55, "P"), "split").cpu().numpy()
    lib.grid.status()
    nref = orc.ob.density(orc.xyz, orc.random(55, "P"), orc.pat)
    li, oi = point_map(lib.ex["point_id"], orc.ids)
    assert rel_fro(n[li], nref[oi]) <= TOL_SPLIT, rel_fro(n[li], nref[oi])


@pytest.mark.parametrize("name", ["water", "cluster", "cluster12"])
def test_backward_split_matches_oracle(name, pairs):
    from gpu_helpers import point_map
    lib, orc = pairs[name]
    g = q.q4c_integrate_backward(lib.tables, lib.grid, lib.G(66), "split").cpu().numpy()
    lib.grid.status()
    gref = orc.ob.adjoint(orc.xyz, orc.w, orc.G(66), orc.pat)
    li, oi = point_map(lib.ex["point_id"], orc.ids)
    assert rel_fro(g[li], gref[oi]) <= TOL_SPLIT, rel_fro(g[li], gref[oi])


def test_backward_split_partial_slots_and_autograd(pairs):
    """NULL G slots count as zero; the autograd wrapper routes through the
    split adjoint; linearity sum_p v_p dL/dv_p = L holds for the split pair."""
    import torch
    lib, orc = pairs["cluster"]
    G = lib.G(8)
    only_w = [None, G[1], None, None, None]
    a = q.q4c_integrate_backward(lib.tables, lib.grid, only_w, "split").cpu().numpy()
    b = q.q4c_integrate_backward(lib.tables, lib.grid, only_w, "fp64").cpu().numpy()
    assert rel_fro(a, b) <= TOL_SPLIT
    v = lib.v.clone().requires_grad_(True)
    outs = q.integrate(v, lib.tables, lib.grid, "split")
    L = sum((Gm * M).sum() for Gm, M in zip(G, outs))
    (gv,) = torch.autograd.grad(L, v)
    ref = q.q4c_integrate_backward(lib.tables, lib.grid, G, "fp64")
    assert rel_fro(gv.cpu().numpy(), ref.cpu().numpy()) <= TOL_SPLIT
    assert abs(float((lib.v * gv).sum()) - float(L)) <= 1e-9 * abs(float(L))


@pytest.mark.parametrize("prec,tol", [("fp64", TOL_FP64), ("split", TOL_SPLIT)])
def test_full_size_density_and_adjoint_sampled_points(prec, tol):
    """Density and adjoint at the full workload against the oracle at 300
    points of the oracle's own grid (matched by raw point id)."""
    from workloads import ADJOINT_KINDS, fill_pattern
    wl = cluster64()
    lib = LibCase(wl)
    xyz, w, ids = O.grid(wl)
    ob = O.OracleBasis(wl)
    pat = ob.pattern()
    rng = np.random.default_rng(77)
    sel = np.sort(rng.choice(len(ids), 300, replace=False))
    P_o = fill_pattern(pat.blk_ptr, pat.blk_col, pat.blk_off, wl.nf_of_atom, 31, "P")
    G_o = [fill_pattern(pat.blk_ptr, pat.blk_col, pat.blk_off, wl.nf_of_atom, 32, k, a) for k, a in ADJOINT_KINDS]
    n_ref = ob.density(xyz[sel], P_o, pat)
    g_ref = ob.adjoint(xyz[sel], w[sel], G_o, pat)
    n = q.q4c_density(lib.tables, lib.grid, lib.random(31, "P"), prec).cpu().numpy()
    g = q.q4c_integrate_backward(lib.tables, lib.grid, [lib.random(32, k, a) for k, a in ADJOINT_KINDS],
                                 prec).cpu().numpy()
    lib.grid.status()
    pos = {int(p): k for k, p in enumerate(lib.ex["point_id"])}
    li = np.array([pos[int(i)] for i in ids[sel]])
    assert rel_fro(n[li], n_ref) <= tol, rel_fro(n[li], n_ref)
    assert rel_fro(g[li], g_ref) <= tol, rel_fro(g[li], g_ref)


def test_split_repeated_calls_agree_with_fp64():
    """Integration, adjoint and density in alternation over several seeds (the
    tensor-core kernels then start on shared memory and tensor memory that the
    other kernels left behind), each against the FP64 path: catches ordering
    faults between the asynchronous copies and the threads that read them."""
    import torch
    wl = small_cluster(12, seed=9)
    lib = LibCase(wl)
    Vref = q.q4c_integrate(lib.tables, lib.grid, lib.v, "fp64")
    for seed in range(6):
        Vs = q.q4c_integrate(lib.tables, lib.grid, lib.v, "split")
        for a, b in zip(Vs[:5], Vref[:5]):
            assert float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) <= TOL_SPLIT, seed
        G = lib.G(100 + seed)
        g = q.q4c_integrate_backward(lib.tables, lib.grid, G, "split")
        q.q4c_integrate(lib.tables, lib.grid, lib.v, "split")
        n = q.q4c_density(lib.tables, lib.grid, G[0], "split")
        gr = q.q4c_integrate_backward(lib.tables, lib.grid, G, "fp64")
        nr = q.q4c_density(lib.tables, lib.grid, G[0], "fp64")
        assert float(torch.linalg.norm(g - gr) / torch.linalg.norm(gr)) <= TOL_SPLIT, seed
        assert float(torch.linalg.norm(n - nr) / torch.linalg.norm(nr)) <= TOL_SPLIT, seed
    lib.grid.status()
