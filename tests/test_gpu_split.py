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
    wl = water(n_rad=40, n_theta=10, n_phi=20, batch_max=400)
    lib = LibCase(wl)
    if lib.grid.info.max_np <= 341:
        pytest.skip("bisection produced small batches")
    with pytest.raises(q.Q4CError) as e:
        lib.integrate("split")
    assert e.value.status == 5


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
