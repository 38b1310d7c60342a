"""Pin of the oracle's listed-pair matrix elements (orc_matrix_pairs).

The full-size parity tests of the integration compare sampled (i, j)
entries of the library against orc_matrix_pairs, so that routine must be
pinned to something other than the GPU.  Here it is compared with the
block-pattern oracle (orc_matrix_blocks), itself pinned by closed forms in
test_oracle_pins.py, at listed pairs: every pair of the water molecule and a
seeded sample of an 8-atom heavy/light cluster that covers diagonal,
off-diagonal, same-atom, heavy/light and transposed pairs, all five outputs
(Eqs. 29-30 with F = v and the kinetic-balance SS reading).  A swapped i/j,
a wrong spin-orbit sign or a wrong list of evaluated functions in
orc_matrix_pairs breaks the equality.  Both routines add the same per-point
products in the same point order, so they agree to the last bit up to the
exact zeros the block routine skips; the bound is 1e-15 of each output's
largest entry.  CPU only.
"""
import numpy as np
import pytest

import oracle as O
from workloads import potential, small_cluster, water


def _dense_all(ob, xyz, w, v):
    pat = ob.pattern()
    return [ob.dense(m, pat) for m in ob.matrix_blocks(xyz, w, v, pat)]


def _check(ob, dense, xyz, w, v, pi, pj):
    got = ob.matrix_pairs(xyz, w, v, pi, pj)
    for k, (g, D) in enumerate(zip(got, dense)):
        ref = D[pi, pj]
        scale = np.abs(D).max()
        assert scale > 0
        err = np.abs(g - ref).max() / scale
        assert err <= 1e-15, (k, err)
    return got


def test_matrix_pairs_equal_blocks_water_every_pair():
    wl = water()
    xyz, w, _ = O.grid(wl)
    v = potential(xyz, wl)
    ob = O.OracleBasis(wl)
    dense = _dense_all(ob, xyz, w, v)
    n = ob.n_fn
    pi, pj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    pi, pj = pi.ravel(), pj.ravel()
    got = _check(ob, dense, xyz, w, v, pi, pj)
    # the listed form keeps the symmetry of V, W0 and the antisymmetry of SO
    V = got[0].reshape(n, n)
    SOx = got[2].reshape(n, n)
    assert np.array_equal(V, V.T)
    assert np.array_equal(SOx, -SOx.T)


@pytest.mark.parametrize("stride", [3])
def test_matrix_pairs_equal_blocks_cluster_sampled(stride):
    wl = small_cluster(8)
    xyz, w, _ = O.grid(wl, stride=stride)
    v = potential(xyz, wl)
    ob = O.OracleBasis(wl)
    dense = _dense_all(ob, xyz, w, v)
    n = ob.n_fn
    rng = np.random.default_rng(2026)
    fa = ob.fn_atom
    pairs = set()
    # diagonal entries, pairs within one atom, pairs across atoms (both orders)
    for i in rng.choice(n, 40, replace=False):
        pairs.add((int(i), int(i)))
    while len(pairs) < 200:
        i, j = (int(x) for x in rng.integers(0, n, 2))
        pairs.add((i, j))
        pairs.add((j, i))
    for A in range(wl.n_atoms):
        idx = np.flatnonzero(fa == A)
        i, j = (int(x) for x in rng.choice(idx, 2, replace=len(idx) < 2))
        pairs.add((i, j))
        pairs.add((j, i))
    pairs = sorted(pairs)
    assert len(pairs) >= 200
    pi = np.array([p[0] for p in pairs], np.int32)
    pj = np.array([p[1] for p in pairs], np.int32)
    # the sample must cover heavy/light combinations and entries that are not zero
    nf = np.asarray(wl.nf_of_atom)
    heavy = nf[fa] > 5
    assert (heavy[pi] & ~heavy[pj]).any() and (heavy[pi] & heavy[pj]).any() and (~heavy[pi] & ~heavy[pj]).any()
    assert (np.abs(dense[0][pi, pj]) > 0).sum() > 100
    got = _check(ob, dense, xyz, w, v, pi, pj)
    # transposed pairs: V, W0 equal, SO opposite
    where = {p: q for q, p in enumerate(pairs)}
    for q, (i, j) in enumerate(pairs):
        r = where.get((j, i))
        if r is None:
            continue
        assert got[0][q] == got[0][r] and got[1][q] == got[1][r]
        for k in (2, 3, 4):
            assert got[k][q] == -got[k][r]
