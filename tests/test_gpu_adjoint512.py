"""The adjoint at the 512-atom configuration (~6,400 functions, 20M raw grid
points, batches <= 128): dL/dv on every point through the autograd function,
checked at sampled points against the oracle (points, Becke weights and
basis of its own grid, matched by raw id), by central differences of L (L is
linear in v, so a large step is exact up to rounding), and along a random
direction."""
import numpy as np
import pytest

import oracle as O
import paper_2608_00773_gb300 as q
from workloads import ADJOINT_KINDS, cluster512, fill_pattern, potential

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def big():
    import torch
    from paper_2608_00773_gb300 import _build
    _build.build()
    O.build()
    import time
    t0 = time.time()
    wl = cluster512()
    tables, grid = q.setup(wl)
    t1 = time.time()
    ex = grid.export()
    pat = (ex["blk_ptr"], ex["blk_col"], ex["blk_off"])
    G_h = [fill_pattern(*pat, wl.nf_of_atom, 2004, k, a) for k, a in ADJOINT_KINDS]
    G = [torch.tensor(g, device="cuda") for g in G_h]
    t2 = time.time()
    v = torch.tensor(potential(ex["xyz"], wl, device="cuda"), device="cuda")
    print(f"grid {t1 - t0:.1f} s, export + G {t2 - t1:.1f} s, v {time.time() - t2:.1f} s")
    return wl, tables, grid, ex, G_h, G, v


def _L(tables, grid, v, G, prec):
    mats = q.q4c_integrate(tables, grid, v, prec)[:5]
    return sum(float((m * g).sum()) for m, g in zip(mats, G))


def test_sizes(big):
    wl, tables, grid, ex, *_ = big
    assert wl.n_raw_points == 20070400 and 6000 < wl.n_basis < 6800
    assert grid.info.max_np <= 128


def test_autograd_equals_backward_and_oracle_samples(big):
    import torch
    wl, tables, grid, ex, G_h, G, v = big
    vv = v.clone().requires_grad_(True)
    outs = q.integrate(vv, tables, grid, "split")
    L = sum((o * g).sum() for o, g in zip(outs, G))
    L.backward()
    g_auto = vv.grad.detach().cpu().numpy()
    g_direct = q.q4c_integrate_backward(tables, grid, G, "split").cpu().numpy()
    grid.status()
    assert np.array_equal(g_auto, g_direct)
    # the oracle at 64 sampled points of its own grid (its own coordinates,
    # Becke weights and basis), matched to the library's points by raw id
    ob = O.OracleBasis(wl)
    pat = ob.pattern()
    assert np.array_equal(pat.blk_off, ex["blk_off"])
    oxyz, ow, oids = O.grid(wl, stride=9973)  # a uniform ~2,000-point sample of the raw grid
    pos = {int(p): k for k, p in enumerate(ex["point_id"])}
    both = np.array([k for k, i in enumerate(oids) if int(i) in pos])
    assert len(both) >= 64
    rng = np.random.default_rng(2004)
    sel = np.sort(rng.choice(both, 64, replace=False))
    li = np.array([pos[int(i)] for i in oids[sel]])
    assert np.allclose(ex["w"][li], ow[sel], rtol=1e-12, atol=0)
    gref = ob.adjoint(oxyz[sel], ow[sel], G_h, pat)
    err = np.abs(g_direct[li] - gref).max() / np.abs(gref).max()
    assert err <= 1e-9, err


def test_central_differences_and_direction(big):
    """(L(v + h e_p) - L(v - h e_p)) / 2h = dL/dv_p for any h (L is linear in v)."""
    import torch
    wl, tables, grid, ex, G_h, G, v = big
    g = q.q4c_integrate_backward(tables, grid, G, "fp64").cpu().numpy()
    rng = np.random.default_rng(7)
    h = 1e4
    scale = np.abs(g).max()
    for p in rng.choice(len(g), 12, replace=False):
        e = torch.zeros_like(v)
        e[int(p)] = h
        fd = (_L(tables, grid, v + e, G, "fp64") - _L(tables, grid, v - e, G, "fp64")) / (2 * h)
        assert abs(fd - g[p]) <= 1e-9 * scale, (p, fd, g[p])
    u = torch.tensor(rng.standard_normal(len(g)), device="cuda")
    dd = (_L(tables, grid, v + u, G, "fp64") - _L(tables, grid, v - u, G, "fp64")) / 2
    assert abs(dd - float(np.dot(u.cpu().numpy(), g))) <= 1e-10 * abs(dd)
