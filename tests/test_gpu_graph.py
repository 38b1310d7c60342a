"""The compute calls inside a captured CUDA graph: integration, density and
adjoint (three calls, and the one-pass call) for a batch of independent
molecules and the per-column operator, captured once on a side stream and
replayed twice with new inputs written into the captured buffers; each
replay must give what the uncaptured calls give on the same inputs.  The
calls enqueue only kernels and asynchronous memsets on the caller's stream
(no host synchronisation, no allocation), so the whole step is one graph
launch."""
import numpy as np
import pytest

import oracle as O
import paper_2608_00773_gb300 as q
from workloads import ADJOINT_KINDS, column_operator, fill_pattern, molecule_batch, molecule_potential

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mol():
    import torch
    from paper_2608_00773_gb300 import _build
    _build.build()
    O.build()
    wl = molecule_batch(24, seed=1003, n_max=20, n_rad=20, n_theta=6, n_phi=12, batch_max=128)
    tables, grid = q.setup(wl)
    ex = grid.export()
    ppa = wl.n_rad * wl.n_theta * wl.n_phi
    v = torch.tensor(molecule_potential(ex["xyz"], ex["point_id"] // ppa, wl, device="cuda"), device="cuda")
    pat = (ex["blk_ptr"], ex["blk_col"], ex["blk_off"])
    P = torch.tensor(fill_pattern(*pat, wl.nf_of_atom, 41, "P"), device="cuda")
    G = [torch.tensor(fill_pattern(*pat, wl.nf_of_atom, 42, k, a), device="cuda") for k, a in ADJOINT_KINDS]
    return wl, tables, grid, v, P, G


def _rel(a, b):
    import torch
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("prec", ["fp64", "split"])
@pytest.mark.parametrize("fused", [False, True])
def test_step_in_cuda_graph(mol, prec, fused):
    import torch
    wl, tables, grid, v0, P0, G0 = mol
    nnz, npts = grid.nnz, grid.n_points
    # captured buffers: inputs the replays read, outputs they write
    v, P = v0.clone(), P0.clone()
    G = [g.clone() for g in G0]
    H = [torch.empty(nnz, dtype=torch.float64, device="cuda") for _ in range(5)] + [
        torch.empty(8 * nnz, dtype=torch.float64, device="cuda")]
    n = torch.empty(npts, dtype=torch.float64, device="cuda")
    g = torch.empty(npts, dtype=torch.float64, device="cuda")

    def step():
        if fused:
            q.q4c_scf_pass(tables, grid, v, [P, None, None, None, None], G, prec, H_out=H, n_out=n, dLdv_out=g)
        else:
            q.q4c_integrate(tables, grid, v, prec, out=H)
            q.q4c_density(tables, grid, P, prec, out=n)
            q.q4c_integrate_backward(tables, grid, G, prec, out=g)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()  # first use of every kernel before the capture
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        step()
    for rep in range(2):
        scale = 1.0 + 0.25 * rep  # new inputs in the captured buffers
        v.copy_(v0 * scale)
        P.copy_(P0 * (2.0 - scale))
        for a, b in zip(G, G0):
            a.copy_(b * scale)
        graph.replay()
        torch.cuda.synchronize()
        grid.status()
        ref_H = q.q4c_integrate(tables, grid, v0 * scale, prec, spinor=True)
        ref_n = q.q4c_density(tables, grid, P0 * (2.0 - scale), prec)
        ref_g = q.q4c_integrate_backward(tables, grid, [b * scale for b in G0], prec)
        torch.cuda.synchronize()
        tol = 1e-13
        for a, b in zip(H, ref_H):
            assert _rel(a, b) <= tol
        assert _rel(n, ref_n) <= tol
        assert _rel(g, ref_g) <= tol


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_columns_in_cuda_graph(mol, prec):
    import torch
    wl, tables, grid, v0, _, _ = mol
    eps, knots = column_operator(wl, 1201)
    q.q4c_tables_set_columns(tables, eps, knots)
    v = v0.clone()
    F = torch.empty(grid.nnz, dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        q.q4c_integrate_columns(tables, grid, v, prec, out=F)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        q.q4c_integrate_columns(tables, grid, v, prec, out=F)
    for rep in range(2):
        v.copy_(v0 * (0.5 + rep))
        graph.replay()
        torch.cuda.synchronize()
        grid.status()
        ref = q.q4c_integrate_columns(tables, grid, v0 * (0.5 + rep), prec)
        torch.cuda.synchronize()
        assert _rel(F, ref) <= 1e-13
