"""q4c_integrate_noalloc: the FP64 integration for callers that cannot
allocate device memory during the call (their memory belongs to their own
pool, or the call sits in a loop that must not pay for cudaMalloc).  Its
workspace is a static 64 MiB device array shared by all calls.

Checked through the C ABI against q4c_integrate(FP64) on two calls in a row,
at the FP64 tolerance of the other tests.  The 64-atom workload needs ~2 GB of
basis tiles, so there the static array is reused over many waves.  Kept in a
file that pytest collects last."""
import ctypes as C

import numpy as np
import pytest

import paper_2608_00773_gb300 as q
from paper_2608_00773_gb300 import binding as B
from workloads import cluster64, potential, small_cluster, water

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2608_00773_gb300 import _build
    _build.build()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("make", [water, lambda: small_cluster(8, seed=7), cluster64],
                         ids=["water", "cluster8", "cluster64"])
def test_noalloc_matches_integrate(make):
    import torch
    wl = make()
    tables, grid = q.setup(wl)
    ex = grid.export()
    v = torch.tensor(potential(ex["xyz"], wl), device="cuda")
    ref = q.q4c_integrate(tables, grid, v, "fp64", spinor=True)
    ref = [r.cpu().numpy() for r in ref]
    L = q.load()
    for call in range(2):
        out = [torch.full((grid.nnz,), np.nan, dtype=torch.float64, device="cuda") for _ in range(5)]
        out.append(torch.full((8 * grid.nnz,), np.nan, dtype=torch.float64, device="cuda"))
        m = B.Matrices(*[t.data_ptr() for t in out])
        st = L.q4c_integrate_noalloc(tables.h, grid.h, v.data_ptr(), C.byref(m),
                                     torch.cuda.current_stream().cuda_stream)
        assert st == 0, L.q4c_last_error()
        torch.cuda.synchronize()
        for name, o, r in zip(["V", "W0", "SOx", "SOy", "SOz", "SS"], out, ref):
            o = o.cpu().numpy()
            assert np.all(np.isfinite(o)), (call, name)
            assert _rel(o, r) <= TOL, (call, name, _rel(o, r))


def test_noalloc_rejects_bad_arguments():
    L = q.load()
    m = B.Matrices(0, 0, 0, 0, 0, 0)
    assert L.q4c_integrate_noalloc(None, None, None, C.byref(m), None) == 1
