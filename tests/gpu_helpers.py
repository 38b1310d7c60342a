"""Shared plumbing of the GPU parity tests: run the library and the oracle on
the same seeded workload and line their outputs up.  The oracle builds its
own tables and grid; nothing it consumes comes from the CUDA path."""
from __future__ import annotations

import functools

import numpy as np

import oracle as O
import paper_2608_00773_gb300 as q
from workloads import ADJOINT_KINDS, fill_pattern, potential


def rel_fro(a, b) -> float:
    a = np.asarray(a, dtype=np.float64); b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


class LibCase:
    """Library side: tables, grid, v on the library's points."""

    def __init__(self, wl, knots=None):
        import torch
        self.wl = wl
        self.tables, self.grid = q.setup(wl, knots)
        self.ex = self.grid.export()
        self.v_host = potential(self.ex["xyz"], wl)
        self.v = torch.tensor(self.v_host, device="cuda")
        self.pat = (self.ex["blk_ptr"], self.ex["blk_col"], self.ex["blk_off"])

    def random(self, seed, kind, antisym=False):
        import torch
        vals = fill_pattern(*self.pat, self.wl.nf_of_atom, seed, kind, antisym, blk_T=self.ex["blk_T"])
        return torch.tensor(vals, device="cuda")

    def G(self, seed):
        return [self.random(seed, k, a) for k, a in ADJOINT_KINDS]

    def integrate(self, prec="fp64", spinor=False):
        outs = q.q4c_integrate(self.tables, self.grid, self.v, prec, spinor=spinor)
        return [None if o is None else o.cpu().numpy() for o in outs]


class OracleCase:
    """Oracle side: its own grid, pattern and v."""

    def __init__(self, wl, knots=None):
        self.wl = wl
        self.xyz, self.w, self.ids = O.grid(wl)
        self.ob = O.OracleBasis(wl, knots=knots)
        self.pat = self.ob.pattern()
        self.v = potential(self.xyz, wl)

    @functools.cached_property
    def mats(self):
        return self.ob.matrix_blocks(self.xyz, self.w, self.v, self.pat)

    def random(self, seed, kind, antisym=False):
        return fill_pattern(self.pat.blk_ptr, self.pat.blk_col, self.pat.blk_off, self.wl.nf_of_atom, seed, kind,
                            antisym, blk_T=self.pat.blk_T)

    def G(self, seed):
        return [self.random(seed, k, a) for k, a in ADJOINT_KINDS]


def point_map(lib_ids, orc_ids):
    """Index arrays (li, oi) pairing library and oracle points by raw id."""
    common, li, oi = np.intersect1d(lib_ids, orc_ids, assume_unique=True, return_indices=True)
    return li, oi
