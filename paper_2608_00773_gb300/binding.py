"""Thin ctypes binding of libq4c.so (include/q4c.h), same names as the C ABI.

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels.  PyTorch provides device memory and streams.  If the
shared library is missing, importing this module raises: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libq4c.so")

Q4C_FP64 = 0
Q4C_SPLIT = 1
PRECISIONS = {"fp64": Q4C_FP64, "split": Q4C_SPLIT}

STATUS = {0: "Q4C_OK", 1: "Q4C_EINVAL", 2: "Q4C_ENOMEM", 3: "Q4C_ECUDA", 4: "Q4C_ETIMEOUT", 5: "Q4C_EUNSUPPORTED"}

# every symbol include/q4c.h declares
EXPORTS = ["nao_tabulate", "nao_tabulate_knots", "q4c_tables_destroy", "q4c_tables_export", "grid_partition", "q4c_grid_destroy",
           "q4c_grid_get_info", "q4c_grid_export", "q4c_grid_export_shifts", "q4c_grid_kpattern", "q4c_kfold", "q4c_grid_points", "q4c_integrate", "q4c_density", "q4c_density_full",
           "q4c_spinor_basis", "q4c_spinor_transform", "q4c_spinor_density_matrices", "q4c_grid_batch_spinors",
           "q4c_tables_set_columns", "q4c_integrate_columns", "q4c_tables_set_kappa", "q4c_spinor_nnz",
           "q4c_integrate_backward", "q4c_scf_pass", "q4c_autotune", "q4c_grid_tiling", "q4c_grid_set_tiling", "q4c_integrate_noalloc", "q4c_basis_eval", "q4c_grid_status", "q4c_set_wait_limit_ns", "q4c_profile", "q4c_profile_read",
           "q4c_last_error"]


class Q4CError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class BasisDesc(C.Structure):
    _fields_ = [("n_species", C.c_int32), ("n_rad", C.c_void_p), ("l", C.c_void_p), ("alpha", C.c_void_p),
                ("r_cut", C.c_double), ("r_on", C.c_double), ("r_min", C.c_double), ("n_log", C.c_int32)]


class GridDesc(C.Structure):
    _fields_ = [("n_atoms", C.c_int32), ("xyz", C.c_void_p), ("species", C.c_void_p),
                ("n_rad_shells", C.c_int32), ("R", C.c_double), ("n_theta", C.c_int32), ("n_phi", C.c_int32),
                ("r_nb", C.c_double), ("batch_max", C.c_int32), ("lattice", C.c_void_p), ("n_shell", C.c_int32),
                ("n_molecules", C.c_int32), ("mol_atom_ptr", C.c_void_p), ("partition", C.c_int32)]


PARTITIONS = {"becke": 0, "stratmann": 1}


class GridInfo(C.Structure):
    _fields_ = [("n_points", C.c_int64), ("n_batches", C.c_int64), ("n_blocks", C.c_int64), ("nnz", C.c_int64),
                ("n_atoms", C.c_int32), ("n_basis", C.c_int32), ("max_nb", C.c_int32), ("max_np", C.c_int32),
                ("flops_alg", C.c_double), ("sum_np_nb", C.c_double), ("scratch_bytes", C.c_int64)]


class Matrices(C.Structure):
    _fields_ = [("V", C.c_void_p), ("W0", C.c_void_p), ("SOx", C.c_void_p), ("SOy", C.c_void_p),
                ("SOz", C.c_void_p), ("spinor_SS", C.c_void_p)]


_lib: Optional[C.CDLL] = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Loads libq4c.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(nvcc for sm_103a); there is no CPU fallback")
    L = C.CDLL(path)
    vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
    L.nao_tabulate.argtypes = [C.POINTER(BasisDesc), C.POINTER(vp)]
    L.nao_tabulate_knots.argtypes = [C.POINTER(BasisDesc), vp, C.POINTER(vp)]
    L.q4c_tables_set_kappa.argtypes = [vp, vp]
    L.q4c_spinor_nnz.argtypes = [vp, vp, C.POINTER(i64)]
    L.q4c_tables_destroy.argtypes = [vp]
    L.q4c_tables_destroy.restype = None
    L.q4c_tables_export.argtypes = [vp, i32, vp]
    L.grid_partition.argtypes = [C.POINTER(GridDesc), vp, C.POINTER(vp)]
    L.q4c_grid_destroy.argtypes = [vp]
    L.q4c_grid_destroy.restype = None
    L.q4c_grid_get_info.argtypes = [vp, C.POINTER(GridInfo)]
    L.q4c_grid_export.argtypes = [vp] + [vp] * 9
    L.q4c_grid_export_shifts.argtypes = [vp, vp]
    L.q4c_grid_kpattern.argtypes = [vp, vp, vp, vp, vp]
    L.q4c_kfold.argtypes = [vp, vp, i32, vp, vp, vp]
    L.q4c_grid_points.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(i64)]
    L.q4c_integrate.argtypes = [vp, vp, vp, C.c_int, C.POINTER(Matrices), vp]
    L.q4c_density.argtypes = [vp, vp, vp, C.c_int, vp, vp]
    L.q4c_integrate_backward.argtypes = [vp, vp, C.POINTER(Matrices), C.c_int, vp, vp]
    L.q4c_density_full.argtypes = [vp, vp, C.POINTER(Matrices), C.c_int, vp, vp]
    L.q4c_spinor_basis.argtypes = [vp, i32, vp, vp, vp, vp]
    L.q4c_tables_set_columns.argtypes = [vp, vp, vp]
    L.q4c_integrate_columns.argtypes = [vp, vp, vp, i32, vp, vp]
    L.q4c_spinor_transform.argtypes = [vp, vp, C.POINTER(Matrices), vp, vp, vp]
    L.q4c_spinor_density_matrices.argtypes = [vp, vp, vp, C.POINTER(Matrices), vp]
    L.q4c_grid_batch_spinors.argtypes = [vp, i64, vp, vp, vp]
    L.q4c_scf_pass.argtypes = [vp, vp, vp, C.POINTER(Matrices), C.POINTER(Matrices), vp, C.POINTER(Matrices), vp,
                               C.c_int, vp]
    L.q4c_integrate_noalloc.argtypes = [vp, vp, vp, C.POINTER(Matrices), vp]
    L.q4c_autotune.argtypes = [vp, vp, vp, vp]
    L.q4c_grid_tiling.argtypes = [vp, i32, vp, vp, vp, vp, vp]
    L.q4c_grid_set_tiling.argtypes = [vp, i32, i32]
    L.q4c_basis_eval.argtypes = [vp, vp, i64, vp, vp, vp, vp]
    L.q4c_grid_status.argtypes = [vp, vp]
    L.q4c_set_wait_limit_ns.argtypes = [C.c_uint64]
    L.q4c_profile.argtypes = [i32]
    L.q4c_profile_read.argtypes = [C.c_char_p, C.POINTER(C.c_double), C.POINTER(i64)]
    L.q4c_last_error.restype = C.c_char_p
    _lib = L
    return L


def _check(status: int):
    if status != 0:
        raise Q4CError(status, load().q4c_last_error().decode())


def _ptr(t) -> int:
    """Device pointer of a torch tensor (None -> NULL)."""
    if t is None:
        return 0
    if not t.is_contiguous():
        raise ValueError("tensors passed to libq4c must be contiguous")
    return t.data_ptr()


def _stream(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


# --------------------------------------------------------------------------
# handles
# --------------------------------------------------------------------------

class Tables:
    """q4c_tables handle (nao_tabulate)."""

    def __init__(self, n_rad: Sequence[int], l: Sequence[int], alpha: Optional[Sequence[float]], r_cut=6.0,
                 r_on=5.0, r_min=1e-4, n_log=200, knots: Optional[np.ndarray] = None):
        """Radials u = r^(l+1) exp(-alpha r^2) c(r) (nao_tabulate), or, with knots
        [sum n_rad][n_log], the given values at the knots (nao_tabulate_knots)."""
        L = load()
        self._n_rad = np.ascontiguousarray(n_rad, np.int32)
        self._l = np.ascontiguousarray(l, np.int32)
        self._alpha = None if alpha is None else np.ascontiguousarray(alpha, np.float64)
        d = BasisDesc(len(self._n_rad), self._n_rad.ctypes.data, self._l.ctypes.data,
                      None if self._alpha is None else self._alpha.ctypes.data, r_cut, r_on, r_min, n_log)
        h = C.c_void_p()
        if knots is None:
            _check(L.nao_tabulate(C.byref(d), C.byref(h)))
        else:
            kn = np.ascontiguousarray(knots, np.float64)
            if kn.shape != (len(self._l), n_log):
                raise ValueError("knots must be [sum n_rad][n_log]")
            _check(L.nao_tabulate_knots(C.byref(d), kn.ctypes.data, C.byref(h)))
        self.h = h
        self.n_log = n_log

    def coefficients(self, radial: int) -> np.ndarray:
        out = np.zeros((self.n_log - 1, 4))
        _check(load().q4c_tables_export(self.h, radial, out.ctypes.data))
        return out

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.q4c_tables_destroy(self.h)
            self.h = None


class Grid:
    """q4c_grid handle (grid_partition)."""

    def __init__(self, tables: Tables, xyz, species, n_rad_shells, R, n_theta, n_phi, r_nb, batch_max,
                 lattice=None, n_shell: int = 0, mol_atom_ptr=None, partition: str = "becke"):
        L = load()
        self.tables = tables
        self._xyz = np.ascontiguousarray(xyz, np.float64).reshape(-1)
        self._sp = np.ascontiguousarray(species, np.int32)
        self._lat = None if lattice is None else np.ascontiguousarray(lattice, np.float64).reshape(-1)
        self._mol = None if mol_atom_ptr is None else np.ascontiguousarray(mol_atom_ptr, np.int32)
        d = GridDesc(len(self._sp), self._xyz.ctypes.data, self._sp.ctypes.data, n_rad_shells, R, n_theta, n_phi,
                     r_nb, batch_max, None if self._lat is None else self._lat.ctypes.data, int(n_shell),
                     0 if self._mol is None else len(self._mol) - 1,
                     None if self._mol is None else self._mol.ctypes.data, PARTITIONS[partition])
        h = C.c_void_p()
        _check(L.grid_partition(C.byref(d), tables.h, C.byref(h)))
        self.h = h
        info = GridInfo()
        _check(L.q4c_grid_get_info(self.h, C.byref(info)))
        self.info = info

    @property
    def n_points(self) -> int:
        return int(self.info.n_points)

    @property
    def nnz(self) -> int:
        return int(self.info.nnz)

    def export(self):
        """Host copies: dict of numpy arrays (points in batch order, batches, pattern)."""
        i = self.info
        xyz = np.zeros((i.n_points, 3)); w = np.zeros(i.n_points); pid = np.zeros(i.n_points, np.int64)
        bptr = np.zeros(i.n_batches + 1, np.int64); baptr = np.zeros(i.n_batches + 1, np.int64)
        _check(load().q4c_grid_export(self.h, None, None, None, None, baptr.ctypes.data, None, None, None, None))
        batoms = np.zeros(max(int(baptr[-1]), 1), np.int32)
        blk_ptr = np.zeros(i.n_atoms + 1, np.int64); blk_col = np.zeros(max(i.n_blocks, 1), np.int32)
        blk_off = np.zeros(i.n_blocks + 1, np.int64)
        _check(load().q4c_grid_export(self.h, xyz.ctypes.data, w.ctypes.data, pid.ctypes.data, bptr.ctypes.data,
                                      baptr.ctypes.data, batoms.ctypes.data, blk_ptr.ctypes.data,
                                      blk_col.ctypes.data, blk_off.ctypes.data))
        blk_T = np.zeros(3 * max(i.n_blocks, 1), np.int32)
        _check(load().q4c_grid_export_shifts(self.h, blk_T.ctypes.data))
        return dict(xyz=xyz, w=w, point_id=pid, batch_ptr=bptr, batch_atom_ptr=baptr,
                    batch_atoms=batoms[:int(baptr[-1])], blk_ptr=blk_ptr, blk_col=blk_col[:i.n_blocks],
                    blk_off=blk_off, blk_T=blk_T[:3 * i.n_blocks].reshape(-1, 3))

    def batch_spinors(self, batch: int):
        """(centre, spinor index within the centre's atom) of the spinor
        functions present on a batch (Algorithm 1)."""
        n = C.c_int32()
        _check(load().q4c_grid_batch_spinors(self.h, batch, C.byref(n), None, None))
        c, m = np.zeros(max(n.value, 1), np.int32), np.zeros(max(n.value, 1), np.int32)
        _check(load().q4c_grid_batch_spinors(self.h, batch, C.byref(n), c.ctypes.data, m.ctypes.data))
        return c[:n.value], m[:n.value]

    def kpattern(self):
        """(kblk_ptr, kblk_col, kblk_off) of the atom pairs with some block (A, B, T)."""
        n = C.c_int64()
        _check(load().q4c_grid_kpattern(self.h, C.byref(n), None, None, None))
        ptr = np.zeros(self.info.n_atoms + 1, np.int64)
        _check(load().q4c_grid_kpattern(self.h, None, ptr.ctypes.data, None, None))
        col = np.zeros(max(int(ptr[-1]), 1), np.int32); off = np.zeros(int(ptr[-1]) + 1, np.int64)
        _check(load().q4c_grid_kpattern(self.h, None, None, col.ctypes.data, off.ctypes.data))
        return ptr, col[:int(ptr[-1])], off

    def status(self, stream=None):
        """Synchronise and raise Q4CError(Q4C_ETIMEOUT) if a bounded wait expired."""
        _check(load().q4c_grid_status(self.h, _stream(stream)))

    def points_device(self):
        """(xyz_ptr, w_ptr, n) device pointers owned by the grid."""
        a, b, n = C.c_void_p(), C.c_void_p(), C.c_int64()
        _check(load().q4c_grid_points(self.h, C.byref(a), C.byref(b), C.byref(n)))
        return a.value, b.value, n.value

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.q4c_grid_destroy(self.h)
            self.h = None


# --------------------------------------------------------------------------
# the five calls of the boundary
# --------------------------------------------------------------------------

def nao_tabulate(n_rad, l, alpha, r_cut=6.0, r_on=5.0, r_min=1e-4, n_log=200) -> Tables:
    return Tables(n_rad, l, alpha, r_cut, r_on, r_min, n_log)


def nao_tabulate_knots(n_rad, l, knots, r_cut=6.0, r_on=5.0, r_min=1e-4, n_log=200) -> Tables:
    return Tables(n_rad, l, None, r_cut, r_on, r_min, n_log, knots=knots)


def grid_partition(tables: Tables, xyz, species, n_rad_shells, R, n_theta, n_phi, r_nb, batch_max,
                   lattice=None, n_shell: int = 0, mol_atom_ptr=None) -> Grid:
    return Grid(tables, xyz, species, n_rad_shells, R, n_theta, n_phi, r_nb, batch_max, lattice, n_shell,
                mol_atom_ptr)


def _prec(prec) -> int:
    return PRECISIONS[prec] if isinstance(prec, str) else int(prec)


def q4c_integrate(tables: Tables, grid: Grid, v, prec="fp64", out=None, spinor: bool = False, stream=None):
    """V, W0, SOx, SOy, SOz (and the SS spinor blocks) on the block pattern."""
    import torch
    if out is None:
        out = [torch.empty(grid.nnz, dtype=torch.float64, device=v.device) for _ in range(5)]
        out.append(torch.empty(8 * grid.nnz, dtype=torch.float64, device=v.device) if spinor else None)
    m = Matrices(*[_ptr(t) for t in out[:5]], _ptr(out[5]) if len(out) > 5 else 0)
    _check(load().q4c_integrate(tables.h, grid.h, _ptr(v), _prec(prec), C.byref(m), _stream(stream)))
    return out


def q4c_integrate_noalloc(tables: Tables, grid: Grid, v, out, stream=None):
    """FP64 integration into caller-provided outputs with the library's static
    workspace (no device allocation in the call)."""
    m = Matrices(*[_ptr(t) for t in out[:5]], _ptr(out[5]) if len(out) > 5 else 0)
    _check(load().q4c_integrate_noalloc(tables.h, grid.h, _ptr(v), C.byref(m), _stream(stream)))
    return out


def q4c_density(tables: Tables, grid: Grid, P, prec="fp64", out=None, stream=None):
    import torch
    if out is None:
        out = torch.empty(grid.n_points, dtype=torch.float64, device=P.device)
    _check(load().q4c_density(tables.h, grid.h, _ptr(P), _prec(prec), _ptr(out), _stream(stream)))
    return out


def q4c_density_full(tables: Tables, grid: Grid, P: Sequence, prec="fp64", out=None, stream=None):
    """n_p = sum_M sum_ij P^M_ij f^M_ij(p) for P = [PV, PW0, PSOx, PSOy, PSOz], None = 0."""
    import torch
    dev = next(x for x in P if x is not None).device
    if out is None:
        out = torch.empty(grid.n_points, dtype=torch.float64, device=dev)
    m = Matrices(*[_ptr(x) for x in P], 0)
    _check(load().q4c_density_full(tables.h, grid.h, C.byref(m), _prec(prec), _ptr(out), _stream(stream)))
    return out


def q4c_tables_set_columns(tables: Tables, eps, knots):
    """eps [sum n_rad] and V at the radial knots [sum n_rad][n_log] of the per-column operator."""
    e = np.ascontiguousarray(eps, np.float64).reshape(-1)
    k = np.ascontiguousarray(knots, np.float64).reshape(-1)
    _check(load().q4c_tables_set_columns(tables.h, e.ctypes.data, k.ctypes.data))


def q4c_integrate_columns(tables: Tables, grid: Grid, v, prec="fp64", out=None, stream=None):
    """F_ij = sum_p w phi_i (eps_j - V_j + v) phi_j on the block pattern ("fp64" or "split")."""
    import torch
    if out is None:
        out = torch.empty(grid.nnz, dtype=torch.float64, device=v.device)
    _check(load().q4c_integrate_columns(tables.h, grid.h, _ptr(v), _prec(prec), _ptr(out), _stream(stream)))
    return out


def q4c_spinor_basis(tables: Tables, species: int):
    """(radial, kappa, two_mj) of the spinor functions of one species."""
    n = C.c_int32()
    _check(load().q4c_spinor_basis(tables.h, species, C.byref(n), None, None, None))
    rad, kap, mj = (np.zeros(n.value, np.int32) for _ in range(3))
    _check(load().q4c_spinor_basis(tables.h, species, C.byref(n), rad.ctypes.data, kap.ctypes.data, mj.ctypes.data))
    return rad, kap, mj


def q4c_tables_set_kappa(tables: Tables, kappa=None):
    """Per radial function the kappa whose spinors it carries (0: both; None: default)."""
    k = None if kappa is None else np.ascontiguousarray(kappa, np.int32)
    _check(load().q4c_tables_set_kappa(tables.h, None if k is None else k.ctypes.data))


def q4c_spinor_nnz(tables: Tables, grid: Grid) -> int:
    """Complex spinor elements of the grid's pattern (4 nnz without a kappa selection)."""
    n = C.c_int64()
    _check(load().q4c_spinor_nnz(tables.h, grid.h, C.byref(n)))
    return n.value


def q4c_spinor_transform(tables: Tables, grid: Grid, F: Sequence, large=True, small=True, stream=None):
    """(HL, HS): complex128 [spinor nnz] spinor blocks G^dagger (V x 1) G and
    G^dagger (W0 1 + i SO.sigma) G of F = [V, W0, SOx, SOy, SOz] (None = 0)."""
    import torch
    dev = next(x for x in F if x is not None).device
    ns = q4c_spinor_nnz(tables, grid)
    HL = torch.empty(ns, dtype=torch.complex128, device=dev) if large else None
    HS = torch.empty(ns, dtype=torch.complex128, device=dev) if small else None
    m = Matrices(*[_ptr(x) for x in F], 0)
    _check(load().q4c_spinor_transform(tables.h, grid.h, C.byref(m), _ptr(HL), _ptr(HS), _stream(stream)))
    return HL, HS


def q4c_spinor_density_matrices(tables: Tables, grid: Grid, D, stream=None):
    """[P^V, P^W0, P^SOx, P^SOy, P^SOz] (real [nnz]) of a spinor density matrix D
    (complex128 [4 nnz] blocks)."""
    import torch
    P = [torch.empty(grid.nnz, dtype=torch.float64, device=D.device) for _ in range(5)]
    m = Matrices(*[_ptr(x) for x in P], 0)
    _check(load().q4c_spinor_density_matrices(tables.h, grid.h, _ptr(D), C.byref(m), _stream(stream)))
    return P


def q4c_kfold(grid: Grid, H, k, out=None, stream=None):
    """H(k)_AB = sum_T exp(2 pi i k.T) H(T)_AB on the k-pattern: complex128 [n_k][nnz_k]."""
    import torch
    k = np.ascontiguousarray(k, np.float64).reshape(-1, 3)
    n = C.c_int64()
    _check(load().q4c_grid_kpattern(grid.h, C.byref(n), None, None, None))
    if out is None:
        out = torch.empty((len(k), n.value), dtype=torch.complex128, device=H.device)
    _check(load().q4c_kfold(grid.h, _ptr(H), len(k), k.ctypes.data, _ptr(out), _stream(stream)))
    return out


def q4c_integrate_backward(tables: Tables, grid: Grid, G: Sequence, prec="fp64", out=None, stream=None):
    """dL/dv for L = sum_M <G^M, M>; G = [GV, GW0, GSOx, GSOy, GSOz], None = 0."""
    import torch
    dev = next(g for g in G if g is not None).device
    if out is None:
        out = torch.empty(grid.n_points, dtype=torch.float64, device=dev)
    m = Matrices(*[_ptr(g) for g in G], 0)
    _check(load().q4c_integrate_backward(tables.h, grid.h, C.byref(m), _prec(prec), _ptr(out), _stream(stream)))
    return out


def q4c_scf_pass(tables: Tables, grid: Grid, v=None, P: Optional[Sequence] = None, G: Optional[Sequence] = None,
                 prec="fp64", H_out=None, n_out=None, dLdv_out=None, spinor: bool = False, stream=None):
    """One pass over the grid with one basis evaluation per wave: H from v (if
    v is given), the density of P = [PV, PW0, PSOx, PSOy, PSOz] (if given) and
    dL/dv of G (if given).  Returns (H list or None, n or None, dLdv or None)."""
    import torch
    ref = next((x for x in ([v] + list(P or []) + list(G or [])) if x is not None), None)
    dev = ref.device if ref is not None else torch.device("cuda", torch.cuda.current_device())
    H = None
    if v is not None:
        H = H_out if H_out is not None else [torch.empty(grid.nnz, dtype=torch.float64, device=dev) for _ in range(5)]
        if H_out is None:
            H.append(torch.empty(8 * grid.nnz, dtype=torch.float64, device=dev) if spinor else None)
    n = None
    if P is not None:
        n = n_out if n_out is not None else torch.empty(grid.n_points, dtype=torch.float64, device=dev)
    g = None
    if G is not None:
        g = dLdv_out if dLdv_out is not None else torch.empty(grid.n_points, dtype=torch.float64, device=dev)
    mH = Matrices(*[_ptr(x) for x in H[:5]], _ptr(H[5]) if len(H) > 5 else 0) if H is not None else None
    mP = Matrices(*[_ptr(x) for x in P], 0) if P is not None else None
    mG = Matrices(*[_ptr(x) for x in G], 0) if G is not None else None
    _check(load().q4c_scf_pass(tables.h, grid.h, _ptr(v), C.byref(mH) if mH else None,
                               C.byref(mP) if mP else None, _ptr(n), C.byref(mG) if mG else None, _ptr(g),
                               _prec(prec), _stream(stream)))
    return H, n, g


TILE_BUCKETS = 4


def q4c_grid_tiling(grid: Grid):
    """Per batch-size bucket of the products kernel, then the density/adjoint
    kernel (last entry): dict(nb_max, k_steps, batches, ms_one, ms_two)."""
    out = []
    for k in range(TILE_BUCKETS + 1):
        nb, ks, nbt = C.c_int32(), C.c_int32(), C.c_int64()
        m1, m2 = C.c_double(), C.c_double()
        _check(load().q4c_grid_tiling(grid.h, k, C.byref(nb), C.byref(ks), C.byref(nbt), C.byref(m1), C.byref(m2)))
        out.append(dict(nb_max=nb.value, k_steps=ks.value, batches=nbt.value, ms_one=m1.value, ms_two=m2.value))
    return out


def q4c_autotune(tables: Tables, grid: Grid, v, stream=None):
    """Choose the split path's stage shape per batch-size bucket by timing both; returns q4c_grid_tiling."""
    _check(load().q4c_autotune(tables.h, grid.h, _ptr(v), _stream(stream)))
    return q4c_grid_tiling(grid)


def q4c_grid_set_tiling(grid: Grid, bucket: int, k_steps: int):
    _check(load().q4c_grid_set_tiling(grid.h, int(bucket), int(k_steps)))


def q4c_basis_eval(tables: Tables, grid: Grid, xyz, stream=None):
    import torch
    n = xyz.shape[0]
    nb = int(grid.info.n_basis)
    phi = torch.empty((nb, n), dtype=torch.float64, device=xyz.device)
    grad = torch.empty((nb, n, 3), dtype=torch.float64, device=xyz.device)
    _check(load().q4c_basis_eval(tables.h, grid.h, n, _ptr(xyz), _ptr(phi), _ptr(grad), _stream(stream)))
    return phi, grad


def q4c_set_wait_limit_ns(ns: int):
    """Limit of the tensor kernels' bounded work waits for later launches (0: 1 s)."""
    _check(load().q4c_set_wait_limit_ns(int(ns)))


def profile(enable: bool):
    """Record CUDA events around every kernel of later compute calls."""
    _check(load().q4c_profile(1 if enable else 0))


def profile_read(prefix: str = ""):
    """(total ms, launches) of recorded kernels whose name starts with prefix."""
    ms, n = C.c_double(), C.c_int64()
    _check(load().q4c_profile_read(prefix.encode(), C.byref(ms), C.byref(n)))
    return ms.value, n.value


# --------------------------------------------------------------------------
# autograd: v -> (V, W0, SOx, SOy, SOz)
# --------------------------------------------------------------------------

def _make_function():
    import torch

    class Q4CIntegrate(torch.autograd.Function):
        """Forward: q4c_integrate.  Backward: q4c_integrate_backward with the
        incoming gradients as G (basis recomputed in the kernel)."""

        @staticmethod
        def forward(ctx, v, tables, grid, prec):
            ctx.tables, ctx.grid, ctx.prec = tables, grid, prec
            outs = q4c_integrate(tables, grid, v.contiguous(), prec)[:5]
            if _prec(prec) == Q4C_SPLIT:
                grid.status()  # a bounded wait that ran out leaves incomplete outputs: raise
            return tuple(outs)

        @staticmethod
        def backward(ctx, gV, gW, gx, gy, gz):
            G = [None if g is None else g.contiguous() for g in (gV, gW, gx, gy, gz)]
            if all(g is None for g in G):
                return None, None, None, None
            dv = q4c_integrate_backward(ctx.tables, ctx.grid, G, ctx.prec)
            if _prec(ctx.prec) == Q4C_SPLIT:
                ctx.grid.status()
            return dv, None, None, None

    return Q4CIntegrate


_fn = None


def integrate(v, tables: Tables, grid: Grid, prec="fp64"):
    """Differentiable integration: returns (V, W0, SOx, SOy, SOz).  On the
    split path forward and backward synchronise and raise Q4CError
    (Q4C_ETIMEOUT) if a bounded wait of a tensor kernel ran out."""
    global _fn
    if _fn is None:
        _fn = _make_function()
    return _fn.apply(v, tables, grid, prec)
