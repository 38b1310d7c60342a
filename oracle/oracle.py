"""ctypes wrapper of the plain C oracle (q4c_oracle.c).  Test infrastructure.

Every function forwards to the C routine of the same name; the docstrings
name the passage of the paper each one follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "q4c_oracle.c")
_SO = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib: Optional[C.CDLL] = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Basis(C.Structure):
    _fields_ = [
        ("n_atoms", C.c_int), ("xyz", C.c_void_p), ("species", C.c_void_p),
        ("n_species", C.c_int), ("n_rad", C.c_void_p), ("rad_l", C.c_void_p), ("rad_alpha", C.c_void_p),
        ("n_log", C.c_int), ("r_min", C.c_double), ("r_c", C.c_double), ("r_on", C.c_double),
        ("tab_u", C.c_void_p), ("tab_M", C.c_void_p), ("analytic", C.c_int),
        ("lattice", C.c_void_p), ("n_shell", C.c_int),
    ]


def lib() -> C.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_gauss_legendre.argtypes = [C.c_int, _dp, _dp]
            L.orc_radial_shells.argtypes = [C.c_int, C.c_double, _dp, _dp]
            L.orc_cutoff.argtypes = [C.c_double, C.c_double, C.c_double]
            L.orc_cutoff.restype = C.c_double
            L.orc_tabulate.argtypes = [C.c_int, C.c_double, C.c_int, C.c_double, C.c_double, C.c_double,
                                       _dp, _dp, _dp]
            L.orc_spline_second.argtypes = [C.c_int, _dp, _dp]
            L.orc_spline_eval.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, _dp, _dp, C.c_double,
                                          C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.orc_K.argtypes = [C.c_int, C.c_int]
            L.orc_K.restype = C.c_double
            L.orc_ylm_spherical.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double]
            L.orc_ylm_spherical.restype = C.c_double
            L.orc_solid_harmonic.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                             C.POINTER(C.c_double), _dp]
            bp = C.POINTER(_Basis)
            L.orc_count_functions.argtypes = [bp]
            L.orc_function_table.argtypes = [bp, _ip, _ip, _ip, _ip]
            L.orc_basis_eval.argtypes = [bp, C.c_int, _dp, C.c_int, _ip, _dp, _dp]
            L.orc_becke_weight.argtypes = [C.c_int, _dp, C.c_int, _dp, C.c_double]
            L.orc_becke_weight.restype = C.c_double
            L.orc_partition_weight.argtypes = [C.c_int, _dp, C.c_int, _dp, C.c_double, C.c_int]
            L.orc_partition_weight.restype = C.c_double
            L.orc_grid.argtypes = [C.c_int, _dp, C.c_int, C.c_double, C.c_int, C.c_int, C.c_double,
                                   C.c_double, C.c_longlong, _dp, _dp, _lp]
            L.orc_grid.restype = C.c_long
            L.orc_grid_cell.argtypes = [C.c_int, _dp, C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_int,
                                        C.c_int, C.c_double, C.c_double, C.c_int, C.c_longlong, _dp, _dp, _lp]
            L.orc_grid_cell.restype = C.c_long
            L.orc_grid_near.argtypes = [C.c_int, _dp, C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_int,
                                        C.c_int, C.c_double, C.c_double, C.c_int, C.c_int, _dp, C.c_long,
                                        _dp, _dp, _lp]
            L.orc_grid_near.restype = C.c_long
            L.orc_pattern.argtypes = [bp, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_pattern.restype = C.c_long
            L.orc_matrix_pairs.argtypes = [bp, C.c_long, _dp, _dp, _dp, C.c_long, _ip, _ip,
                                           _dp, _dp, _dp, _dp, _dp]
            L.orc_matrix_entries.argtypes = [bp, C.c_long, _dp, _dp, _dp, C.c_long, _ip, _ip, _ip, _ip, _ip,
                                             _dp, _dp, _dp, _dp, _dp]
            L.orc_matrix_blocks.argtypes = [bp, C.c_long, _dp, _dp, _dp, _lp, _ip, _ip, _lp,
                                            _dp, _dp, _dp, _dp, _dp]
            L.orc_matrix_blocks.restype = C.c_int
            L.orc_density.argtypes = [bp, C.c_long, _dp, _lp, _ip, _ip, _lp, _dp, _dp]
            vp = C.c_void_p
            L.orc_adjoint.argtypes = [bp, C.c_long, _dp, _dp, _lp, _ip, _ip, _lp, vp, vp, vp, vp, vp, _dp]
            L.orc_spinor_ss.argtypes = [bp, _lp, _ip, _lp, _dp, _dp, _dp, _dp, _dp]
            L.orc_matrix_columns.argtypes = [bp, C.c_long, _dp, _dp, _dp, _dp, _dp, _lp, _ip, _ip, _lp, _dp]
            L.orc_matrix_columns.restype = None
            L.orc_kpattern.argtypes = [bp, _lp, _ip, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_kpattern.restype = C.c_long
            L.orc_kfold.argtypes = [bp, _lp, _ip, _ip, _lp, _dp, C.c_int, _dp, _lp, _ip, _lp, _dp]
            _lib = L
        return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# quadrature and radial pieces
# --------------------------------------------------------------------------

def gauss_legendre(n: int):
    x = np.zeros(n); w = np.zeros(n)
    lib().orc_gauss_legendre(n, x, w)
    return x, w


def radial_shells(N: int, R: float = 1.0):
    """Gauss-Chebyshev (2nd kind) shells with Becke's map (integrates F(r) r^2 dr)."""
    r = np.zeros(N); w = np.zeros(N)
    lib().orc_radial_shells(N, R, r, w)
    return r, w


def cutoff(r: float, r_on: float = 5.0, r_c: float = 6.0) -> float:
    return lib().orc_cutoff(r, r_on, r_c)


def tabulate(l: int, alpha: float, n: int = 200, r_min: float = 1e-4, r_c: float = 6.0, r_on: float = 5.0):
    """Knots, knot values u_k and natural-spline second derivatives (Eq. 12 radial)."""
    r = np.zeros(n); u = np.zeros(n); M = np.zeros(n)
    rc = lib().orc_tabulate(l, alpha, n, r_min, r_c, r_on, r, u, M)
    if rc != 0:
        raise ValueError("tabulate failed")
    return r, u, M


def spline_eval(l: int, u: np.ndarray, M: np.ndarray, r: float, r_min: float = 1e-4, r_c: float = 6.0):
    a = C.c_double(); b = C.c_double()
    lib().orc_spline_eval(l, len(u), r_min, r_c, _f64(u), _f64(M), r, C.byref(a), C.byref(b))
    return a.value, b.value


def K_lm(l: int, m: int) -> float:
    return lib().orc_K(l, m)


def ylm_spherical(l: int, m: int, theta: float, phi: float) -> float:
    """Y_l^m from Eqs. B1-B3 in spherical coordinates."""
    return lib().orc_ylm_spherical(l, m, theta, phi)


def solid_harmonic(l: int, m: int, x: float, y: float, z: float):
    """S_lm = r^l Y_lm and its Cartesian gradient."""
    S = C.c_double(); dS = np.zeros(3)
    lib().orc_solid_harmonic(l, m, x, y, z, C.byref(S), dS)
    return S.value, dS


def becke_weight(centres: np.ndarray, owner: int, p, r_nb: float = 1e300) -> float:
    c = _f64(centres).reshape(-1)
    return lib().orc_becke_weight(len(c) // 3, c, owner, _f64(p), r_nb)


PARTITIONS = {"becke": 0, "stratmann": 1}


def partition_weight(centres: np.ndarray, owner: int, p, r_nb: float = 1e300, scheme: str = "becke") -> float:
    """p_owner(r) with Becke's (1988) or Stratmann, Scuseria and Frisch's (1996) cell function."""
    c = _f64(centres).reshape(-1)
    return lib().orc_partition_weight(len(c) // 3, c, owner, _f64(p), r_nb, PARTITIONS[scheme])


def grid(wl, stride: int = 1):
    """Kept grid points of a workload: (xyz (n,3), w (n,), raw id (n,)).
    stride > 1 evaluates only the raw points whose id is a multiple of it.
    A periodic workload (wl.lattice set) partitions over the atoms' images too."""
    n_raw = (wl.n_raw_points + stride - 1) // stride
    xyz = np.zeros(3 * n_raw); w = np.zeros(n_raw); ids = np.zeros(n_raw, dtype=np.int64)
    lat = None if wl.lattice is None else _f64(wl.lattice).reshape(-1)
    n = lib().orc_grid_cell(wl.n_atoms, _f64(wl.xyz).reshape(-1), None if lat is None else lat.ctypes.data,
                            wl.n_shell, wl.n_rad, wl.R, wl.n_theta, wl.n_phi, wl.r_c, wl.r_nb,
                            PARTITIONS[wl.partition], stride, xyz, w, ids)
    return xyz[:3 * n].reshape(n, 3).copy(), w[:n].copy(), ids[:n].copy()


def centres(wl) -> np.ndarray:
    """Positions of the atoms and, in a periodic cell, their images in the
    oracle's centre order (cell-major, T lexicographic in [-n_shell, n_shell]^3)."""
    if wl.lattice is None:
        return _f64(wl.xyz).reshape(-1, 3).copy()
    s = wl.n_shell
    L = _f64(wl.lattice).reshape(3, 3)
    T = np.array([(a, b, c) for a in range(-s, s + 1) for b in range(-s, s + 1) for c in range(-s, s + 1)],
                 dtype=np.float64)
    return ((T @ L)[:, None, :] + _f64(wl.xyz).reshape(1, -1, 3)).reshape(-1, 3)


def grid_near(wl, targets):
    """The kept grid points (stride 1) within r_c of at least one target
    position: (xyz, w, raw id), the same points and weights as grid(wl)
    restricted to them, in raw id order."""
    targets = _f64(targets).reshape(-1, 3)
    # buffer bound: the raw points of atoms within r_c + r_nb of a target
    d = np.linalg.norm(_f64(wl.xyz).reshape(-1, 1, 3) - targets[None], axis=2)
    cap = max(1, int((d < wl.r_c + wl.r_nb).any(axis=1).sum()) * wl.n_rad * wl.n_theta * wl.n_phi)
    xyz = np.zeros(3 * cap); w = np.zeros(cap); ids = np.zeros(cap, dtype=np.int64)
    lat = None if wl.lattice is None else _f64(wl.lattice).reshape(-1)
    n = lib().orc_grid_near(wl.n_atoms, _f64(wl.xyz).reshape(-1), None if lat is None else lat.ctypes.data,
                            wl.n_shell, wl.n_rad, wl.R, wl.n_theta, wl.n_phi, wl.r_c, wl.r_nb,
                            PARTITIONS[wl.partition], len(targets), targets.reshape(-1), cap, xyz, w, ids)
    if n > cap:
        raise RuntimeError("grid_near: buffer bound exceeded")
    return xyz[:3 * n].reshape(n, 3).copy(), w[:n].copy(), ids[:n].copy()


# --------------------------------------------------------------------------
# basis, pattern, matrices
# --------------------------------------------------------------------------

class Pattern:
    """CSR block pattern over atoms: block (A, B, T) iff |R_A - R_B - T.L| < 2 r_c
    (T = 0 for a molecule); blk_T holds the integer shifts, [n_blocks][3]."""

    def __init__(self, blk_ptr, blk_col, blk_off, blk_T=None):
        self.blk_ptr = blk_ptr
        self.blk_col = blk_col
        self.blk_off = blk_off
        self.blk_T = (np.zeros((len(blk_col), 3), np.int32) if blk_T is None
                      else np.ascontiguousarray(blk_T, np.int32).reshape(-1, 3))

    @property
    def nnz(self) -> int:
        return int(self.blk_off[-1])


class OracleBasis:
    """Basis of a workload with radial tables built by the oracle itself."""

    def __init__(self, wl, analytic: bool = False, knots: Optional[np.ndarray] = None):
        """knots [n_rad_tot][n_log]: radial values u(r_k) at the knots instead of
        r^(l+1) exp(-alpha r^2) c(r) (the small-component Q radials, Eq. 12b)."""
        self.wl = wl
        self._xyz = _f64(wl.xyz).reshape(-1)
        self._species = np.ascontiguousarray(wl.species_of_atom, dtype=np.int32)
        self._n_rad = wl.n_rad_per_species
        self._l = wl.rad_l
        self._alpha = wl.rad_alpha
        nr = len(self._l)
        self.tab_r = np.zeros((nr, wl.n_log)); self.tab_u = np.zeros((nr, wl.n_log))
        self.tab_M = np.zeros((nr, wl.n_log))
        for k in range(nr):
            if knots is None:
                r, u, M = tabulate(int(self._l[k]), float(self._alpha[k]), wl.n_log, wl.r_min, wl.r_c, wl.r_on)
            else:
                if analytic:
                    raise ValueError("knot values and the analytic radial exclude each other")
                r = wl.r_min * (wl.r_c / wl.r_min) ** (np.arange(wl.n_log) / (wl.n_log - 1))
                u = _f64(knots[k]).copy(); M = np.zeros(wl.n_log)
                lib().orc_spline_second(wl.n_log, u, M)
            self.tab_r[k] = r; self.tab_u[k] = u; self.tab_M[k] = M
        self._lat = None if wl.lattice is None else _f64(wl.lattice).reshape(-1)
        self.s = _Basis(wl.n_atoms, self._xyz.ctypes.data, self._species.ctypes.data, len(wl.species),
                        self._n_rad.ctypes.data, self._l.ctypes.data, self._alpha.ctypes.data, wl.n_log,
                        wl.r_min, wl.r_c, wl.r_on, self.tab_u.ctypes.data, self.tab_M.ctypes.data,
                        1 if analytic else 0, None if self._lat is None else self._lat.ctypes.data,
                        wl.n_shell)
        self.n_fn = lib().orc_count_functions(C.byref(self.s))
        self.fn_atom = np.zeros(self.n_fn, np.int32); self.fn_rad = np.zeros(self.n_fn, np.int32)
        self.fn_l = np.zeros(self.n_fn, np.int32); self.fn_m = np.zeros(self.n_fn, np.int32)
        lib().orc_function_table(C.byref(self.s), self.fn_atom, self.fn_rad, self.fn_l, self.fn_m)

    def eval(self, pts: np.ndarray, fns: Optional[Sequence[int]] = None):
        """phi (n_fn, n_pts) and grad (n_fn, n_pts, 3) at points."""
        pts = _f64(pts).reshape(-1, 3)
        fns = np.arange(self.n_fn, dtype=np.int32) if fns is None else np.ascontiguousarray(fns, np.int32)
        phi = np.zeros(len(fns) * len(pts)); grad = np.zeros(len(fns) * len(pts) * 3)
        lib().orc_basis_eval(C.byref(self.s), len(pts), pts.reshape(-1), len(fns), fns, phi, grad)
        return phi.reshape(len(fns), len(pts)), grad.reshape(len(fns), len(pts), 3)

    def pattern(self) -> Pattern:
        nb = lib().orc_pattern(C.byref(self.s), None, None, None, None)
        ptr = np.zeros(self.wl.n_atoms + 1, np.int64); col = np.zeros(max(nb, 1), np.int32)
        T = np.zeros(3 * max(nb, 1), np.int32); off = np.zeros(nb + 1, np.int64)
        lib().orc_pattern(C.byref(self.s), ptr.ctypes.data, col.ctypes.data, T.ctypes.data, off.ctypes.data)
        return Pattern(ptr, col[:nb].copy(), off, T[:3 * nb].copy())

    def matrix_pairs(self, xyz, w, v, pi, pj):
        """V, W0, SOx, SOy, SOz at listed (i, j) pairs (Eqs. 29-30 + the SS reading)."""
        xyz = _f64(xyz).reshape(-1); w = _f64(w); v = _f64(v)
        pi = np.ascontiguousarray(pi, np.int32); pj = np.ascontiguousarray(pj, np.int32)
        outs = [np.zeros(len(pi)) for _ in range(5)]
        lib().orc_matrix_pairs(C.byref(self.s), len(w), xyz, w, v, len(pi), pi, pj, *outs)
        return outs

    def matrix_entries(self, xyz, w, v, A, B, T, i, j):
        """V, W0, SOx, SOy, SOz at listed elements (i, j) (local function
        indices) of blocks (A, B, T), periodic images included (Eqs. 24-25,
        29-30 and the SS reading)."""
        xyz = _f64(xyz).reshape(-1); w = _f64(w); v = _f64(v)
        ia = lambda x: np.ascontiguousarray(x, np.int32).reshape(-1)
        A, B, i, j = ia(A), ia(B), ia(i), ia(j)
        T = np.ascontiguousarray(T, np.int32).reshape(-1, 3)
        outs = [np.zeros(len(A)) for _ in range(5)]
        lib().orc_matrix_entries(C.byref(self.s), len(w), xyz, w, v, len(A), A, B, T.reshape(-1), i, j, *outs)
        return outs

    def matrix_blocks(self, xyz, w, v, pat: Pattern):
        """Full V, W0, SOx, SOy, SOz on the block pattern."""
        xyz = _f64(xyz).reshape(-1); w = _f64(w); v = _f64(v)
        outs = [np.zeros(pat.nnz) for _ in range(5)]
        miss = lib().orc_matrix_blocks(C.byref(self.s), len(w), xyz, w, v, pat.blk_ptr, pat.blk_col,
                                       pat.blk_T.reshape(-1), pat.blk_off, *outs)
        if miss:
            raise RuntimeError("active atom pair outside the block pattern")
        return outs

    def matrix_columns(self, xyz, w, v, eps, knots, pat: Pattern):
        """F_ij = sum_p w phi_i (eps_j - V_j(|p - R_j|) + v) phi_j (Eq. 19, large component,
        per-column operator): eps [n_rad_tot], knots [n_rad_tot][n_log] values of V at the
        radial knots; flat array on the block pattern (not symmetric)."""
        xyz = _f64(xyz).reshape(-1); w = _f64(w); v = _f64(v)
        out = np.zeros(pat.nnz)
        lib().orc_matrix_columns(C.byref(self.s), len(w), xyz, w, v, _f64(eps), _f64(knots).reshape(-1),
                                 pat.blk_ptr, pat.blk_col, pat.blk_T.reshape(-1), pat.blk_off, out)
        return out

    def density(self, xyz, P, pat: Pattern):
        """n_p = sum_ij P_ij phi_i phi_j (Eqs. 39-40)."""
        xyz = _f64(xyz).reshape(-1)
        n = np.zeros(len(xyz) // 3)
        lib().orc_density(C.byref(self.s), len(n), xyz, pat.blk_ptr, pat.blk_col, pat.blk_T.reshape(-1),
                          pat.blk_off, _f64(P), n)
        return n

    def adjoint(self, xyz, w, G, pat: Pattern):
        """dL/dv_p for L = sum_M <G^M, M>, G = [GV, GW0, GSOx, GSOy, GSOz] (None = 0)."""
        xyz = _f64(xyz).reshape(-1); w = _f64(w)
        keep = [None if g is None else _f64(g) for g in G]
        ptrs = [None if g is None else g.ctypes.data for g in keep]
        out = np.zeros(len(w))
        lib().orc_adjoint(C.byref(self.s), len(w), xyz, w, pat.blk_ptr, pat.blk_col, pat.blk_T.reshape(-1),
                          pat.blk_off, *ptrs, out)
        return out

    def density_full(self, xyz, P, pat: Pattern):
        """n_p = sum_M sum_ij P^M_ij f^M_ij(p), P = [PV, PW0, PSOx, PSOy, PSOz] (None = 0):
        the density with the gradient terms, i.e. the adjoint's sum with unit weights."""
        n = len(_f64(xyz).reshape(-1)) // 3
        return self.adjoint(xyz, np.ones(n), P, pat)

    def spinor_ss(self, W0, SOx, SOy, SOz, pat: Pattern):
        """Complex SS spinor blocks (Eq. 16, kinetic-balance reading), complex128 [4*nnz]."""
        out = np.zeros(8 * pat.nnz)
        lib().orc_spinor_ss(C.byref(self.s), pat.blk_ptr, pat.blk_col, pat.blk_off, _f64(W0), _f64(SOx),
                            _f64(SOy), _f64(SOz), out)
        return out.view(np.complex128)

    def kpattern(self, pat: Pattern):
        """(kblk_ptr, kblk_col, kblk_off): the atom pairs with some block (A, B, T)."""
        nkb = lib().orc_kpattern(C.byref(self.s), pat.blk_ptr, pat.blk_col, None, None, None)
        ptr = np.zeros(self.wl.n_atoms + 1, np.int64); col = np.zeros(max(nkb, 1), np.int32)
        off = np.zeros(nkb + 1, np.int64)
        lib().orc_kpattern(C.byref(self.s), pat.blk_ptr, pat.blk_col, ptr.ctypes.data, col.ctypes.data,
                           off.ctypes.data)
        return ptr, col[:nkb].copy(), off

    def kfold(self, H, k, pat: Pattern):
        """H(k)_AB = sum_T exp(2 pi i k.T) H(T)_AB (Eqs. 24-26), k [n_k][3] reduced
        coordinates; complex128 [n_k][nnz_k] on the k-pattern."""
        kptr, kcol, koff = self.kpattern(pat)
        k = _f64(k).reshape(-1, 3)
        out = np.zeros(2 * len(k) * int(koff[-1]))
        lib().orc_kfold(C.byref(self.s), pat.blk_ptr, pat.blk_col, pat.blk_T.reshape(-1), pat.blk_off, _f64(H),
                        len(k), k.reshape(-1), kptr, kcol, koff, out)
        return out.view(np.complex128).reshape(len(k), -1)

    def dense(self, vals, pat: Pattern) -> np.ndarray:
        """Scatter a block-pattern array into a dense n_fn x n_fn matrix."""
        nf = self.wl.nf_of_atom
        first = np.concatenate([[0], np.cumsum(nf)])
        D = np.zeros((self.n_fn, self.n_fn))
        for A in range(self.wl.n_atoms):
            for q in range(int(pat.blk_ptr[A]), int(pat.blk_ptr[A + 1])):
                B = int(pat.blk_col[q])
                o = int(pat.blk_off[q])
                D[first[A]:first[A + 1], first[B]:first[B + 1]] = \
                    np.asarray(vals[o:o + nf[A] * nf[B]]).reshape(nf[A], nf[B])
        return D
