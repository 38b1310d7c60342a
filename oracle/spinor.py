"""Scalar -> spinor transformation of the Q4C method, plain numpy.

Test infrastructure (part of the oracle): only tests/, __graft_entry__.smoke()
and bench.py use it.  It shares no code with the library.

What it follows:
* Section II, Eqs. 9-11: the spinor basis chi_mu of an atom-centred radial
  function with angular momentum l has kappa = -l-1 (j = l + 1/2) and, for
  l > 0, kappa = l (j = l - 1/2), m_j = -j..j; its large component couples
  the complex harmonics Y~_l^(m_j -+ 1/2) with the spin functions through
  the coefficients C_alpha, C_beta.
* Appendix A: C_alpha = <l, m_j - 1/2; 1/2, +1/2 | j m_j>,
  C_beta = <l, m_j + 1/2; 1/2, -1/2 | j m_j>, computed here from the Racah
  formula (not from the closed form of Eq. 10).
* Eq. 13 and Appendix B: the complex harmonics as combinations of the real
  ones.  Reading (see `complex_harmonic_in_real`): Y~ are the complex
  harmonics with the Condon-Shortley phase, the convention the paper names;
  the phases printed in Eq. 13, applied to the real harmonics of Appendix B,
  give (-1)^m times them, and with those the coupled functions are not
  eigenfunctions of j (tests/test_oracle_spinor.py shows both).
* Eq. 14: chi_mu = sum_t G_(t s),mu phi_t eta_s, G block-diagonal per
  radial shell (rows: scalar function t and spin s, interleaved as 2t + s).
* Eqs. 33-34: F~_mu,nu = sum_ab conj(G_a,mu) F_ab G_b,nu for an operator
  given in the scalar-spin basis (F_ab = V_ij delta_ss' for the large
  component; the 2 x 2 blocks of Eq. 16 for the kinetic-balance small
  component).
* Eqs. 37-38: the reverse map D'_ab = sum_mu,nu conj(G_a,mu) D_mu,nu G_b,nu and
  the density n = Re sum_ab D'_ab chi-products, i.e. the real scalar density
  matrices P^V = P^W0 = Re tr_s D'_ij and P^SOk = Re(i sum_ss' (sigma_k)_ss' D'_(is)(js')).
* Algorithm 1: the local-to-global spinor index map of a set of local scalar
  functions.
* Eqs. 11-12b, 14: the small component of spinor (kappa, m_j) is
  i Q(r)/r Upsilon_(-kappa, m_j); a basis of Q radials carries, per radial,
  the spinors of one kappa~ = -kappa (`kappas` below), so its G is G^S of
  Eq. 14 and G^S^dagger (F^S x 1) G^S is the SS block of Eq. 19.
"""
from __future__ import annotations

import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

SQ2 = math.sqrt(2.0)
PAULI = (np.array([[0, 1], [1, 0]], complex), np.array([[0, -1j], [1j, 0]], complex),
         np.array([[1, 0], [0, -1]], complex))


def clebsch_gordan(j1x2: int, m1x2: int, j2x2: int, m2x2: int, Jx2: int, Mx2: int) -> float:
    """<j1 m1; j2 m2 | J M> by the Racah formula; all arguments doubled (2j, 2m)."""
    if m1x2 + m2x2 != Mx2 or abs(m1x2) > j1x2 or abs(m2x2) > j2x2 or abs(Mx2) > Jx2:
        return 0.0
    if Jx2 < abs(j1x2 - j2x2) or Jx2 > j1x2 + j2x2 or (j1x2 + j2x2 + Jx2) % 2:
        return 0.0
    f = math.factorial

    def h(x2):  # (x2 / 2) as an integer, x2 even
        assert x2 % 2 == 0, x2
        return x2 // 2

    pref = math.sqrt((Jx2 + 1) * f(h(j1x2 + j2x2 - Jx2)) * f(h(j1x2 - j2x2 + Jx2)) * f(h(-j1x2 + j2x2 + Jx2))
                     / f(h(j1x2 + j2x2 + Jx2 + 2)))
    pref *= math.sqrt(f(h(j1x2 + m1x2)) * f(h(j1x2 - m1x2)) * f(h(j2x2 + m2x2)) * f(h(j2x2 - m2x2))
                      * f(h(Jx2 + Mx2)) * f(h(Jx2 - Mx2)))
    s = 0.0
    for k in range(0, h(j1x2 + j2x2 + Jx2) + 1):
        args = (k, h(j1x2 + j2x2 - Jx2) - k, h(j1x2 - m1x2) - k, h(j2x2 + m2x2) - k,
                h(Jx2 - j2x2 + m1x2) + k, h(Jx2 - j1x2 - m2x2) + k)
        if min(args) < 0:
            continue
        d = 1
        for a in args:
            d *= f(a)
        s += (-1) ** k / d
    return pref * s


def complex_harmonic_in_real(l: int, m: int, phase: str = "cs") -> Dict[int, complex]:
    """Coefficients c_m' with Y~_l^m = sum_m' c_m' Y_(l,m') (Y_(l,m') the real
    harmonics of Appendix B, for which Y_(l,|m|) + i Y_(l,-|m|) = sqrt(2) Y_l^|m|
    with scipy's Condon-Shortley Y).  phase "cs": Y~ with the Condon-Shortley
    phase; "eq13": the phases as printed in Eq. 13 (used only to show that
    they break the coupling)."""
    if m == 0:
        return {0: 1.0 + 0j}
    a = abs(m)
    if phase == "cs":
        if m > 0:
            return {a: 1 / SQ2, -a: 1j / SQ2}
        return {a: (-1) ** a / SQ2, -a: -1j * (-1) ** a / SQ2}
    if m > 0:  # Eq. 13 as printed
        return {a: (-1) ** m / SQ2, -a: 1j * (-1) ** m / SQ2}
    return {a: 1 / SQ2, -a: -1j / SQ2}


def spinor_functions(l_list: Sequence[int], kappas: Optional[Sequence[int]] = None
                     ) -> List[Tuple[int, int, int, int, int]]:
    """(radial q, l, 2j, 2m_j, kappa) of one atom's spinor functions: per radial
    function in order, j = l - 1/2 (kappa = l, only for l > 0) then j = l + 1/2
    (kappa = -l - 1), m_j ascending (Eqs. 9-11).  kappas[q] != 0 keeps only
    that kappa of radial q (its j = |kappa| - 1/2)."""
    out = []
    for q, l in enumerate(l_list):
        for jx2 in ((2 * l - 1, 2 * l + 1) if l > 0 else (1,)):
            kappa = l if jx2 == 2 * l - 1 else -l - 1
            if kappas is not None and kappas[q] != 0 and kappas[q] != kappa:
                continue
            for mjx2 in range(-jx2, jx2 + 1, 2):
                out.append((q, l, jx2, mjx2, kappa))
    return out


def transformation_matrix(l_list: Sequence[int], phase: str = "cs",
                          kappas: Optional[Sequence[int]] = None) -> np.ndarray:
    """G of one atom (Eq. 14): (2 n_fn, n_spinor) complex, rows 2t + s (scalar
    function t in radial-then-m order, spin s = 0 up, 1 down), columns the
    spinor functions of `spinor_functions` (n_spinor = 2 n_fn without kappas)."""
    first, t0 = [], 0
    for l in l_list:
        first.append(t0)
        t0 += 2 * l + 1
    n = t0
    fns = spinor_functions(l_list, kappas)
    G = np.zeros((2 * n, len(fns)), complex)
    for mu, (q, l, jx2, mjx2, _) in enumerate(fns):
        for s, msx2 in ((0, 1), (1, -1)):
            mlx2 = mjx2 - msx2  # m_l = m_j - m_s
            if abs(mlx2) > 2 * l:
                continue
            cg = clebsch_gordan(2 * l, mlx2, 1, msx2, jx2, mjx2)
            for mr, c in complex_harmonic_in_real(l, mlx2 // 2, phase).items():
                t = first[q] + mr + l
                G[2 * t + s, mu] += cg * c
    return G


def atom_matrices(wl, phase: str = "cs", kappas: Optional[Sequence[int]] = None) -> List[np.ndarray]:
    """G of each atom of a workload; kappas: per radial function, species-major
    (the selection of `spinor_functions`)."""
    per_species, r0 = [], 0
    for sp in wl.species:
        ks = None if kappas is None else list(kappas[r0:r0 + len(sp.l)])
        per_species.append(transformation_matrix(sp.l, phase, ks))
        r0 += len(sp.l)
    return [per_species[s] for s in wl.species_of_atom]


def scalar_spin_large(V: np.ndarray) -> np.ndarray:
    """F_(is),(js') = V_ij delta_ss' (interleaved 2i + s)."""
    return np.kron(V, np.eye(2))


def scalar_spin_small(W0, SOx, SOy, SOz) -> np.ndarray:
    """The kinetic-balance small-component operator per scalar pair, the 2 x 2
    block [[W0 + i SOz, SOy + i SOx], [-SOy + i SOx, W0 - i SOz]] = W0 1 + i SO.sigma."""
    out = np.kron(W0, np.eye(2)).astype(complex)
    for S, P in zip((SOx, SOy, SOz), PAULI):
        out += 1j * np.kron(S, P)
    return out


def transform_blocks(F2: Sequence[np.ndarray], pat, Gs: Sequence[np.ndarray], nf) -> List[np.ndarray]:
    """F~ = G_A^dagger F G_B for every pattern block (A, B, T) (Eqs. 33-34);
    F2[q] is block q in the scalar-spin basis."""
    out = []
    for A in range(len(pat.blk_ptr) - 1):
        for q in range(int(pat.blk_ptr[A]), int(pat.blk_ptr[A + 1])):
            B = int(pat.blk_col[q])
            out.append(Gs[A].conj().T @ F2[q] @ Gs[B])
    return out


def blocks_of(vals, pat, nf) -> List[np.ndarray]:
    """Dense (nf_A, nf_B) blocks of a pattern array, in pattern order."""
    out = []
    for A in range(len(pat.blk_ptr) - 1):
        for q in range(int(pat.blk_ptr[A]), int(pat.blk_ptr[A + 1])):
            B = int(pat.blk_col[q])
            o = int(pat.blk_off[q])
            out.append(np.asarray(vals[o:o + nf[A] * nf[B]]).reshape(nf[A], nf[B]))
    return out


def scalar_density_matrices(D: Sequence[np.ndarray], pat, Gs: Sequence[np.ndarray], nf):
    """Eqs. 37-38: per block D'_ab = sum conj(G_a,mu) D_mu,nu G_b,nu, then the real
    scalar matrices (P^V, P^W0, P^SOx, P^SOy, P^SOz) as flat pattern arrays."""
    nnz = int(pat.blk_off[-1])
    P = [np.zeros(nnz) for _ in range(5)]
    q = 0
    for A in range(len(pat.blk_ptr) - 1):
        for qq in range(int(pat.blk_ptr[A]), int(pat.blk_ptr[A + 1])):
            B = int(pat.blk_col[qq])
            Dp = Gs[A].conj() @ D[q] @ Gs[B].T
            Dp4 = Dp.reshape(nf[A], 2, nf[B], 2)  # [i, s, j, s']
            tr = Dp4[:, 0, :, 0] + Dp4[:, 1, :, 1]
            o = int(pat.blk_off[qq])
            n = nf[A] * nf[B]
            P[0][o:o + n] = tr.real.reshape(-1)
            P[1][o:o + n] = tr.real.reshape(-1)
            for k, S in enumerate(PAULI):
                val = 1j * np.einsum("isjt,st->ij", Dp4, S)
                P[2 + k][o:o + n] = val.real.reshape(-1)
            q += 1
    return P


def batch_spinors(local_fns: Sequence[int], fn_shell: Sequence[int], shell_spinors: Dict[int, List[int]]):
    """Algorithm 1 for one set of local scalar functions: a global spinor
    function is present when one of the scalar functions of its relation-table
    entry (its radial shell, here identified by fn_shell) is local; returns the
    local-to-global spinor index array in ascending global order."""
    local_shells = {fn_shell[i] for i in local_fns}
    out = []
    for sh in sorted(shell_spinors):
        if sh in local_shells:
            out.extend(shell_spinors[sh])
    return out
