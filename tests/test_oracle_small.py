"""Pins of the small-component basis (Eq. 12b: phi^S = i Q(r)/r Y_(l~ m~)) as the
oracle evaluates it from radial values at the knots, with the synthetic Q
radials of the atomic-ZORA balance (Eq. 8b).  CPU only.

- the knot-value path of the oracle reproduces its (l, alpha) path exactly;
- near the nucleus Q ~ r^(l~+1) with the limit the balance fixes
  (kappa = -l-1: -2 alpha c/(2c^2 - V(0)); kappa = l: (2l+1) c/(2c^2 - V(0))),
  which pins l~ = l +- 1 and the sign of kappa;
- for one atom the overlap of the small-component functions is
  delta_(l~ l~') delta_(m~ m~') int Q_i Q_j dr (1-D quadrature of the closed form);
- with V = 0 the balance is (1/2c) sigma.p, and (2c)^2 int Q_kappa^2 dr equals
  int |grad phi^L|^2 for both kappa of a shell: the identity that links the
  paper's small component to the kinetic-balance gradients W0 (the 1 in the
  (sigma.a)(sigma.b) = a.b + i sigma.(a x b) expansion)."""

import numpy as np
import pytest
from scipy.integrate import quad

import oracle as O
from workloads import C_LIGHT, column_operator, single_atom, small_component, small_radial, water


def knots_r(wl):
    return wl.r_min * (wl.r_c / wl.r_min) ** (np.arange(wl.n_log) / (wl.n_log - 1))


def test_knot_values_reproduce_the_analytic_tabulation():
    wl = water()
    ob = O.OracleBasis(wl)
    ok = O.OracleBasis(wl, knots=ob.tab_u)
    assert np.array_equal(ok.tab_M, ob.tab_M)
    rng = np.random.default_rng(3)
    pts = wl.xyz[rng.integers(0, wl.n_atoms, 200)] + rng.normal(0, 1.5, (200, 3))
    a, ga = ob.eval(pts)
    b, gb = ok.eval(pts)
    assert np.array_equal(a, b) and np.array_equal(ga, gb)


def test_small_r_power_law_fixes_l_tilde_and_kappa():
    wl = water()
    _, Vk = column_operator(wl, 5)
    ws, Q, parent, kappa = small_component(wl, Vk)
    r = knots_r(wl)
    l_par = wl.rad_l[parent]
    a_par = wl.rad_alpha[parent]
    lt = ws.rad_l
    assert np.array_equal(lt, np.where(kappa < 0, l_par + 1, l_par - 1))
    for k in range(len(lt)):
        g = Q[k, :3] / r[:3] ** (lt[k] + 1)
        pref = C_LIGHT / (2 * C_LIGHT ** 2 - Vk[parent[k], 0])
        lim = -2 * a_par[k] * pref if kappa[k] < 0 else (2 * l_par[k] + 1) * pref
        assert abs(g[0] - lim) <= 1e-6 * abs(lim)
        assert abs(g[2] - g[0]) <= 1e-6 * abs(g[0])
        # the large component's l instead of l~ is not a power law here
        g_wrong = Q[k, :3] / r[:3] ** (l_par[k] + 1)
        assert abs(g_wrong[2] / g_wrong[0] - 1) > 1e-3


@pytest.fixture(scope="module")
def atom():
    wl = single_atom([0, 1, 2, 3], [1.4, 1.6, 1.9, 2.2], Z=3.0, n_rad=80)  # l~ up to 4
    xyz, w, _ = O.grid(wl)
    return wl, xyz, w


def test_one_atom_overlap_is_the_radial_integral(atom):
    wl, xyz, w = atom
    _, Vk = column_operator(wl, 8)
    Vk = np.zeros_like(Vk) + 0.7  # a constant V keeps Q in closed form at any r
    ws, Q, parent, kappa = small_component(wl, Vk)
    ob = O.OracleBasis(ws, knots=Q)
    pat = ob.pattern()
    S = ob.dense(ob.matrix_blocks(xyz, w, np.ones(len(w)), pat)[0], pat)
    nrad = len(parent)
    R = np.zeros((nrad, nrad))
    for i in range(nrad):
        for j in range(i, nrad):
            if ws.rad_l[i] != ws.rad_l[j]:
                continue
            f = lambda r: (small_radial(r, wl.rad_l[parent[i]], wl.rad_alpha[parent[i]], kappa[i], 0.7, wl.r_on, wl.r_c)
                           * small_radial(r, wl.rad_l[parent[j]], wl.rad_alpha[parent[j]], kappa[j], 0.7, wl.r_on,
                                          wl.r_c))
            R[i, j] = R[j, i] = quad(f, wl.r_min, wl.r_c, limit=400, epsabs=0, epsrel=1e-13)[0]
    ref = R[ob.fn_rad][:, ob.fn_rad] * (ob.fn_l[:, None] == ob.fn_l[None, :]) * (ob.fn_m[:, None] == ob.fn_m[None, :])
    # the grid integrates the natural spline of Q through 200 log knots; the
    # spline's interpolation error of Q^2 is ~1e-6 relative
    assert np.abs(S - ref).max() <= 3e-6 * np.abs(ref).max()


def test_kinetic_identity_links_q_to_the_gradients(atom):
    wl, xyz, w = atom
    _, Vk = column_operator(wl, 9)
    ws, Q, parent, kappa = small_component(wl, 0 * Vk)
    oS = O.OracleBasis(ws, knots=Q)
    oL = O.OracleBasis(wl)
    one = np.ones(len(w))
    SS = oS.dense(oS.matrix_blocks(xyz, w, one, oS.pattern())[0], oS.pattern())
    patL = oL.pattern()
    W0 = oL.dense(oL.matrix_blocks(xyz, w, one, patL)[1], patL)
    for k in range(len(parent)):
        iS = int(np.flatnonzero(oS.fn_rad == k)[0])
        iL = int(np.flatnonzero(oL.fn_rad == parent[k])[0])
        lhs = (2 * C_LIGHT) ** 2 * SS[iS, iS]
        # both sides integrate splines of different functions (Q, and P with
        # its derivative): ~1e-6 relative apart
        assert abs(lhs - W0[iL, iL]) <= 5e-6 * W0[iL, iL], (k, lhs, W0[iL, iL])
    # dropping the kappa P/r term breaks it for l >= 1
    k = int(np.flatnonzero(wl.rad_l[parent] >= 1)[0])
    r = np.linspace(1e-3, wl.r_c, 20001)
    l, a = wl.rad_l[parent[k]], wl.rad_alpha[parent[k]]
    dP_only = small_radial(r, l, a, 0, 0.0, wl.r_on, wl.r_c)
    full = small_radial(r, l, a, kappa[k], 0.0, wl.r_on, wl.r_c)
    assert abs(np.trapezoid(dP_only ** 2, r) / np.trapezoid(full ** 2, r) - 1) > 1e-2
