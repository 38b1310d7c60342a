"""Pins of the oracle's Stratmann partition (Stratmann, Scuseria and Frisch
1996; the partition the paper names, Section III A), fixed by what the
cell function must satisfy rather than by retyping its polynomial:
exactly 1 and 0 beyond |mu| = 0.64, one half at the midpoint, antisymmetry
s(mu) + s(-mu) = 1, a C^3 join at |mu| = 0.64, monotone decrease, partition
of unity over many centres, and the closed-form Gaussian overlap and kinetic
integrals of two centres integrated on a grid weighted with it.  CPU only."""
import dataclasses
import math

import numpy as np

import oracle as O
from workloads import Species, Workload

A_CUT = 0.64


def _s(mu):
    """Two-centre weight of centre A at a point with mu_AB = mu (R = 2 on the z axis)."""
    centres = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 2.0]])
    # |p - A| - |p - B| = 2 mu at z = 1 + mu, x = y = 0 (on the axis between the centres)
    p = np.array([0.0, 0.0, 1.0 + mu])
    return O.partition_weight(centres, 0, p, scheme="stratmann")


def test_stratmann_limits_midpoint_and_antisymmetry():
    for mu in (-0.99, -0.8, -0.65, -0.6400001):
        assert _s(mu) == 1.0
    for mu in (0.6400001, 0.7, 0.95):
        assert _s(mu) == 0.0
    assert abs(_s(0.0) - 0.5) < 1e-15
    for mu in np.linspace(-0.63, 0.63, 27):
        assert abs(_s(mu) + _s(-mu) - 1.0) < 1e-15
    vals = [_s(mu) for mu in np.linspace(-0.7, 0.7, 141)]
    assert all(b <= a + 1e-16 for a, b in zip(vals, vals[1:]))


def test_stratmann_joins_smoothly_at_a():
    """s - 0 vanishes like (a - mu)^4 below mu = a: value and first three
    derivatives are continuous there (a wrong coefficient leaves a lower power)."""
    for h in (2e-2, 1e-2, 5e-3):
        r = _s(A_CUT - h) / _s(A_CUT - 2 * h)
        assert abs(r - 1 / 16) < 0.05 * (1 / 16) + 0.5 * h
        r2 = (1 - _s(-A_CUT + h)) / (1 - _s(-A_CUT + 2 * h))
        assert abs(r2 - 1 / 16) < 0.05 * (1 / 16) + 0.5 * h


def test_stratmann_partition_of_unity():
    rng = np.random.default_rng(4)
    centres = rng.uniform(-2.5, 2.5, (6, 3))
    for _ in range(40):
        p = rng.uniform(-3, 3, 3)
        tot = sum(O.partition_weight(centres, a, p, scheme="stratmann") for a in range(len(centres)))
        assert abs(tot - 1.0) < 1e-14


def test_two_centre_integrals_with_stratmann_weights():
    """The closed-form Gaussian overlap and kinetic integrals of the Becke pin,
    integrated on a grid with Stratmann weights."""
    a, b = 1.3, 1.7
    sp = [Species("A", 1.0, [0], [a]), Species("B", 1.0, [0], [b])]
    wl = Workload("pair", np.array([[0.0, 0.0, 0.0], [0.3, 0.5, 1.4]]), np.array([0, 1], np.int32), sp,
                  n_rad=80, n_theta=20, n_phi=40, partition="stratmann")
    xyz, w, _ = O.grid(wl)
    ob = O.OracleBasis(wl, analytic=True)
    pat = ob.pattern()
    V, W0, *_ = ob.matrix_blocks(xyz, w, np.ones(len(w)), pat)
    S, T2 = ob.dense(V, pat), ob.dense(W0, pat)
    R2 = float(((wl.xyz[1] - wl.xyz[0]) ** 2).sum())
    p, mu = a + b, a * b / (a + b)
    Sab = (math.pi / p) ** 1.5 * math.exp(-mu * R2) / (4 * math.pi)
    Tab = mu * (3 - 2 * mu * R2) * Sab
    # quadrature error on this grid: ~1e-8 (S) and ~1.3e-7 (T, a partly cancelling
    # integrand; the Stratmann cell function is steeper than Becke's); a wrong
    # weight misses by orders of magnitude more
    assert abs(S[0, 1] / Sab - 1) < 1e-7
    assert abs(T2[0, 1] / (2 * Tab) - 1) < 1e-6
    # the weights differ from Becke's (it is another partition), the integrals do not
    wb = O.grid(dataclasses.replace(wl, partition="becke"))[1]
    assert len(wb) != len(w) or np.abs(wb - w).max() > 1e-6 * w.max()
