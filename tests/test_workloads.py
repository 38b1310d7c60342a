"""The seeded inputs: the periodic potential summed per chunk over the images
near the chunk equals the plain sum over every image within reach (the
dropped terms are exact zeros), and the slab generator keeps the layering,
composition and separations it states.  CPU only."""
import numpy as np

import workloads as W


def _full_periodic_potential(points, wl):
    sh = W._images(wl, 2.0 * wl.r_c + wl.r_nb)
    cen = (wl.xyz[None, :, :] + sh[:, None, :]).reshape(-1, 3)
    Zc = np.tile(wl.Z_of_atom, len(sh))
    d = np.sqrt(((points[:, None, :] - cen[None, :, :]) ** 2).sum(-1))
    f = W._erf(d) / d * W._smoothstep_cut(d, 2.0 * wl.r_c - 1.0, 2.0 * wl.r_c)
    return -(f * Zc[None, :]).sum(-1)


def test_periodic_potential_restricted_sum():
    wl = W.periodic_cell()
    rng = np.random.default_rng(3)
    pts = rng.uniform(-6.0, 18.0, size=(6000, 3))  # inside, near and beyond the cell
    got = W.potential(pts, wl)
    ref = _full_periodic_potential(pts, wl)
    assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-14
    # the chunking does not matter beyond rounding order
    assert np.max(np.abs(W.potential(pts, wl, chunk=17) - got) / np.abs(ref)) < 1e-14


def _min_image(d, L):
    return d - L * np.round(d / L)


def test_slab_layering_composition_and_separations():
    wl = W.small_slab()
    L = np.diag(wl.lattice)
    nf = wl.nf_of_atom
    heavy = nf == 64
    assert heavy.sum() == round(0.3 * wl.n_atoms)
    zc = 0.5 * L[2]
    assert np.all(np.abs(wl.xyz[heavy, 2] - zc) < 8.0)          # heavy layer
    assert np.all(np.abs(wl.xyz[~heavy, 2] - zc) >= 8.0 - 1e-12)  # light atoms outside it
    assert np.all((wl.xyz >= 0.0) & (wl.xyz < L[None, :]))
    d = _min_image(wl.xyz[:, None, :] - wl.xyz[None, :, :], L)
    r = np.sqrt((d ** 2).sum(-1)) + np.eye(wl.n_atoms) * 1e9
    assert r[np.ix_(heavy, heavy)].min() >= 4.0
    assert r.min() >= 1.8
    sp = [s.name for s in wl.species]
    names = [sp[k] for k in wl.species_of_atom]
    assert set(names[i] for i in np.where(heavy)[0]) == {"Pb", "I"}
    assert set(names[i] for i in np.where(~heavy)[0]) <= {"H", "C", "N"}
    assert {s.name: s.n_fn for s in wl.species} == {"Pb": 64, "I": 64, "H": 5, "C": 14, "N": 14}
    assert min(L) >= 2.0 * wl.r_nb  # the image shell {-1, 0, 1}^3 covers r_nb from any point of the cell
