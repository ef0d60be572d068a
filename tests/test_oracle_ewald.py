"""Pins of the ionic-melt oracle (oracle/ewald.py) against what physics and
mathematics fix: the Madelung constant of rock salt, the alpha independence
of the Ewald sum, finite differences of the energy for forces and for every
virial component (the box strained by a cell matrix), SPME converging to the
plain k-space sum, cardinal B-spline identities, and per-particle sums.
CPU only."""
import math

import numpy as np
import pytest

from oracle import ewald
from paper_2503_07526_gb300 import synth

BUCK = dict(A=1200.0, rho=0.32, C=10.0)
MADELUNG_NACL = 1.747564594633182  # rock salt, per ion pair, in units of ke q^2 / a_nn


def melt_config(n_pairs, L, seed, dmin=1.6):
    """n_pairs cations and anions at random positions with no pair closer
    than dmin (rejection sampling), charges +1 / -1."""
    pts = []
    u = synth.uniform01(seed, 3 * 200 * n_pairs).reshape(-1, 3) * L
    for p in u:
        if all(np.linalg.norm(ewald._min_image((p - x)[:, None], ewald.cell_matrix(L))) >= dmin for x in pts):
            pts.append(p)
        if len(pts) == 2 * n_pairs:
            break
    assert len(pts) == 2 * n_pairs
    r = np.ascontiguousarray(np.array(pts).T)
    q = np.concatenate([np.ones(n_pairs), -np.ones(n_pairs)])
    return r, q


def test_bspline_identities():
    u = np.linspace(-0.3, 9.3, 97)
    for n in (2, 4, 6, 8):
        # partition of unity, symmetry, support
        x = synth.uniform01(n, 50) * 3.0 + 2.0
        tot = sum(ewald.bspline(x - k, n) for k in range(-12, 12))
        assert np.allclose(tot, 1.0, atol=1e-14)
        assert np.allclose(ewald.bspline(u, n), ewald.bspline(n - u, n), atol=1e-14)
        assert np.all(ewald.bspline(u[(u <= 0) | (u >= n)], n) == 0.0)
    assert ewald.bspline(1.0, 4) == pytest.approx(1 / 6, rel=1e-15)
    assert ewald.bspline(2.0, 4) == pytest.approx(2 / 3, rel=1e-15)


def test_madelung_constant_of_rock_salt():
    a = 5.64
    r, q, L = ewald.rock_salt(2, a)
    alpha, rc = 0.8, L / 2 - 1e-9
    _, _, _, Ur = ewald.real_space(r, q, L, A=0.0, rho=1.0, C=0.0, alpha=alpha, rc=rc)
    Erec = ewald.ewald_reciprocal(r, q, L, alpha=alpha, nmax=14)[3]
    U = Ur + Erec + ewald.self_energy(q, alpha).sum()
    want = -(len(q) / 2) * MADELUNG_NACL * ewald.KE / (a / 2)
    assert U == pytest.approx(want, rel=1e-9)


def test_ewald_total_is_independent_of_alpha():
    L = 11.0
    r, q = melt_config(16, L, 3)
    tot = []
    for alpha, nmax in ((0.75, 12), (0.9, 14)):
        _, _, _, Ur = ewald.real_space(r, q, L, A=0.0, rho=1.0, C=0.0, alpha=alpha, rc=L / 2 - 1e-9)
        Erec = ewald.ewald_reciprocal(r, q, L, alpha=alpha, nmax=nmax)[3]
        tot.append(Ur + Erec + ewald.self_energy(q, alpha).sum())
    assert tot[0] == pytest.approx(tot[1], rel=1e-9)


def test_forces_are_minus_the_energy_gradient():
    L, alpha, rc = 10.0, 0.45, 4.5
    r, q = melt_config(8, L, 5)
    F = ewald.real_space(r, q, L, alpha=alpha, rc=rc, **BUCK)[0] + \
        ewald.ewald_reciprocal(r, q, L, alpha=alpha, nmax=8)[0]
    h = 1e-5
    for j, a in ((0, 0), (3, 1), (9, 2), (15, 0)):
        rp, rm = r.copy(), r.copy()
        rp[a, j] += h
        rm[a, j] -= h
        up = ewald.total_energy(rp, q, L, alpha=alpha, rc=rc, nmax=8, **BUCK)
        um = ewald.total_energy(rm, q, L, alpha=alpha, rc=rc, nmax=8, **BUCK)
        assert F[a, j] == pytest.approx(-(up - um) / (2 * h), rel=1e-6, abs=1e-8)


def _strained(h_eps, r, L):
    h = ewald.cell_matrix(L)
    return (np.eye(3) + h_eps) @ h, (np.eye(3) + h_eps) @ r


@pytest.mark.parametrize("part", ["reciprocal", "real"])
def test_virial_is_minus_the_strain_derivative(part):
    """W_ab = -dU/d eps_ab for a symmetric strain of box and coordinates:
    uniaxial strains pin xx, yy, zz; shears pin xy, xz, yz."""
    L, alpha, rc = 10.0, 0.45, 4.5
    r, q = melt_config(8, L, 7)
    if part == "real":
        # no pair within 1e-3 of the cut-off, so the strain moves none across it
        d = np.array([[np.linalg.norm(ewald._min_image((r[:, i] - r[:, j])[:, None], ewald.cell_matrix(L)))
                       for j in range(r.shape[1])] for i in range(r.shape[1])])
        assert np.all(np.abs(d - rc) > 1e-3)

        def energy(hc, rr):
            return ewald.real_space(rr, q, hc, alpha=alpha, rc=rc, **BUCK)[3]

        W = ewald.real_space(r, q, L, alpha=alpha, rc=rc, **BUCK)[2].sum(axis=1)
    else:
        def energy(hc, rr):
            return ewald.ewald_reciprocal(rr, q, hc, alpha=alpha, nmax=9)[3]

        W = ewald.ewald_reciprocal(r, q, L, alpha=alpha, nmax=9)[4]
    h = 1e-6
    comps = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))
    for c, (a, b) in enumerate(comps):
        e = np.zeros((3, 3))
        e[a, b] = e[b, a] = h
        up = energy(*_strained(e, r, L))
        um = energy(*_strained(-e, r, L))
        dU = (up - um) / (2 * h)
        want = -dU if a == b else -dU / 2
        assert W[c] == pytest.approx(want, rel=1e-5, abs=1e-6), (part, c)


def test_spme_converges_to_the_kspace_sum():
    L, alpha = 12.0, 0.5
    r, q = melt_config(24, L, 11)
    Fd, Ed, Wd, Erd, Wrd = ewald.ewald_reciprocal(r, q, L, alpha=alpha, nmax=12)
    assert Ed.sum() == pytest.approx(Erd, rel=1e-12)
    assert np.allclose(Wd.sum(axis=1), Wrd, rtol=1e-11, atol=1e-12 * np.abs(Wrd).max())
    assert np.abs(Fd.sum(axis=1)).max() <= 1e-10 * np.abs(Fd).max()
    errs = []
    for K, order in ((16, 4), (32, 8)):
        F, E, W, Er, Wr = ewald.spme_reciprocal(r, q, L, alpha=alpha, K=K, order=order)
        Wt = ewald.spme_reciprocal(r, q, L, alpha=alpha, K=K, order=order, virial="tensor")[2]
        errs.append((abs(Er - Erd) / abs(Erd), np.abs(W - Wd).max() / np.abs(Wd).max()))
        # the energies and the tensor-form virials sum exactly to the mesh totals
        assert E.sum() == pytest.approx(Er, rel=1e-12)
        assert np.allclose(Wt.sum(axis=1), Wr, rtol=1e-11, atol=1e-12 * np.abs(Wr).max())
        if K == 32:
            assert Er == pytest.approx(Erd, rel=1e-7)
            assert np.abs(Wr - Wrd).max() <= 1e-6 * np.abs(Wrd).max()
            assert np.abs(F - Fd).max() <= 1e-5 * np.abs(Fd).max()
            assert np.abs(E - Ed).max() <= 1e-5 * np.abs(Ed).max()
            # Appendix B's derivative form and the tensor form both reach the
            # k-space sum's per-particle virial
            assert np.abs(W - Wd).max() <= 1e-5 * np.abs(Wd).max()
            assert np.abs(Wt - Wd).max() <= 1e-5 * np.abs(Wd).max()
            assert np.abs(W.sum(axis=1) - Wrd).max() <= 1e-5 * np.abs(Wrd).max()
    assert errs[1][0] < 0.01 * errs[0][0] and errs[1][1] < 0.01 * errs[0][1]


def test_buckingham_dimer_closed_form():
    L, rc = 30.0, 10.0
    d = 2.7
    r = np.array([[1.0, 1.0 + d], [2.0, 2.0], [3.0, 3.0]])
    q = np.zeros(2)
    F, E, W, U = ewald.real_space(r, q, L, alpha=0.3, rc=rc, **BUCK)
    u = BUCK["A"] * math.exp(-d / BUCK["rho"]) - BUCK["C"] / d ** 6
    f = BUCK["A"] / BUCK["rho"] * math.exp(-d / BUCK["rho"]) - 6 * BUCK["C"] / d ** 7  # -dU/dr
    assert U == pytest.approx(u, rel=1e-14)
    assert E[0] == E[1] == pytest.approx(u / 2, rel=1e-14)
    assert F[0, 1] == pytest.approx(f, rel=1e-14) and F[0, 0] == pytest.approx(-f, rel=1e-14)
    assert W[0, 0] == pytest.approx(0.5 * d * f, rel=1e-14)
