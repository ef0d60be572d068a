"""Pins of the FP64 CPU oracle against what the paper and the mathematics
fix (no GPU).  Each test would fail on a plausible slip in the oracle: a
dropped factor 1/2, a wrong sign, a transposed operand, an off-by-one lag.

Paper: arXiv 2503.07526.  Sec. 2.2 Eq. (cor) and Appendix D Algorithms 1-2
(correlator); Sec. 2.3 Eqs. (visc), (stress), (therm) and the heat-flux
definition; Sec. 1 velocity Verlet.
"""
import math
import os

import numpy as np
import pytest

from paper_2503_07526_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def perturbed_fcc(cells, rho, amp, seed):
    r, L = synth.fcc_lattice(cells, rho)
    r = r + amp * (synth.uniform01(seed, r.size).reshape(r.shape) - 0.5)
    return r, L


def cluster(n, spacing, seed, centre):
    """n atoms on a jittered simple-cubic patch (an isolated droplet)."""
    k = int(math.ceil(n ** (1 / 3)))
    g = np.arange(k) * spacing
    gz, gy, gx = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([gx.ravel(), gy.ravel(), gz.ravel()])[:, :n]
    pos = pos + 0.1 * (synth.uniform01(seed, pos.size).reshape(pos.shape) - 0.5)
    return pos - pos.mean(axis=1, keepdims=True) + centre


# ---------------------------------------------------------------- forces


def test_two_atom_closed_forms(oracle_mod):
    """LJ minimum at r = 2^(1/6): zero force, pair energy -1 - U(rc); at
    r = 1: energy -U(rc), force 24; beyond rc: nothing (shifted potential,
    readings R9-R10)."""
    uc = 4.0 * (2.5 ** -12 - 2.5 ** -6)
    for dist, u_pair, f_pair in [(2 ** (1 / 6), -1.0 - uc, 0.0), (1.0, -uc, 24.0), (1.5, None, None), (2.6, 0.0, 0.0)]:
        r = np.array([[10.0, 10.0 + dist], [10.0, 10.0], [10.0, 10.0]])
        F, e, W = oracle_mod.lj_forces(r, 50.0, method="brute", periodic=False)
        if u_pair is None:  # generic distance: U(1.5) and -U'(1.5) by the textbook formula
            s6 = dist ** -6
            u_pair = 4 * (s6 * s6 - s6) - uc
            f_pair = 24 * (2 * s6 * s6 - s6) / dist
        assert e == pytest.approx([u_pair / 2, u_pair / 2], abs=1e-14)
        # f on atom 0 points away from atom 1 (-x) when repulsive
        assert F[0, 0] == pytest.approx(-f_pair, abs=1e-12)
        assert F[0, 1] == pytest.approx(f_pair, abs=1e-12)
        # each atom carries half of r_ij (x) f_ij: xx = dist * f_pair / 2
        assert W[0] == pytest.approx([dist * f_pair / 2] * 2, abs=1e-12)
        assert np.abs(W[1:]).max() < 1e-14


def test_unshifted_potential_at_cutoff(oracle_mod):
    r = np.array([[10.0, 12.49999], [10.0, 10.0], [10.0, 10.0]])
    _, e, _ = oracle_mod.lj_forces(r, 50.0, method="brute", periodic=False, shift=False)
    s6 = 2.49999 ** -6
    assert e.sum() == pytest.approx(4 * (s6 * s6 - s6), rel=1e-13)


@pytest.mark.parametrize("cells,rho", [(5, 0.8442), (6, 0.8442), (7, 0.8), (8, 0.8442)])
def test_link_cells_equal_brute_force(oracle_mod, cells, rho):
    """Link cells (3, 4 and 5 cells per side) against all pairs."""
    r, L = perturbed_fcc(cells, rho, 0.3, seed=cells)
    assert 3 <= int(L // 2.5) <= 5
    Fb, eb, Wb = oracle_mod.lj_forces(r, L, method="brute")
    Fc, ec, Wc = oracle_mod.lj_forces(r, L, method="cells")
    for a, b in [(Fb, Fc), (eb, ec), (Wb, Wc)]:
        assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()


def brute_near_cutoff(r, L, rc, band):
    """Per atom, the neighbours at minimum-image distance within band of rc,
    over all pairs (no cells)."""
    d = r[:, :, None] - r[:, None, :]
    d -= L * np.round(d / L)
    dist = np.sqrt((d ** 2).sum(axis=0))
    np.fill_diagonal(dist, np.inf)
    return (np.abs(dist - rc) <= band).sum(axis=1)


def test_near_cutoff_count_equals_brute_force(oracle_mod):
    """The near-cutoff pair count (the allowance of the FP32 force parity
    test) against all pairs: random atoms in a 3-cell box, and planted pairs
    just inside and outside rc +- band, across the periodic boundary and
    along a body diagonal, in a box whose cells are exactly rc wide (a pair
    at rc + band/2 there can lie two cells apart)."""
    rc, band = 2.5, 0.2
    L = 9.0
    r = L * synth.uniform01(77, 3 * 200).reshape(3, 200)
    got = oracle_mod.near_cutoff_pairs(r, L, rc, band)
    want = brute_near_cutoff(r, L, rc, band)
    assert want.sum() > 100
    assert np.array_equal(got, want)
    # planted pairs, L = 3 rc: one cell of edge rc per third of the box
    L, band = 3 * rc, 1e-3
    dirs = np.array([[1, 0, 0], [0, 1, 0], [1, 1, 1], [1, -1, 0]], dtype=float)
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    starts = np.array([[0.2, 3.0, 3.0], [7.4, 0.3, 5.0], [1.0, 1.0, 1.0], [6.0, 6.2, 2.0]])
    offsets = [-0.4 * band, 0.4 * band, -1.5 * band, 1.5 * band]
    pos = []
    for k, off in enumerate(offsets):
        a = starts[k]
        pos += [a, a + (rc + off) * dirs[k]]
    r = np.mod(np.array(pos).T, L)
    got = oracle_mod.near_cutoff_pairs(r, L, rc, band)
    want = brute_near_cutoff(r, L, rc, band)
    assert want.tolist() == [1, 1, 1, 1, 0, 0, 0, 0]
    assert np.array_equal(got, want)
    # L = 5 rc: a pair at rc + band/2 whose atoms sit in cells 0 and 2
    L = 5 * rc
    r = np.array([[2.4998, 2.4998 + rc + 0.4 * band], [1.0, 1.0], [1.0, 1.0]])
    assert np.array_equal(oracle_mod.near_cutoff_pairs(r, L, rc, band), [1, 1])


def test_newton_third_law_and_energy_sum(oracle_mod):
    r, L = perturbed_fcc(6, 0.8442, 0.4, seed=3)
    F, e, W = oracle_mod.lj_forces(r, L, method="cells")
    assert np.abs(F.sum(axis=1)).max() <= 1e-12 * np.abs(F).sum()
    # total energy over unordered pairs, each pair once, from distances only
    n = r.shape[1]
    d = r[:, :, None] - r[:, None, :]
    d -= L * np.round(d / L)
    r2 = (d * d).sum(axis=0)
    iu = np.triu_indices(n, 1)
    rr = np.sqrt(r2[iu])
    rr = rr[rr < 2.5]
    u = 4 * (rr ** -12 - rr ** -6) - 4 * (2.5 ** -12 - 2.5 ** -6)
    assert e.sum() == pytest.approx(u.sum(), rel=1e-13)


def test_force_is_minus_energy_gradient(oracle_mod):
    """F_i = -dU/dr_i by central differences (U is the oracle's total)."""
    r, L = perturbed_fcc(5, 0.8442, 0.3, seed=7)
    F, _, _ = oracle_mod.lj_forces(r, L, method="cells")
    h = 1e-6
    for i, a in [(0, 0), (17, 1), (333, 2)]:
        rp, rm = r.copy(), r.copy()
        rp[a, i] += h
        rm[a, i] -= h
        up = oracle_mod.lj_forces(rp, L, method="cells")[1].sum()
        um = oracle_mod.lj_forces(rm, L, method="cells")[1].sum()
        assert -(up - um) / (2 * h) == pytest.approx(F[a, i], rel=1e-6, abs=1e-6)


PAIRS = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]


def test_virial_is_minus_strain_derivative_isolated(oracle_mod):
    """Sum_i W_i,ab = -dU/d eps_ab under the affine deformation r -> (1+eps) r
    (fixes the factor 1/2 and the sign of Eq. (stress), reading R8)."""
    r = cluster(40, 1.15, seed=11, centre=25.0)
    _, _, W = oracle_mod.lj_forces(r, 50.0, method="brute", periodic=False)
    Wt = W.sum(axis=1)
    c = r.mean(axis=1, keepdims=True)
    h = 1e-6
    for comp, (a, b) in enumerate(PAIRS):
        def energy(eps):
            Dm = np.eye(3)
            Dm[a, b] += eps
            return oracle_mod.lj_forces(Dm @ (r - c) + c, 50.0, method="brute", periodic=False)[1].sum()

        dU = (energy(h) - energy(-h)) / (2 * h)
        assert Wt[comp] == pytest.approx(-dU, rel=1e-6, abs=1e-6)
    # symmetric virial: xy from the (x,y) and (y,x) strains agree
    assert np.abs(Wt).max() > 1.0


def test_virial_trace_under_periodic_scaling(oracle_mod):
    r, L = perturbed_fcc(5, 0.8442, 0.3, seed=5)
    _, _, W = oracle_mod.lj_forces(r, L, method="cells")
    h = 1e-6
    up = oracle_mod.lj_forces(r * (1 + h), L * (1 + h), method="cells")[1].sum()
    um = oracle_mod.lj_forces(r * (1 - h), L * (1 - h), method="cells")[1].sum()
    assert W[:3].sum() == pytest.approx(-(up - um) / (2 * h), rel=1e-6)


def test_ideal_gas_pressure(oracle_mod):
    """No interactions: trace(sigma)/3 = 2K/(3V), sigma off-diagonals are the
    kinetic ones only; T uses 3n-3 degrees of freedom."""
    n, V = 100, 1000.0
    v = synth.maxwell_velocities(n, 1.3, seed=4)
    m = np.full(n, 2.0)
    obs = oracle_mod.observables(V, m, v, np.zeros(n), np.zeros((6, n)))
    K = 0.5 * (m * (v * v).sum(axis=0)).sum()
    assert obs[1] == pytest.approx(K, rel=1e-14)
    assert obs[2] == pytest.approx(2 * K / (3 * n - 3), rel=1e-14)
    assert obs[3:6].sum() / 3 == pytest.approx(2 * K / (3 * V), rel=1e-13)


def heat_current_G(oracle_md, masses_of):
    s = oracle_md.get()
    E = 0.5 * masses_of * (s["v"] ** 2).sum(axis=0) + s["epot"]
    return (s["r"] * E[None, :]).sum(axis=1), s


@pytest.mark.parametrize("dt", [0.002])
def test_heat_flux_is_energy_moment_rate(oracle_mod, dt):
    """Isolated droplet: V q = d/dt sum_i r_i E_i (exact for the equal energy
    split, reading R9), by central differences along the velocity-Verlet
    trajectory; the error must fall as dt^2."""
    errs = []
    for h in (dt, dt / 2):
        r = cluster(30, 1.12, seed=2, centre=40.0)
        v = synth.maxwell_velocities(30, 0.4, seed=9)
        md = oracle_mod.MD(r, v, 80.0, dt=h, cells=False)
        md.step(int(round(0.2 / h)))
        G0, _ = heat_current_G(md, np.ones(30))
        md.step(1)
        _, s1 = heat_current_G(md, np.ones(30))
        Vq = s1["obs"][9:12] * 80.0 ** 3
        md.step(1)
        G2, _ = heat_current_G(md, np.ones(30))
        dG = (G2 - G0) / (2 * h)
        errs.append(np.abs(dG - Vq).max() / np.abs(Vq).max())
    assert errs[0] < 5e-3
    assert 2.5 < errs[0] / errs[1] < 6.0


def test_velocity_verlet_energy_fluctuation_scales_dt2(oracle_mod):
    s = synth.lj_system(5, rho=0.8442, T=0.722, seed=1)
    rms = []
    for dt, n in [(0.004, 200), (0.002, 400)]:
        md = oracle_mod.MD(s["r"], s["v"], s["L"], dt=dt, rc=2.5, shift=True)
        o = md.step(n, record=True)
        E = o[:, 0] + o[:, 1]
        rms.append(E.std())
    assert 2.5 < rms[0] / rms[1] < 6.0


def test_velocity_verlet_time_reversible(oracle_mod):
    s = synth.lj_system(5, seed=2)
    md = oracle_mod.MD(s["r"], s["v"], s["L"], dt=0.004)
    md.step(50)
    st = md.get()
    md2 = oracle_mod.MD(st["r"], -st["v"], s["L"], dt=0.004)
    md2.step(50)
    back = md2.get()
    d = back["r"] - s["r"]
    d -= s["L"] * np.round(d / s["L"])
    assert np.abs(d).max() < 1e-8
    assert np.abs(back["v"] + s["v"]).max() < 1e-8


# ----------------------------------------------------------- correlator


def test_multitau_hand_worked_example(oracle_mod):
    want = np.loadtxt(os.path.join(GOLDEN, "multitau_tiny.txt"))
    c = oracle_mod.Corr(2, 4, 2, 1)
    for x in [1, 2, 3, 4, 5, 6]:
        c.push([float(x)])
    t, v = c.read(0)
    assert np.array_equal(t, want[:, 0])
    assert np.allclose(v, want[:, 1], rtol=1e-15, atol=0)


def test_direct_estimator_definition(oracle_mod):
    x = np.array([1.0, -2.0, 3.0, 0.5])
    y = np.array([2.0, 1.0, -1.0, 4.0])
    out = oracle_mod.direct_corr(x, y, 4)
    # by hand: lag 1 = (1*1 + -2*-1 + 3*4)/3, lag 3 = 1*4/1
    assert out[1] == pytest.approx((1 + 2 + 12) / 3)
    assert out[3] == pytest.approx(4.0)
    assert out[0] == pytest.approx((2 - 2 - 3 + 2) / 4)


def block_means(x, M):
    n = x.shape[0] // M
    return x[: n * M].reshape(n, M, *x.shape[1:]).mean(axis=1)


@pytest.mark.parametrize("b,p,m", [(5, 16, 2), (4, 8, 4), (3, 12, 3), (6, 16, 4)])
def test_multitau_each_level_is_direct_estimator_of_block_means(oracle_mod, b, p, m):
    """Level k at lag l equals Eq. (cor) on the means of aligned blocks of
    m^(k-1) samples, over the samples that reached level k (readings R1-R4)."""
    S = 700
    x = synth.ar1_series(3, S, 0.7, seed=b * 100 + p)
    c = oracle_mod.Corr(b, p, m, 3)
    for t in range(S):
        c.push(x[t])
    vals, cnt, used = c.raw()
    for k in range(used):
        xk = block_means(x, m ** k)
        nk = xk.shape[0]
        lo = 0 if k == 0 else p // m
        for lag in range(lo, p):
            want_cnt = max(0, nk - lag)
            assert cnt[k, lag] == want_cnt
            if want_cnt == 0:
                continue
            for s in range(3):
                d = oracle_mod.direct_corr(xk[:, s], xk[:, s], lag + 1)[lag]
                assert vals[s, k, lag] / cnt[k, lag] == pytest.approx(d, rel=1e-12, abs=1e-14)
        # lags below p/m are never formed on higher levels
        if k > 0:
            assert np.all(cnt[k, :lo] == 0)


def test_multitau_level1_equals_fft_correlation(oracle_mod):
    S, p = 512, 32
    x = synth.ar1_series(1, S, 0.9, seed=5)[:, 0]
    c = oracle_mod.Corr(3, p, 2, 1)
    for t in range(S):
        c.push([x[t]])
    t, v = c.read(0)
    f = np.fft.rfft(x, 2 * S)
    ac = np.fft.irfft(f * np.conj(f), 2 * S)[:p] / (S - np.arange(p))
    assert np.allclose(v[:p], ac, rtol=1e-11, atol=1e-12)
    assert np.array_equal(t[:p], np.arange(p))


def test_cross_correlation_order_older_x_newer_y(oracle_mod):
    """Eq. (cor) is X(s) Y(s+l): the older x times the newer y (R5)."""
    S = 300
    a = synth.ar1_series(2, S, 0.8, seed=8)
    x, y = a[:, 0], 0.5 * np.roll(a[:, 0], 3) + a[:, 1]
    c = oracle_mod.Corr(2, 16, 2, 1, cross=True)
    for t in range(S):
        c.push([x[t]], [y[t]])
    _, v = c.read(0)
    want = oracle_mod.direct_corr(x, y, 16)
    assert np.allclose(v[:16], want, rtol=1e-12)
    swapped = oracle_mod.direct_corr(y, x, 16)
    assert not np.allclose(v[:16], swapped, rtol=1e-3)


def test_readout_times_and_blocks_used(oracle_mod):
    b, p, m = 6, 16, 2
    c = oracle_mod.Corr(b, p, m, 1)
    S = 2 ** 4 + 5  # block 5 needs 2^4 samples, block 6 needs 2^5
    for t in range(S):
        c.push([1.0])
    t, v = c.read(0)
    _, cnt, used = c.raw()
    assert used == 5
    want = list(range(p))
    for k in range(1, used):
        for lag in range(p // m, p):
            if cnt[k, lag] > 0:
                want.append(lag * m ** k)
    assert np.array_equal(t, np.array(want, dtype=float))
    assert np.all(np.diff(t) > 0)
    assert np.allclose(v, 1.0)  # constant series: every lag correlates to 1


def test_samples_past_last_block_dropped(oracle_mod):
    c = oracle_mod.Corr(2, 4, 2, 1)
    for t in range(200):
        c.push([float(t % 5)])
    _, cnt, used = c.raw()
    assert used == 2
    assert cnt[1, 2] == 100 - 2 and cnt[1, 3] == 100 - 3


def test_group_readout_is_mean_of_series(oracle_mod):
    S, ns, gs = 200, 12, 4
    x = synth.ar1_series(ns, S, 0.6, seed=12)
    cg = oracle_mod.Corr(3, 8, 2, ns, gs=gs)
    cs = oracle_mod.Corr(3, 8, 2, ns, gs=1)
    for t in range(S):
        cg.push(x[t])
        cs.push(x[t])
    for g in range(ns // gs):
        tg, vg = cg.read(g)
        vs = np.mean([cs.read(s)[1] for s in range(g * gs, (g + 1) * gs)], axis=0)
        assert np.allclose(vg, vs, rtol=1e-13)


def ar1_block_expectation(phi, M, lag):
    """E[mean(block t) * mean(block t+lag)] for unit-variance AR(1), blocks
    of M samples: (1/M^2) sum_{a, b} phi^|a - b|."""
    a = np.arange(M)[:, None]
    bb = (np.arange(M) + lag * M)[None, :]
    return (phi ** np.abs(a - bb)).sum() / M ** 2


def test_multitau_ar1_closed_form(oracle_mod):
    """Seeded AR(1): E C(l) = phi^l on level 1; block levels match the closed
    double sum; the mean over 64 seeds lies within 4 standard errors."""
    phi, b, p, m, S, seeds = 0.8, 4, 16, 2, 4000, 64
    ests = []
    for s in range(seeds):
        x = synth.ar1_series(1, S, phi, seed=1000 + s)
        c = oracle_mod.Corr(b, p, m, 1)
        for t in range(S):
            c.push(x[t])
        vals, cnt, used = c.raw()
        ests.append(vals[0] / np.maximum(cnt, 1))
    ests = np.array(ests)
    mean, se = ests.mean(axis=0), ests.std(axis=0, ddof=1) / math.sqrt(seeds)
    for k in range(b):
        lo = 0 if k == 0 else p // m
        for lag in range(lo, p):
            want = ar1_block_expectation(phi, m ** k, lag)
            # finite-S bias of Eq. (cor) with a known mean is zero; allow 4 SE
            assert abs(mean[k, lag] - want) < 4 * se[k, lag] + 1e-3, (k, lag)


# -------------------------------------------------------------- Green-Kubo


def test_trapezoid_geometric_closed_form(oracle_mod):
    phi, L, dt = 0.9, 40, 0.25
    t = np.arange(L + 1) * dt
    c = phi ** np.arange(L + 1)
    I, run = oracle_mod.gk_trapz(t, c, prefactor=2.0)
    want = dt * (0.5 + phi * (1 - phi ** L) / (1 - phi) - 0.5 * phi ** L)
    assert I == pytest.approx(2.0 * want, rel=1e-14)
    assert run[-1] == pytest.approx(I, rel=1e-14)


def test_trapezoid_exact_for_linear_on_nonuniform_grid(oracle_mod):
    t = np.array([0.0, 0.1, 0.3, 0.7, 1.5, 3.1])
    c = 2.0 - 0.5 * t
    I, run = oracle_mod.gk_trapz(t, c)
    assert I == pytest.approx(2.0 * 3.1 - 0.25 * 3.1 ** 2, rel=1e-14)
    assert run[3] == pytest.approx(2.0 * 0.7 - 0.25 * 0.7 ** 2, rel=1e-14)
    Icut, _ = oracle_mod.gk_trapz(t, c, t_cut=1.0)
    assert Icut == pytest.approx(2.0 - 0.25, rel=1e-14)


def test_trapezoid_rejects_unsorted_times(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.gk_trapz([0.0, 2.0, 1.0], [1.0, 1.0, 1.0])
