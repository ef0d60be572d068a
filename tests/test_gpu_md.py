"""GPU MD path parity against the FP64 oracle (Sec. 1 link cells and velocity
Verlet; Sec. 2.3 stress tensor and heat flux; Sec. 2.2 correlators).

Tolerances.  FP64: max|GPU - oracle| / max|oracle| <= 1e-11 per array (only
summation order differs; over 10 steps chaotic growth of rounding is far
below that).  Mixed form: every force component within 2e-5 of
max(|F_ia|, F_rms) (see check_mixed_forces), against the FP64 oracle at the
same positions; the per-particle energy and virial within 2e-5 of their
largest magnitude.
"""
import numpy as np
import pytest

from paper_2503_07526_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_07526_gb300 as pkg

    pkg.lib(build=True)
    return pkg


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def min_image(d, L):
    return d - L * np.round(d / L)


def jittered(cells, seed, rho=0.8442, T=0.722, amp=0.2):
    s = synth.lj_system(cells, rho=rho, T=T, seed=seed)
    s["r"] = s["r"] + amp * (synth.uniform01(seed + 99, s["r"].size).reshape(s["r"].shape) - 0.5)
    return s


def params(pkg, s, **kw):
    kw.setdefault("stress", (6, 16, 2, 1))
    kw.setdefault("heatflux", (6, 16, 2, 1))
    kw.setdefault("vacf", (4, 16, 2, 1))
    return pkg.make_params(s["n"], s["L"], **kw)


F_AT_RC = 24 * (2 * 2.5 ** -12 - 2.5 ** -6) / 2.5  # truncated LJ force at the cutoff


def check_mixed_forces(F, Fo, r=None, L=None, oracle_mod=None):
    """FP32 forces against FP64 at the same positions, per force component:
    |dF_ia| <= 2e-5 max(|F_ia|, F_rms) for every atom i and axis a, plus one
    force jump |f(rc)| for each pair of atom i within 1e-5 rc of the cutoff,
    where FP32 and FP64 distances may fall on opposite sides of rc (both
    results valid: the truncated force is discontinuous there).  The
    normwise error max_i |dF_ia| / max_i |F_ia| is printed beside it."""
    frms = np.sqrt((Fo ** 2).mean())
    allow = np.zeros(F.shape[1])
    if r is not None:
        near = oracle_mod.near_cutoff_pairs(r, L, 2.5, 1e-5 * 2.5)
        allow = 1.001 * abs(F_AT_RC) * near
    dF = np.abs(F - Fo)
    clean = allow == 0
    normwise = max((dF[a, clean]).max() / np.abs(Fo[a]).max() for a in range(3))
    ratio = np.maximum(dF - allow[None, :], 0.0) / np.maximum(np.abs(Fo), frms)
    print(f"mixed forces: elementwise max |dF|/max(|F|, F_rms) = {ratio.max():.3e}, normwise {normwise:.3e} "
          f"(F_rms {frms:.3f}); atoms with a pair within 1e-5 rc of the cutoff: {(~clean).sum()}")
    assert ratio.max() <= 2e-5
    return ratio.max()


@pytest.mark.parametrize("cells", [6, 8, 10, 11])
@pytest.mark.parametrize("mode", ["verlet", "cells"])
def test_initial_forces_fp64(pkg, oracle_mod, cells, mode):
    s = jittered(cells, seed=cells)
    pm = pkg.MD_PAIR_VERLET if mode == "verlet" else pkg.MD_PAIR_CELLS
    g = pkg.System(params(pkg, s, precision=pkg.MD_PREC_FP64, pair_mode=pm), s["r"], s["v"])
    got = g.particles()
    F, e, W = oracle_mod.lj_forces(s["r"], s["L"], method="cells")
    assert rel(got["F"], F) <= 1e-11
    assert rel(got["epot"], e) <= 1e-11
    assert rel(got["W"], W) <= 1e-11
    assert np.abs(min_image(got["r"] - s["r"], s["L"])).max() <= 1e-12
    assert np.array_equal(got["v"], s["v"])
    obs = g.observables()
    want = oracle_mod.observables(s["L"] ** 3, np.ones(s["n"]), s["v"], e, W)
    assert obs["U"] == pytest.approx(want[0], rel=1e-12)
    assert obs["K"] == pytest.approx(want[1], rel=1e-12)
    assert rel(obs["sigma"], want[3:9]) <= 1e-11
    assert rel(obs["q"], want[9:12]) <= 1e-11


@pytest.mark.parametrize("cells", [6, 10])
@pytest.mark.parametrize("mode", ["verlet", "cells"])
def test_initial_forces_mixed(pkg, oracle_mod, cells, mode):
    s = jittered(cells, seed=cells + 1)
    pm = pkg.MD_PAIR_VERLET if mode == "verlet" else pkg.MD_PAIR_CELLS
    g = pkg.System(params(pkg, s, precision=pkg.MD_PREC_MIXED, pair_mode=pm), s["r"], s["v"])
    got = g.particles()
    F, e, W = oracle_mod.lj_forces(s["r"], s["L"], method="cells")
    check_mixed_forces(got["F"], F, s["r"], s["L"], oracle_mod)
    assert np.abs(got["epot"] - e).max() <= 2e-5 * np.abs(e).max()
    assert np.abs(got["W"] - W).max() <= 2e-5 * np.abs(W).max()


@pytest.mark.parametrize("mode,skin,graph", [("verlet", 0.3, True), ("verlet", 0.05, True),
                                             ("verlet", 0.05, False), ("cells", 0.0, True)])
def test_ten_steps_fp64(pkg, oracle_mod, mode, skin, graph):
    """Per-step parity over 10 steps; skin 0.05 forces neighbour-list rebuilds
    inside the window."""
    s = jittered(8, seed=5, T=1.2)
    pm = pkg.MD_PAIR_VERLET if mode == "verlet" else pkg.MD_PAIR_CELLS
    g = pkg.System(params(pkg, s, precision=pkg.MD_PREC_FP64, pair_mode=pm, skin=skin, use_graph=graph),
                   s["r"], s["v"])
    md = oracle_mod.MD(s["r"], s["v"], s["L"])
    for step in range(10):
        g.step(1)
        o = md.step(1, record=True)[0]
        obs = g.observables()
        assert obs["step"] == step + 1
        assert obs["U"] == pytest.approx(o[0], rel=1e-11)
        assert obs["K"] == pytest.approx(o[1], rel=1e-11)
        assert rel(obs["sigma"], o[3:9]) <= 1e-11
        assert rel(obs["q"], o[9:12]) <= 1e-11
    got, want = g.particles(), md.get()
    assert np.abs(min_image(got["r"] - want["r"], s["L"])).max() <= 1e-11 * s["L"]
    assert rel(got["v"], want["v"]) <= 1e-11
    assert rel(got["F"], want["F"]) <= 1e-11
    assert rel(got["W"], want["W"]) <= 1e-11


def test_mixed_forces_along_trajectory(pkg, oracle_mod):
    """Mixed form: at every step the FP32 forces meet the per-component
    bound against FP64 forces at the GPU's own positions, and the stress,
    heat flux and energies equal the FP64 reduction (Sec. 2.3) of the same
    particles to 1e-10."""
    s = jittered(10, seed=2)
    g = pkg.System(params(pkg, s, precision=pkg.MD_PREC_MIXED, skin=0.1), s["r"], s["v"])
    for _ in range(10):
        g.step(1)
        got = g.particles()
        F, e, W = oracle_mod.lj_forces(got["r"], s["L"], method="cells")
        check_mixed_forces(got["F"], F, got["r"], s["L"], oracle_mod)
        obs = g.observables()
        want = oracle_mod.observables(s["L"] ** 3, np.ones(s["n"]), got["v"], got["epot"], got["W"])
        # the reduction itself is FP64-class (double-float terms, compensated
        # partials, FP64 tree): 1e-10 relative to the FP64 reduction of the
        # same per-particle arrays
        assert rel(obs["sigma"], want[3:9]) <= 1e-10
        assert rel(obs["q"], want[9:12]) <= 1e-10
        assert obs["U"] == pytest.approx(want[0], rel=1e-10)
        assert obs["K"] == pytest.approx(want[1], rel=1e-10)


@pytest.mark.parametrize("prec", [0, 1])
def test_md_correlators_match_oracle(pkg, oracle_mod, prec):
    """The stress, heat-flux and velocity correlators fed by md_step equal
    oracle correlators fed by the oracle's own run (FP64, 64 steps), or by
    the GPU's recorded series (mixed form, where trajectories differ)."""
    s = jittered(8, seed=11, T=1.0)
    n = s["n"]
    g = pkg.System(params(pkg, s, precision=prec, stress=(5, 16, 2, 1), heatflux=(5, 8, 2, 2),
                          vacf=(4, 16, 2, 1)), s["r"], s["v"])
    cs = oracle_mod.Corr(5, 16, 2, 3)
    ch = oracle_mod.Corr(5, 8, 2, 3)
    cv = oracle_mod.Corr(4, 16, 2, 3 * n, gs=n)
    if prec == 0:
        md = oracle_mod.MD(s["r"], s["v"], s["L"])
    for step in range(1, 65):
        g.step(1)
        if prec == 0:
            o = md.step(1, record=True)[0]
            st = md.get()
            sig, q, v = o[6:9], o[9:12], st["v"]
        else:
            obs = g.observables()
            sig, q, v = obs["sigma"][3:6], obs["q"], g.particles()["v"]
        cs.push(sig)
        if step % 2 == 0:
            ch.push(q)
        cv.push(v)
    tol = 1e-11 if prec == 0 else 2e-5
    for which, orc, dtu in [(pkg.MD_CORR_STRESS, cs, 1), (pkg.MD_CORR_HEATFLUX, ch, 2), (pkg.MD_CORR_VACF, cv, 1)]:
        c = g.corr(which)
        for grp in range(3):
            tg, vg = c.read(grp)
            to, vo = orc.read(grp)
            assert np.allclose(tg, to * dtu * 0.005, rtol=1e-14)
            assert np.abs(vg - vo).max() <= (1e-11 if (prec == 0 or which != pkg.MD_CORR_VACF) else tol) * abs(vo[0])
    assert g.corr(pkg.MD_CORR_HEATFLUX).pushes() == 32


def test_reset_and_scale_velocities(pkg, oracle_mod):
    s = jittered(8, seed=4)
    g = pkg.System(params(pkg, s), s["r"], s["v"])
    g.step(7)
    T0 = g.observables()["T"]
    g.scale_velocities(0.5)
    assert g.observables()["T"] == pytest.approx(0.25 * T0, rel=1e-12)
    g.reset_correlators()
    assert g.corr(pkg.MD_CORR_VACF).pushes() == 0
    g.step(5)
    assert g.corr(pkg.MD_CORR_STRESS).pushes() == 5
    assert g.observables()["step"] == 12


def test_energy_conservation_fp64_and_mixed(pkg):
    s = jittered(10, seed=8, amp=0.05)
    for prec in (0, 1):
        g = pkg.System(params(pkg, s, precision=prec), s["r"], s["v"])
        E = []
        for _ in range(40):
            g.step(10)
            o = g.observables()
            E.append(o["U"] + o["K"])
        E = np.array(E)
        assert np.abs(E - E[0]).max() / s["n"] < 2e-3, prec


def test_invalid_inputs_are_errors(pkg):
    s = synth.lj_system(5)  # L = 8.40: only 2 cells of rc + skin
    with pytest.raises(pkg.MdError) as ei:
        pkg.System(params(pkg, s), s["r"], s["v"])
    assert ei.value.code == -1
    s = synth.lj_system(6)
    r = s["r"].copy()
    r[1, 5] = np.nan
    with pytest.raises(pkg.MdError) as ei:
        pkg.System(params(pkg, s), r, s["v"])
    assert ei.value.code == -4
    with pytest.raises(pkg.MdError) as ei:
        pkg.System(params(pkg, s, max_neighbors=8), s["r"], s["v"])
    assert ei.value.code == -4
    with pytest.raises(pkg.MdError):
        pkg.System(params(pkg, s), s["r"], s["v"], types=np.full(s["n"], 3, dtype=np.int32))


def test_device_inputs_and_outputs(pkg, oracle_mod):
    import torch

    s = jittered(6, seed=3)
    rd = torch.tensor(s["r"], device="cuda")
    vd = torch.tensor(s["v"], device="cuda")
    g = pkg.System(params(pkg, s), rd, vd)
    F = torch.empty((3, s["n"]), dtype=torch.float64, device="cuda")
    g.particles_device(F=F)
    Fo, _, _ = oracle_mod.lj_forces(s["r"], s["L"], method="cells")
    assert rel(F.cpu().numpy(), Fo) <= 1e-11


def melted(pkg, cells, seed):
    """A liquid at T* = 0.722 (the benchmark's state): fcc start rescaled to
    T* = 2.0 for 600 steps, then to 0.722 for 600 steps."""
    s = synth.lj_system(cells, seed=seed)
    g = pkg.System(params(pkg, s, precision=pkg.MD_PREC_MIXED, stress=None, heatflux=None, vacf=None),
                   s["r"], s["v"])
    for target in (2.0, 0.722):
        for _ in range(60):
            g.step(10)
            g.scale_velocities(np.sqrt(target / g.observables()["T"]))
    st = g.particles()
    g.close()
    return s, st


def test_full_size_mixed_forces_and_reduction(pkg, oracle_mod):
    """The 2,048,000-atom mixed-precision liquid of the benchmark: every force
    component against the FP64 oracle at the GPU's positions, and the stress /
    heat-flux reduction against the FP64 reduction of the same particles."""
    s, st = melted(pkg, 80, seed=1)
    g = pkg.System(params(pkg, s, precision=pkg.MD_PREC_MIXED), st["r"], st["v"])
    g.step(2)
    got = g.particles()
    F, e, W = oracle_mod.lj_forces(got["r"], s["L"], method="cells")
    check_mixed_forces(got["F"], F, got["r"], s["L"], oracle_mod)
    obs = g.observables()
    want = oracle_mod.observables(s["L"] ** 3, np.ones(s["n"]), got["v"], got["epot"], got["W"])
    assert rel(obs["sigma"], want[3:9]) <= 1e-10
    assert rel(obs["q"], want[9:12]) <= 1e-10


def test_full_size_mixed_velocity_correlator(pkg, oracle_mod):
    """The per-atom velocity correlator of the 2,048,000-atom mixed-form
    benchmark, pushes applied eight at a time by the blocked kernels, against
    the oracle's Algorithm 1 correlator fed the GPU's velocities after every
    step (three whole blocks and a partial one); FP32 samples and products,
    FP64 lag sums: 2e-5 of C(0)."""
    s, st = melted(pkg, 80, seed=2)
    n = s["n"]
    spec = dict(stress=None, heatflux=None, vacf=(4, 16, 2, 1))
    g = pkg.System(params(pkg, s, precision=pkg.MD_PREC_MIXED, **spec), st["r"], st["v"])
    for k in (13, 8, 9):  # graph-replayed calls; pushes 1..30
        g.step(k)
    # the same system one step per call, its velocities recorded for the oracle
    g1 = pkg.System(params(pkg, s, precision=pkg.MD_PREC_MIXED, **spec), st["r"], st["v"])
    cv = oracle_mod.Corr(4, 16, 2, 3 * n, gs=n)
    for _ in range(30):
        g1.step(1)
        cv.push(g1.particles()["v"])
    assert np.array_equal(g1.particles()["v"], g.particles()["v"])
    g1.close()
    c = g.corr(pkg.MD_CORR_VACF)
    for grp in range(3):
        tg, vg = c.read(grp)
        to, vo = cv.read(grp)
        assert np.allclose(tg, to * 0.005, rtol=1e-14)
        err = np.abs(vg - vo).max() / abs(vo[0])
        print(f"component {grp}: max |C_gpu - C_oracle| / C(0) = {err:.2e}")
        assert err <= 2e-5, grp
    assert c.pushes() == 30


def test_velocity_slots_only_with_the_velocity_correlator(pkg):
    """The per-atom velocity correlator's input slots are allocated only when
    that correlator is on (8 slots of 3n samples for p <= 16)."""
    s = jittered(6, seed=3)
    for prec, esz in ((pkg.MD_PREC_FP64, 8), (pkg.MD_PREC_MIXED, 4)):
        g = pkg.System(params(pkg, s, precision=prec, vacf=None), s["r"], s["v"])
        assert g.config()["vacf_input_bytes"] == 0
        g.step(3)
        g.close()
        g = pkg.System(params(pkg, s, precision=prec), s["r"], s["v"])
        assert g.config()["vacf_input_bytes"] == 8 * 3 * s["n"] * esz
        g.close()


def test_lattice_start_mixed_forces(pkg, oracle_mod):
    """fcc start (small net forces, F_rms ~ 0.6, from pair forces ~ 2): the
    hardest case for FP32 positions; 32,000 atoms."""
    s = synth.lj_system(20, seed=1)
    g = pkg.System(params(pkg, s, precision=pkg.MD_PREC_MIXED), s["r"], s["v"])
    g.step(2)
    got = g.particles()
    F, _, _ = oracle_mod.lj_forces(got["r"], s["L"], method="cells")
    check_mixed_forces(got["F"], F, got["r"], s["L"], oracle_mod)


@pytest.mark.parametrize("precision", [0, 1])
def test_list_builds_agree(pkg, precision):
    """The j-parallel, i-parallel and staged list builds produce the same
    lists in the same order, so the forces agree bit for bit, over rebuilds,
    for a single system and a batch with short (3-cell) rows."""
    s = synth.lj_system(12, rho=0.8442, T=2.5, seed=8)
    r = s["r"] + 0.15 * (synth.uniform01(9, s["r"].size).reshape(s["r"].shape) - 0.5)
    out = []
    for lb in (1, 2, 3):
        p = pkg.make_params(s["n"], s["L"], precision=precision, list_build=lb)
        g = pkg.System(p, r, s["v"])
        g.step(40)
        out.append(g.particles())
        assert g.observables()["rebuilds"] >= 2
        g.close()
    for key in ("r", "v", "F", "W", "epot"):
        for o in out[1:]:
            assert np.array_equal(out[0][key], o[key]), key
    reps = []
    for k, (cells, rho) in enumerate(((5, 0.7), (5, 0.9), (7, 0.8))):
        t = synth.lj_system(cells, rho=rho, T=1.5, seed=20 + k)
        reps.append(dict(r=t["r"], v=t["v"], box=t["L"]))
    outb = []
    for lb in (1, 2, 3):
        p = pkg.make_params(1, 1.0, precision=precision, skin=0.2, list_build=lb, vacf=None)
        g = pkg.System(p, replicas=reps)
        g.step(30)
        outb.append(g.particles())
        g.close()
    for key in ("r", "v", "F", "W"):
        for o in outb[1:]:
            assert np.array_equal(outb[0][key], o[key]), key


@pytest.mark.parametrize("precision", [0, 1])
def test_launch_paths_agree(pkg, precision):
    """Direct launches, the 8-step graphs (each step's velocity-correlator push
    running on a second stream beside the next step's kernels) and the timed
    graphs give the same particles, observables and correlators bit for bit,
    over neighbour-list rebuilds and calls that are not multiples of 8 steps;
    the timed run counts one event bracket per kernel class and step (two for
    the reduction class: the reduction and the scalar correlator samples)."""
    s = jittered(8, seed=13, T=1.2)
    out = []
    for graph, timing in ((False, False), (True, False), (True, True)):
        g = pkg.System(params(pkg, s, precision=precision, skin=0.1, use_graph=graph), s["r"], s["v"])
        g.set_timing(timing)
        g.step(21)
        g.step(16)
        o = g.observables()
        res = dict(g.particles(), U=o["U"], sigma=o["sigma"], q=o["q"])
        for which in (pkg.MD_CORR_STRESS, pkg.MD_CORR_HEATFLUX, pkg.MD_CORR_VACF):
            c = g.corr(which)
            for grp in range(3):
                res[f"c{which}_{grp}"] = c.read(grp)[1]
        assert o["rebuilds"] >= 2
        if timing:
            kt = g.kernel_times()
            for name in ("integrate", "rebuild", "pair", "reduce", "vacf"):
                assert kt[name][1] == (74 if name == "reduce" else 37) and kt[name][0] > 0.0, name
        g.close()
        out.append(res)
    for key in out[0]:
        for o in out[1:]:
            assert np.array_equal(out[0][key], o[key]), key


@pytest.mark.parametrize("prec,p,u", [(0, 16, 1), (0, 16, 2), (0, 8, 1), (1, 16, 1)])
def test_blocked_velocity_pushes(pkg, oracle_mod, prec, p, u):
    """The per-atom velocity correlator's pushes wait in input slots and are
    applied a block at a time (8 pushes, or p - m + 1 when smaller).  Calls
    of 13, 8, 3 and 40 steps start blocks at several offsets and end in
    partial blocks.  FP64: against the oracle correlator fed the oracle's
    own velocities after every step (push every u steps), 1e-11 of C(0);
    mixed: against the oracle correlator fed the velocities of the same
    system stepped one step per call (the same trajectory bit for bit), 2e-5
    of C(0) (FP32 samples and products, FP64 lag sums)."""
    s = jittered(8, seed=11, T=1.0)
    n = s["n"]
    spec = dict(stress=(5, 16, 2, 1), heatflux=(5, 8, 2, 2), vacf=(4, p, 2, u))
    g = pkg.System(params(pkg, s, precision=prec, **spec), s["r"], s["v"])
    for k in (13, 8, 3, 40):
        g.step(k)
    c = g.corr(pkg.MD_CORR_VACF)
    if prec == 0:
        cv = oracle_mod.Corr(4, p, 2, 3 * n, gs=n)
        md = oracle_mod.MD(s["r"], s["v"], s["L"])
        for step in range(1, 65):
            md.step(1)
            if step % u == 0:
                cv.push(md.get()["v"])
        for grp in range(3):
            tg, vg = c.read(grp)
            to, vo = cv.read(grp)
            assert np.allclose(tg, to * u * 0.005, rtol=1e-14)
            assert np.abs(vg - vo).max() <= 1e-11 * abs(vo[0]), grp
    else:
        g1 = pkg.System(params(pkg, s, precision=prec, **spec), s["r"], s["v"])
        cv = oracle_mod.Corr(4, p, 2, 3 * n, gs=n)
        for step in range(1, 65):
            g1.step(1)
            if step % u == 0:
                cv.push(g1.particles()["v"])
        assert np.array_equal(g1.particles()["v"], g.particles()["v"])
        for grp in range(3):
            tg, vg = c.read(grp)
            to, vo = cv.read(grp)
            assert np.allclose(tg, to * u * 0.005, rtol=1e-14)
            assert np.abs(vg - vo).max() <= 2e-5 * abs(vo[0]), grp
    assert c.pushes() == 64 // u
