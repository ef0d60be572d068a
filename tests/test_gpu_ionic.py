"""The ionic-melt path (Buckingham + Ewald with SPME, per-particle energy and
virial, Sec. 5.3 and Appendix B) on the GPU against the FP64 oracle
(oracle/ewald.py): per-particle forces, energies and virials, and the
per-step observables (stress tensor and heat flux, Sec. 2.3) built from them.

System: 1,728 ions (rock salt 6^3 x 8 at 0.031 ions / A^3, L = 38.2 A, every
ion displaced by up to 0.3 A), charges +1 / -1 e, Na / Cl masses, Buckingham
A = 1200 eV, rho = 0.32 A, C = 10 eV A^6 for every pair, rc = 10 A, Ewald
alpha = 0.3 / A, order-8 splines on a 16^3 mesh (the chunks of a cell row fit
the kernels' shared tiles) and on a 32^3 mesh (they do not: the kernels take
the global mesh directly); units eV, A, amu, e.

Tolerances.  FP64: the charge mesh is summed in 128-bit fixed point with
2^-80 resolution per contribution (so that the sums do not depend on the
order of the atomic adds), far below FP64 rounding; 1e-11 normwise per
array, as for Lennard-Jones.  Mixed: FP32 pair terms, FP32 spreading, FFTs and
gathers; 2e-5 normwise per force component, as for Lennard-Jones, and 1e-4
for the per-particle energies and virials (sums of large cancelling
terms)."""
import numpy as np
import pytest

from paper_2503_07526_gb300 import synth

pytestmark = pytest.mark.gpu

RHO, T_EV = 0.031, 0.112025  # ions / A^3, kB x 1300 K in eV
BUCK = dict(A=1200.0, rho=0.32, C=10.0)
RC, ALPHA, K, ORDER = 10.0, 0.3, 32, 8  # K: the mesh of the runs below the parity tests
MASSES = (22.99, 35.45)


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_07526_gb300 as pkg

    pkg.lib(build=True)
    return pkg


@pytest.fixture(scope="module")
def system():
    return synth.ionic_system(6, RHO, T_EV, seed=4, masses=MASSES, jitter=0.3)


_REF = {}


def reference(system, mesh):
    """Oracle per-particle forces, energies, virials (cached per mesh)."""
    from oracle import ewald

    if mesh not in _REF:
        s = system
        q = np.where(s["types"] == 0, 1.0, -1.0)
        r = np.mod(s["r"], s["L"])
        Fr, Er, Wr, _ = ewald.real_space(r, q, s["L"], alpha=ALPHA, rc=RC, **BUCK)
        Fk, Ek, Wk, _, _ = ewald.spme_reciprocal(r, q, s["L"], alpha=ALPHA, K=mesh, order=ORDER)
        _REF[mesh] = dict(F=Fr + Fk, epot=Er + Ek + ewald.self_energy(q, ALPHA), W=Wr + Wk)
    return _REF[mesh]


def params(pkg, s, precision, skin=1.0, mesh=K):
    return pkg.make_params(s["n"], s["L"], rc=RC, dt=0.098227, skin=skin, precision=precision,
                           masses=MASSES, potential=pkg.MD_POT_BUCK_EWALD, charges=(1.0, -1.0),
                           buckingham=(BUCK["A"], BUCK["rho"], BUCK["C"]), ewald_alpha=ALPHA, mesh=mesh, order=ORDER,
                           stress=(8, 16, 2, 1), heatflux=(8, 16, 2, 1), vacf=None)


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("mesh", [16, 32])
@pytest.mark.parametrize("precision", [0, 1])
def test_forces_energies_virials_match_oracle(pkg, system, precision, mesh):
    s = system
    ref = reference(s, mesh)
    g = pkg.System(params(pkg, s, precision, mesh=mesh), s["r"], s["v"], types=s["types"])
    got = g.particles()
    g.close()
    tol = {0: (1e-11, 1e-11), 1: (2e-5, 1e-4)}[precision]
    for key, t in (("F", tol[0]), ("epot", tol[1]), ("W", tol[1])):
        e = rel(got[key], ref[key])
        print(f"precision {precision} mesh {mesh}: {key} {e:.2e}")
        assert e <= t, key
    # SPME forces do not sum to zero exactly (the interpolated energy is not
    # translation invariant); the net force is the oracle's
    net, want_net = got["F"].sum(axis=1), ref["F"].sum(axis=1)
    assert np.abs(net - want_net).max() <= (1e-9 if precision == 0 else 2e-3) * np.abs(ref["F"]).max()


@pytest.mark.parametrize("precision", [0, 1])
def test_observables_match_oracle(pkg, system, precision, oracle_mod):
    """Stress tensor and heat flux of the initial state (Sec. 2.3) from the
    per-particle terms, against the oracle's reduction of the oracle's
    per-particle terms."""
    s = system
    g = pkg.System(params(pkg, s, precision), s["r"], s["v"], types=s["types"])
    o = g.observables()
    g.close()
    mass_of = np.asarray(MASSES)[s["types"]]
    ref = reference(s, K)
    want = oracle_mod.observables(s["L"] ** 3, mass_of, s["v"], ref["epot"], ref["W"])
    tol = 1e-11 if precision == 0 else 1e-4
    assert o["U"] == pytest.approx(want[0], rel=tol)
    assert o["K"] == pytest.approx(want[1], rel=1e-12 if precision == 0 else 1e-6)
    assert rel(o["sigma"], want[3:9]) <= tol
    assert rel(o["q"], want[9:12]) <= max(tol, 1e-4 if precision else tol)


def test_mass_flux_correlations(pkg, system, oracle_mod):
    """The partial momentum density of the cations, j = sum m v / V over
    them, and its correlations with the heat flux (Sec. 2.3, the mass-flux
    correction of kappa for multi-component systems): j against its
    definition from the velocities (and against minus the anions' share, up
    to SPME's small net force), and the device's cross correlator against the
    oracle's correlator fed the same per-step (q, j) samples."""
    s = system
    p = params(pkg, s, 0, mesh=16)
    p.massflux.b, p.massflux.p, p.massflux.m, p.massflux.u = 4, 16, 2, 1
    g = pkg.System(p, s["r"], s["v"], types=s["types"])
    qs, js = [], []
    for _ in range(80):
        g.step(1)
        o = g.observables()
        qs.append(o["q"])
        js.append(o["j"])
    part = g.particles()
    V = s["L"] ** 3
    mass_of = np.asarray(MASSES)[s["types"]]
    mv = mass_of[None, :] * part["v"]
    want = mv[:, s["types"] == 0].sum(axis=1) / V
    other = mv[:, s["types"] == 1].sum(axis=1) / V
    assert rel(o["j"], want) <= 1e-12
    # the two species' shares cancel up to the momentum SPME's small net force
    # has added since the start (the interpolated energy is not translation
    # invariant)
    assert np.abs(want + other).max() <= 1e-2 * np.abs(want).max()
    c = g.corr(pkg.MD_CORR_MASSFLUX)
    oc = oracle_mod.Corr(4, 16, 2, 6, cross=True)
    for q, j in zip(qs, js):
        oc.push(np.concatenate([q, j]), np.concatenate([j, j]))
    for k in range(6):
        t, v = c.read(k)
        to, vo = oc.read(k)
        assert np.allclose(t / p.dt, to, rtol=1e-12)
        assert np.abs(v - vo).max() <= 1e-12 * np.abs(vo).max(), k
    g.close()


def test_short_run_conserves_energy(pkg, system):
    """200 NVE steps of 1 fs in the mixed form: total energy drift below
    1e-4 of the kinetic energy per step, no state error."""
    s = system
    g = pkg.System(params(pkg, s, 1), s["r"], s["v"], types=s["types"])
    o0 = g.observables()
    e0 = o0["U"] + o0["K"]
    g.step(200)
    o1 = g.observables()
    e1 = o1["U"] + o1["K"]
    g.close()
    print(f"E0 {e0:.6f} E1 {e1:.6f} K {o0['K']:.4f} rebuilds {o1['rebuilds']}")
    assert abs(e1 - e0) <= 200 * 1e-4 * o0["K"]


@pytest.mark.parametrize("mesh", [16, 32])
def test_runs_are_bitwise_reproducible(pkg, system, mesh):
    """The charge mesh is summed in integers (tile columns in a fixed atom
    order, fixed-point global adds), so two runs of the same input agree
    bit for bit (mesh 16: shared tiles; mesh 32: direct global adds)."""
    s = system
    out = []
    for _ in range(2):
        g = pkg.System(params(pkg, s, 1, mesh=mesh), s["r"], s["v"], types=s["types"])
        g.step(25)
        out.append(g.particles())
        g.close()
    for key in ("r", "v", "F", "W", "epot"):
        assert np.array_equal(out[0][key], out[1][key]), key


def test_ionic_rejects_bad_setups(pkg, system):
    s = system
    with pytest.raises(pkg.MdError):  # odd mesh
        pkg.System(pkg.make_params(s["n"], s["L"], rc=RC, potential=pkg.MD_POT_BUCK_EWALD, charges=(1, -1),
                                   masses=MASSES, buckingham=(1200, 0.32, 10), ewald_alpha=0.3, mesh=33,
                                   order=8, vacf=None), s["r"], s["v"], types=s["types"])
    with pytest.raises(pkg.MdError):  # replicas are Lennard-Jones only
        reps = [dict(r=s["r"], v=s["v"], box=s["L"], types=s["types"])] * 2
        pkg.System(params(pkg, s, 1), replicas=reps)
