"""The tile-window pair path (MD_PAIR_TILES, mixed-precision Lennard-Jones):
the same parity bars as the mixed Verlet path (Sec. 1 link cells and
velocity Verlet; Sec. 2.3 Eq. (stress), the per-particle energy split and the
heat flux).  Forces: every component within 2e-5 of max(|F_ia|, F_rms) of
the FP64 oracle at the GPU's own positions (plus the cutoff-jump allowance
of check_mixed_forces); per-particle energy and virial within 2e-5 of their
largest magnitude; the stress and heat-flux reduction within 1e-10 of the
FP64 reduction of the same particles."""
import numpy as np
import pytest

from paper_2503_07526_gb300 import synth
from test_gpu_md import F_AT_RC, check_mixed_forces, jittered, melted, params, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_07526_gb300 as pkg

    pkg.lib(build=True)
    return pkg


def tiles(pkg, s, **kw):
    kw.setdefault("precision", pkg.MD_PREC_MIXED)
    return params(pkg, s, pair_mode=pkg.MD_PAIR_TILES, **kw)


def check_particles(got, oracle_mod, L):
    """Forces as check_mixed_forces; per-particle energy and virial within
    2e-5 of their largest magnitude.  The shifted energy is continuous at the
    cutoff, the virial is not: a pair within 1e-5 rc of rc may fall on either
    side in FP32 and in FP64, which moves each virial component of both atoms
    by up to rc |f(rc)| / 2, allowed per such pair as for the forces."""
    F, e, W = oracle_mod.lj_forces(got["r"], L, method="cells")
    check_mixed_forces(got["F"], F, got["r"], L, oracle_mod)
    assert np.abs(got["epot"] - e).max() <= 2e-5 * np.abs(e).max()
    near = oracle_mod.near_cutoff_pairs(got["r"], L, 2.5, 1e-5 * 2.5)
    allow = 1.001 * 0.5 * 2.5 * abs(F_AT_RC) * near
    assert (np.abs(got["W"] - W) - allow[None, :]).max() <= 2e-5 * np.abs(W).max()


@pytest.mark.parametrize("cells", [6, 7, 9, 12])
def test_initial_forces_tiles(pkg, oracle_mod, cells):
    """Boxes of 3 to 7 cells per side (3- and 4-cell boxes: windows that wrap
    onto themselves, one atom seen at two images) against the oracle."""
    s = jittered(cells, seed=cells + 11)
    g = pkg.System(tiles(pkg, s), s["r"], s["v"])
    cfg = g.config()
    assert cfg["build_kind"] == 3 and cfg["tiles"] > 0 and cfg["window_capacity"] <= 4096
    check_particles(g.particles(), oracle_mod, s["L"])


def test_tiles_along_trajectory(pkg, oracle_mod):
    """Ten steps with a 0.1 skin (list rebuilds inside the window): forces at
    every step, and the reduction against the FP64 reduction (1e-10)."""
    s = jittered(10, seed=2)
    g = pkg.System(tiles(pkg, s, skin=0.1), s["r"], s["v"])
    for _ in range(10):
        g.step(1)
        got = g.particles()
        check_particles(got, oracle_mod, s["L"])
        obs = g.observables()
        want = oracle_mod.observables(s["L"] ** 3, np.ones(s["n"]), got["v"], got["epot"], got["W"])
        assert rel(obs["sigma"], want[3:9]) <= 1e-10
        assert rel(obs["q"], want[9:12]) <= 1e-10
        assert obs["U"] == pytest.approx(want[0], rel=1e-10)
    assert g.observables()["rebuilds"] >= 2


def test_tiles_agree_with_verlet_lists(pkg):
    """Same state, both mixed list paths: forces within FP32 rounding of each
    other (the tile path rounds each displacement from tile-frame
    coordinates, the list path from cell-frame ones)."""
    s = jittered(8, seed=21)
    a = pkg.System(tiles(pkg, s), s["r"], s["v"]).particles()
    b = pkg.System(params(pkg, s, precision=pkg.MD_PREC_MIXED), s["r"], s["v"]).particles()
    frms = np.sqrt((b["F"] ** 2).mean())
    assert np.abs(a["F"] - b["F"]).max() <= 4e-5 * max(np.abs(b["F"]).max(), frms)


@pytest.mark.parametrize("skin", [0.3, 0.4])
def test_full_size_tiles_forces_and_reduction(pkg, oracle_mod, skin):
    """The 2,048,000-atom liquid of the benchmark on the tile path (skin 0.4
    is the benchmark's: 46^3 cells, a close segment out to 1.43 sigma)."""
    s, st = melted(pkg, 80, seed=1)
    g = pkg.System(tiles(pkg, s, skin=skin), st["r"], st["v"])
    g.step(2)
    got = g.particles()
    F, e, W = oracle_mod.lj_forces(got["r"], s["L"], method="cells")
    check_mixed_forces(got["F"], F, got["r"], s["L"], oracle_mod)
    obs = g.observables()
    want = oracle_mod.observables(s["L"] ** 3, np.ones(s["n"]), got["v"], got["epot"], got["W"])
    assert rel(obs["sigma"], want[3:9]) <= 1e-10
    assert rel(obs["q"], want[9:12]) <= 1e-10


def test_lattice_start_tiles(pkg, oracle_mod):
    """fcc start (small net forces from cancelling pair forces), 32,000 atoms."""
    s = synth.lj_system(20, seed=1)
    g = pkg.System(tiles(pkg, s), s["r"], s["v"])
    g.step(2)
    check_particles(g.particles(), oracle_mod, s["L"])


def test_tiles_batch_equals_replicas_run_alone(pkg, oracle_mod):
    """Replicas of 3 to 7 cells per side in one handle: each bit for bit the
    replica run alone, and each within the mixed bound of the oracle."""
    reps = []
    for k, (cells, rho, T) in enumerate(((5, 0.70, 1.5), (6, 0.85, 0.9), (7, 0.80, 1.2), (8, 0.90, 1.0))):
        t = synth.lj_system(cells, rho=rho, T=T, seed=40 + k)
        t["r"] = t["r"] + 0.15 * (synth.uniform01(50 + k, t["r"].size).reshape(t["r"].shape) - 0.5)
        reps.append(dict(r=t["r"], v=t["v"], box=t["L"], n=t["n"]))
    p = pkg.make_params(1, 1.0, precision=pkg.MD_PREC_MIXED, pair_mode=pkg.MD_PAIR_TILES, skin=0.2,
                        stress=(6, 16, 2, 1), heatflux=(6, 16, 2, 1), vacf=None)
    b = pkg.System(p, replicas=reps)
    b.step(20)
    got = b.particles()
    a0 = 0
    for k, rp in enumerate(reps):
        sl = slice(a0, a0 + rp["n"])
        a0 += rp["n"]
        pa = pkg.make_params(rp["n"], rp["box"], precision=pkg.MD_PREC_MIXED, pair_mode=pkg.MD_PAIR_TILES,
                             skin=0.2, stress=(6, 16, 2, 1), heatflux=(6, 16, 2, 1), vacf=None)
        alone = pkg.System(pa, rp["r"], rp["v"])
        alone.step(20)
        want = alone.particles()
        for key in ("r", "v", "F", "W", "epot"):
            assert np.array_equal(got[key][..., sl], want[key]), (k, key)
        assert b.replica_observables(k)["sigma"].tolist() == alone.observables()["sigma"].tolist()
        part = {key: got[key][..., sl] for key in ("r", "F", "epot", "W")}
        check_particles(part, oracle_mod, rp["box"])


def test_tiles_launch_paths_agree(pkg):
    """Direct launches, 8-step graphs and timed graphs: identical particles
    and observables over list rebuilds."""
    s = jittered(8, seed=13, T=1.2)
    out = []
    for graph, timing in ((False, False), (True, False), (True, True)):
        g = pkg.System(tiles(pkg, s, skin=0.1, use_graph=graph), s["r"], s["v"])
        g.set_timing(timing)
        g.step(21)
        g.step(16)
        o = g.observables()
        out.append(dict(g.particles(), U=o["U"], sigma=o["sigma"], q=o["q"]))
        assert o["rebuilds"] >= 2
        g.close()
    for key in out[0]:
        for o in out[1:]:
            assert np.array_equal(out[0][key], o[key]), key


def test_tiles_only_for_mixed_lennard_jones(pkg):
    s = jittered(6, seed=3)
    with pytest.raises(pkg.MdError) as ei:
        pkg.System(tiles(pkg, s, precision=pkg.MD_PREC_FP64), s["r"], s["v"])
    assert ei.value.code == -1


def test_window_capacity_is_checked(pkg):
    """A window that needs more slots than the capacity is an error (the
    build marks the tile and writes nothing; MD_ESTATE), a capacity given
    explicitly changes nothing else, and a capacity that is not a multiple of
    16 up to 4,096 is refused."""
    s = jittered(8, seed=5)
    with pytest.raises(pkg.MdError) as ei:
        pkg.System(tiles(pkg, s, window_slots=64), s["r"], s["v"])
    assert ei.value.code == -4
    a = pkg.System(tiles(pkg, s), s["r"], s["v"])
    b = pkg.System(tiles(pkg, s, window_slots=4096), s["r"], s["v"])
    assert b.config()["window_capacity"] == 4096 and a.config()["window_capacity"] < 4096
    a.step(12)
    b.step(12)
    pa, pb = a.particles(), b.particles()
    for key in ("r", "v", "F", "W", "epot"):
        assert np.array_equal(pa[key], pb[key]), key
    for bad in (17, 4112, -16):
        with pytest.raises(pkg.MdError) as ei:
            pkg.System(tiles(pkg, s, window_slots=bad), s["r"], s["v"])
        assert ei.value.code == -1


def test_tiles_autotune(pkg, oracle_mod):
    """md_params.autotune on the tile path picks a candidate tiling (tiles of
    at most 3x2x2, 2x2x2 or 3x3x2 cells) and a CTA size in whole warps; the
    forces with it stay within the mixed bound of the oracle at init and
    after ten steps over list rebuilds."""
    s = jittered(12, seed=31)
    g = pkg.System(tiles(pkg, s, autotune=True, skin=0.1), s["r"], s["v"])
    cfg = g.config()
    assert cfg["tile_extent"] in ((3, 2, 2), (2, 2, 2), (3, 3, 2))
    assert 128 <= cfg["tile_threads"] <= 384 and cfg["tile_threads"] % 32 == 0
    check_particles(g.particles(), oracle_mod, s["L"])
    g.step(10)
    check_particles(g.particles(), oracle_mod, s["L"])
    assert g.observables()["rebuilds"] >= 2
    assert pkg.System(tiles(pkg, s), s["r"], s["v"]).config()["tile_extent"] == (3, 2, 2)


def test_tiles_autotune_batch(pkg, oracle_mod):
    """The autotuner on an uneven batch (replicas of 5 to 8 cells per side):
    every replica within the mixed bound of the oracle after 20 steps."""
    reps = []
    for k, (cells, rho, T) in enumerate(((5, 0.70, 1.5), (6, 0.85, 0.9), (7, 0.80, 1.2), (8, 0.90, 1.0))):
        t = synth.lj_system(cells, rho=rho, T=T, seed=60 + k)
        t["r"] = t["r"] + 0.15 * (synth.uniform01(70 + k, t["r"].size).reshape(t["r"].shape) - 0.5)
        reps.append(dict(r=t["r"], v=t["v"], box=t["L"], n=t["n"]))
    p = pkg.make_params(1, 1.0, precision=pkg.MD_PREC_MIXED, pair_mode=pkg.MD_PAIR_TILES, skin=0.2, autotune=True,
                        stress=(6, 16, 2, 1), heatflux=(6, 16, 2, 1), vacf=None)
    b = pkg.System(p, replicas=reps)
    assert b.config()["tile_extent"] in ((3, 2, 2), (2, 2, 2), (3, 3, 2))
    b.step(20)
    got = b.particles()
    a0 = 0
    for rp in reps:
        sl = slice(a0, a0 + rp["n"])
        a0 += rp["n"]
        check_particles({key: got[key][..., sl] for key in ("r", "F", "epot", "W")}, oracle_mod, rp["box"])
