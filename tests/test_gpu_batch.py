"""Batched replicas (one handle, all replicas advanced by the same kernels
and graph launch): each replica must behave exactly as the same system run
alone, and as the FP64 oracle (Sec. 1, Sec. 2.3, Alg. 1).  FP64 tolerance
1e-11 relative per array, as in the other parity tests."""
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


def replica(cells, rho, T, seed, amp=0.15):
    s = synth.lj_system(cells, rho=rho, T=T, seed=seed)
    s["r"] = s["r"] + amp * (synth.uniform01(seed + 7, s["r"].size).reshape(s["r"].shape) - 0.5)
    return dict(r=s["r"], v=s["v"], box=s["L"], n=s["n"])


REPS = [(7, 0.80, 1.5, 3), (9, 0.85, 0.9, 4), (6, 0.75, 2.0, 5), (8, 0.88, 0.7, 6)]


def batch_params(pkg, **kw):
    kw.setdefault("stress", (6, 16, 2, 1))
    kw.setdefault("heatflux", (6, 16, 2, 1))
    kw.setdefault("vacf", None)
    kw.setdefault("skin", 0.2)
    return pkg.make_params(1, 1.0, **kw)


def split(arr, sizes):
    out, a0 = [], 0
    for n in sizes:
        out.append(arr[..., a0:a0 + n])
        a0 += n
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_replicas_run_alone(pkg, precision):
    reps = [replica(*x) for x in REPS]
    p = batch_params(pkg, precision=precision)
    b = pkg.System(p, replicas=reps)
    b.step(25)
    got = b.particles()
    sizes = [x["n"] for x in reps]
    for k, rp in enumerate(reps):
        pa = pkg.make_params(rp["n"], rp["box"], precision=precision, skin=0.2, stress=(6, 16, 2, 1),
                             heatflux=(6, 16, 2, 1), vacf=None)
        alone = pkg.System(pa, rp["r"], rp["v"])
        alone.step(25)
        want = alone.particles()
        for key in ("r", "v", "F", "W"):
            assert rel(split(got[key], sizes)[k], want[key]) <= 1e-13, (k, key)
        ob, oa = b.replica_observables(k), alone.observables()
        assert ob["step"] == oa["step"] == 25
        for key in ("U", "K", "T", "T_mean"):
            assert ob[key] == pytest.approx(oa[key], rel=1e-13)
        assert rel(ob["sigma"], oa["sigma"]) <= 1e-13
        # the replica's stress correlator is series 3k..3k+2 of the batch's
        cb, ca = b.corr(pkg.MD_CORR_STRESS), alone.corr(pkg.MD_CORR_STRESS)
        for comp in range(3):
            tb, vb = cb.read(3 * k + comp)
            ta, va = ca.read(comp)
            assert np.array_equal(tb, ta)
            assert np.abs(vb - va).max() <= 1e-12 * abs(va[0])


def test_batch_matches_oracle_per_replica(pkg, oracle_mod):
    reps = [replica(*x) for x in REPS[:3]]
    b = pkg.System(batch_params(pkg, precision=0), replicas=reps)
    mds = [oracle_mod.MD(rp["r"], rp["v"], rp["box"]) for rp in reps]
    for _ in range(8):
        b.step(1)
        for k, md in enumerate(mds):
            o = md.step(1, record=True)[0]
            ob = b.replica_observables(k)
            assert ob["U"] == pytest.approx(o[0], rel=1e-11)
            assert rel(ob["sigma"], o[3:9]) <= 1e-11
            assert rel(ob["q"], o[9:12]) <= 1e-11
    got = b.particles()
    for k, (md, F) in enumerate(zip(mds, split(got["F"], [x["n"] for x in reps]))):
        assert rel(F, md.get()["F"]) <= 1e-11


def test_replica_scaling_and_autotune(pkg):
    reps = [replica(*x) for x in REPS]
    lam = np.array([0.5, 1.0, 0.9, 1.1])
    b = pkg.System(batch_params(pkg, precision=1), replicas=reps)
    T0 = [b.replica_observables(k)["T"] for k in range(4)]
    b.replica_scale_velocities(lam)
    for k in range(4):
        assert b.replica_observables(k)["T"] == pytest.approx(lam[k] ** 2 * T0[k], rel=1e-6)
    # autotuning picks launch shapes only: identical trajectories
    bt = pkg.System(batch_params(pkg, precision=1, autotune=True), replicas=reps)
    cfg = bt.config()
    assert cfg["pair_threads"] in (64, 128, 256) and cfg["build_warps"] in (2, 4, 8)
    assert cfg["replicas"] == 4 and cfg["atoms"] == sum(x["n"] for x in reps)
    b2 = pkg.System(batch_params(pkg, precision=1), replicas=reps)
    bt.step(15)
    b2.step(15)
    assert np.array_equal(bt.particles()["F"], b2.particles()["F"])


def test_batch_rejects_bad_replicas(pkg):
    tiny = replica(3, 0.8, 1.0, 1)  # 108 atoms, below 256 per replica
    with pytest.raises(pkg.MdError):
        pkg.System(batch_params(pkg), replicas=[tiny, replica(7, 0.8, 1.0, 2)])
    with pytest.raises(pkg.MdError):  # per-atom VACF is for single systems
        pkg.System(batch_params(pkg, vacf=(4, 16, 2, 1)), replicas=[replica(7, 0.8, 1.0, 2)] * 2)
