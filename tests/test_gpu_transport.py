"""Green-Kubo viscosity and thermal conductivity (Sec. 2.3 Eqs. (visc) and
(therm)) from the GPU's on-the-fly correlators against the FP64 oracle, on
the 4,000-atom LJ liquid (fcc 10^3 x 4, rho* = 0.8442, T* = 0.722, rc = 2.5,
dt = 0.005): melt with velocity rescaling (T* = 2.0 for 2,000 steps, then
0.722 for 3,000 steps, every 10 steps), then 4,000 NVE steps with the
stress / heat-flux correlators (b = 12, p = 16, m = 2, u = 1).  Both sides
integrate the readout to t_cut = 2 tau (400 steps), past the decay of both
autocorrelations; the paper leaves the cutoff lag to the user.  Trajectories
are chaotic, so each side is a sample of the same ensemble: over 8 seeds
the two means must agree within 2 standard errors of their difference.
eta = V / T * int C_sigma (mean of xy, xz, yz; Sec. 2.3 averages congruent
correlations); kappa = V / (3 T^2) * int <q(t).q(0)>."""
import math
import os

import numpy as np
import pytest

from paper_2503_07526_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

SEEDS = range(1, 9)
CELLS, RHO, T_STAR, DT = 10, 0.8442, 0.722, 0.005
MELT_HOT, MELT_COLD, PROD = 2000, 3000, 4000
T_CUT = 2.0


def _melt(step, scale, temp):
    for target, nsteps in ((2.0, MELT_HOT), (T_STAR, MELT_COLD)):
        for _ in range(nsteps // 10):
            step(10)
            scale(math.sqrt(target / temp()))


def _oracle_seed(seed):
    """One oracle run (worker process): returns (eta, kappa, T_mean)."""
    os.environ.setdefault("OMP_NUM_THREADS", "2")
    import oracle

    s = synth.lj_system(CELLS, rho=RHO, T=T_STAR, seed=seed)
    md = oracle.MD(s["r"], s["v"], s["L"], dt=DT)
    _melt(lambda k: md.step(k), md.scale_velocities, lambda: md.get()["obs"][2])
    cs = oracle.Corr(12, 16, 2, 6)  # sigma_xy, sigma_xz, sigma_yz, q_x, q_y, q_z
    obs = md.step(PROD, cs=cs, record=True)
    T = obs[:, 2].mean()
    V = s["L"] ** 3
    t, _ = cs.read(0)
    c_sig = np.mean([cs.read(g)[1] for g in range(3)], axis=0)
    c_q = np.mean([cs.read(g)[1] for g in range(3, 6)], axis=0)
    eta, _ = oracle.gk_trapz(t * DT, c_sig, t_cut=T_CUT, prefactor=V / T)
    kappa, _ = oracle.gk_trapz(t * DT, c_q, t_cut=T_CUT, prefactor=V / T ** 2)  # V/(3T^2) * 3 mean
    return eta, kappa, T


@pytest.fixture(scope="module")
def oracle_results():
    # the pool is started with spawn, before this module touches the GPU
    import concurrent.futures as cf
    import multiprocessing as mp

    import oracle

    oracle.build()
    with cf.ProcessPoolExecutor(max_workers=8, mp_context=mp.get_context("spawn")) as ex:
        return np.array(list(ex.map(_oracle_seed, SEEDS)))


@pytest.fixture(scope="module")
def pkg(oracle_results):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_07526_gb300 as pkg

    pkg.lib(build=True)
    return pkg


def _gpu_seed(pkg, seed, precision):
    s = synth.lj_system(CELLS, rho=RHO, T=T_STAR, seed=seed)
    p = pkg.make_params(s["n"], s["L"], dt=DT, precision=precision, stress=(12, 16, 2, 1),
                        heatflux=(12, 16, 2, 1), vacf=(8, 16, 2, 1))
    g = pkg.System(p, s["r"], s["v"])
    _melt(g.step, g.scale_velocities, lambda: g.observables()["T"])
    g.reset_correlators()
    g.step(PROD)
    T = g.observables()["T_mean"]
    V = s["L"] ** 3
    t, c_sig = g.corr(pkg.MD_CORR_STRESS).read(-1)
    tq, c_q = g.corr(pkg.MD_CORR_HEATFLUX).read(-1)
    eta, _ = pkg.gk_integrate(t, c_sig, t_cut=T_CUT, prefactor=V / T)
    kappa, _ = pkg.gk_integrate(tq, c_q, t_cut=T_CUT, prefactor=V / T ** 2)
    g.close()
    return eta, kappa, T


@pytest.mark.parametrize("precision", [0, 1])
def test_transport_coefficients_within_two_standard_errors(pkg, oracle_results, precision):
    gpu = np.array([_gpu_seed(pkg, seed, precision) for seed in SEEDS])
    n = len(SEEDS)
    for k, name in ((0, "eta"), (1, "kappa")):
        a, b = gpu[:, k], oracle_results[:, k]
        se = math.sqrt(a.var(ddof=1) / n + b.var(ddof=1) / n)
        diff = a.mean() - b.mean()
        print(f"{name} ({'fp64' if precision == 0 else 'mixed'}): GPU {a.mean():.4f} +- {a.std(ddof=1) / math.sqrt(n):.4f}"
              f"  oracle {b.mean():.4f} +- {b.std(ddof=1) / math.sqrt(n):.4f}  diff/SE {diff / se:+.2f}")
        assert abs(diff) <= 2.0 * se
    # the temperatures of the correlated runs agree closely
    assert abs(gpu[:, 2].mean() - oracle_results[:, 2].mean()) < 0.02
