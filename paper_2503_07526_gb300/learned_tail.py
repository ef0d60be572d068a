"""Learned Green-Kubo tail: the replica workload that trains it and the call
that applies it.  Orchestration only: the MD, the correlators, the feature
builder, the Green-Kubo integrals and the network all run in libotfmd.so.

A run's short on-the-fly correlators (the first 64 multiple-tau readout
points of the shear-stress and heat-flux autocorrelations, arXiv 2503.07526
Sec. 2.2 and Appendix D Algorithm 2) and its temperature and density go into
a tensor-core network trained to output the Green-Kubo viscosity and thermal
conductivity (Sec. 2.3) that a much longer run of the same replica reaches.
The long run's correlator integral is the training target and the judge.
The short run's own integral is the fallback: it is returned outside the
temperature-density box of the training set, and wherever the run is long
enough that this integral is expected to be more accurate than the network.
The expected error of a run's own integral falls as 1/sqrt(steps) and does
not fall with the number of atoms: the Green-Kubo integrand is the
autocorrelation of one global flux, whose relative fluctuation is the same
for any box size (measured on 4,096 replicas of 500 to 32,000 atoms: 0.29 to
0.31 rms at every size).  The network's error is measured on validation
replicas.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import _lib, synth

N_FEATURES = 132
T_CUT = 2.0    # Green-Kubo cut-off in LJ time units (400 steps at dt = 0.005)
DT = 0.005
RC = 2.5
SPEC = (12, 16, 2, 1)  # stress and heat-flux correlators: b, p, m, u


def ensemble_specs(count, seed, n_range=(500, 32000), rho_range=(0.7, 0.9), T_range=(0.7, 2.0)):
    """count LJ replicas with sizes drawn log-uniformly in n_range (fcc
    k^3 x 4, k in [5, 20]), densities and temperatures uniform in their
    ranges.  Returns a list of dicts (cells, rho, T, seed)."""
    u = synth.uniform01(seed, 3 * count).reshape(3, count)
    out = []
    lo, hi = math.log(n_range[0]), math.log(n_range[1])
    for k in range(count):
        cells = synth.cells_for_atoms(math.exp(lo + u[0, k] * (hi - lo)))
        out.append(dict(cells=cells, rho=rho_range[0] + (rho_range[1] - rho_range[0]) * u[1, k],
                        T=T_range[0] + (T_range[1] - T_range[0]) * u[2, k], seed=seed * 100003 + k))
    return out


def build_replicas(specs):
    reps = []
    for s in specs:
        sysd = synth.lj_system(s["cells"], rho=s["rho"], T=s["T"], seed=s["seed"])
        reps.append(dict(r=sysd["r"], v=sysd["v"], box=sysd["L"]))
    return reps


def melt(g, temps, steps_hot=600, steps_cold=600, every=10):
    """Velocity rescaling of every replica: to T* = 2.0, then each to its
    own T* (one device read and one scaling call per stride)."""
    temps = np.asarray(temps, dtype=np.float64)
    for target, steps in ((np.full(temps.size, 2.0), steps_hot), (temps, steps_cold)):
        for _ in range(steps // every):
            g.step(every)
            T = g.replica_observables_all()["T"]
            g.replica_scale_velocities(np.sqrt(target / T))


def transport(g, volumes, t_cut=T_CUT):
    """Per-replica readouts and Green-Kubo integrals of a batch handle:
    C_sigma (mean of xy, xz, yz), C_q (mean of x, y, z), T (mean over the
    correlated run), eta = V/T int C_sigma, kappa = V/T^2 int C_q."""
    nrep = g.nrep
    t, Cs = g.corr(_lib.MD_CORR_STRESS).read_rows(0, nrep, 3)
    _, Cq = g.corr(_lib.MD_CORR_HEATFLUX).read_rows(0, nrep, 3)
    T = g.replica_observables_all()["T_mean"]
    V = np.asarray(volumes, dtype=np.float64)
    eta = np.array([_lib.gk_integrate(t, Cs[r], t_cut=t_cut, prefactor=V[r] / T[r])[0] for r in range(nrep)])
    kappa = np.array([_lib.gk_integrate(t, Cq[r], t_cut=t_cut, prefactor=V[r] / T[r] ** 2)[0] for r in range(nrep)])
    return dict(t=t, Cs=Cs, Cq=Cq, T=T, eta=eta, kappa=kappa)


def generate(specs, short, long, *, precision=_lib.MD_PREC_MIXED, melt_steps=(600, 600), max_atoms=40_000_000,
             stream=None, sync=None):
    """Runs the replicas (batched, in handles of at most max_atoms atoms):
    melt, reset the correlators, `short` steps (features and short-run
    integrals), then on to `long` steps (the targets).  Returns a dict of
    arrays: X [n, 132], eta_short, kappa_short, eta_long, kappa_long, T, rho,
    V, atoms, steps_short, steps_long, and the seconds spent in the short
    and long phases."""
    out = {k: [] for k in ("X", "eta_short", "kappa_short", "eta_long", "kappa_long", "T", "rho", "V", "atoms")}
    t_short = t_long = 0.0
    sync = sync or (lambda: None)
    i = 0
    while i < len(specs):
        j, atoms = i, 0
        while j < len(specs) and (j == i or atoms + 4 * specs[j]["cells"] ** 3 <= max_atoms):
            atoms += 4 * specs[j]["cells"] ** 3
            j += 1
        chunk = specs[i:j]
        reps = build_replicas(chunk)
        mode = _lib.MD_PAIR_TILES if precision == _lib.MD_PREC_MIXED else _lib.MD_PAIR_VERLET
        p = _lib.make_params(1, 1.0, rc=RC, dt=DT, skin=0.2, precision=precision, pair_mode=mode, stress=SPEC,
                             heatflux=SPEC, vacf=None)
        g = _lib.System(p, replicas=reps, stream=stream)
        melt(g, [s["T"] for s in chunk], *melt_steps)
        g.reset_correlators()
        V = np.array([rp["box"] ** 3 for rp in reps])
        n = np.array([rp["r"].shape[1] for rp in reps])
        sync()
        t0 = time.perf_counter()
        g.step(short)
        sync()
        t_short += time.perf_counter() - t0
        a = transport(g, V)
        X = _lib.gk_tail_features(a["Cs"][:, :64], a["Cq"][:, :64], V, a["T"], n / V)
        t0 = time.perf_counter()
        g.step(long - short)
        sync()
        t_long += time.perf_counter() - t0
        b = transport(g, V)
        g.close()
        out["X"].append(X)
        out["eta_short"].append(a["eta"])
        out["kappa_short"].append(a["kappa"])
        out["eta_long"].append(b["eta"])
        out["kappa_long"].append(b["kappa"])
        out["T"].append(b["T"])
        out["rho"].append(n / V)
        out["V"].append(V)
        out["atoms"].append(n)
        i = j
    res = {k: np.concatenate(v) for k, v in out.items()}
    res["steps_short"] = np.full(len(specs), float(short))
    res["steps_long"] = np.full(len(specs), float(long))
    res["seconds_short"], res["seconds_long"] = t_short, t_long
    return res


class LearnedTail:
    """The network (3 x 128 tanh, bfloat16 tensor-core products) with the
    rule that decides where it is used (gk_tail_rule of the C ABI: the
    temperature-density box of its training set, its error on validation
    replicas, and the short-run integral's error coefficient).  Outputs
    (eta, kappa)."""

    def __init__(self, *, depth=3, batch=128, lr=1e-3, weight_decay=1e-3, seed=1, stream=None):
        self.net = _lib.MLP(N_FEATURES, 2, depth=depth, batch=batch, lr=lr, weight_decay=weight_decay, seed=seed,
                            stream=stream)
        self.rule = None

    @property
    def val_error(self):
        return tuple(self.rule.net_error)

    @property
    def short_coeff(self):
        return tuple(self.rule.short_coeff)

    def fit(self, train, val, epochs, shuffle_seed=1):
        """train, val: dicts as returned by generate() (rows with a
        non-positive long-run target are left out).  Trains on
        log(eta_long), log(kappa_long); returns the loss per epoch."""
        tr = _usable(train)
        X = np.ascontiguousarray(train["X"][tr], dtype=np.float32)
        Y = np.stack([np.log(train["eta_long"][tr]), np.log(train["kappa_long"][tr])], 1).astype(np.float32)
        self.net.fit_scaler(X, Y)
        rule = _lib.gk_tail_box(X[:, 130], X[:, 131])
        hist = self.net.train(X, Y, epochs, shuffle_seed=shuffle_seed)
        va = _usable(val)
        eta, kappa = self._net(val["X"][va])
        rule.net_error[0] = _lib.gk_tail_rms_rel(eta, val["eta_long"][va])
        rule.net_error[1] = _lib.gk_tail_rms_rel(kappa, val["kappa_long"][va])
        # the short-run integral's error falls as 1/sqrt(steps), whatever the size
        both = {k: np.concatenate([train[k][tr], val[k][va]])
                for k in ("eta_short", "kappa_short", "eta_long", "kappa_long", "steps_short")}
        for i, k in enumerate(("eta", "kappa")):
            rule.short_coeff[i] = _lib.gk_tail_rms_rel(both[k + "_short"], both[k + "_long"], both["steps_short"])
        self.rule = rule
        return hist

    def _net(self, X):
        Y = self.net.forward(np.ascontiguousarray(X, dtype=np.float32))
        return np.exp(Y[:, 0].astype(np.float64)), np.exp(Y[:, 1].astype(np.float64))

    def predict(self, X, eta_short, kappa_short, steps):
        """(eta, kappa, used_eta, used_kappa): per output, the network's value
        or the run's own integral, as gk_tail_choose decides."""
        X = np.ascontiguousarray(X, dtype=np.float32)
        eta, kappa = self._net(X)
        out, used = _lib.gk_tail_choose(self.rule, X[:, 130], X[:, 131], steps, np.stack([eta, kappa], 1),
                                        np.stack([np.asarray(eta_short, dtype=np.float64),
                                                  np.asarray(kappa_short, dtype=np.float64)], 1))
        return out[:, 0], out[:, 1], used[:, 0], used[:, 1]


def _usable(d):
    return (d["eta_long"] > 0) & (d["kappa_long"] > 0)


def _rms_rel(a, b):
    return float(np.sqrt(np.mean(((np.asarray(a) - b) / b) ** 2)))


def split(d, rows):
    """The rows `rows` (a slice or index array) of a generate() result."""
    return {k: (v[rows] if isinstance(v, np.ndarray) and v.ndim > 0 else v) for k, v in d.items()}
