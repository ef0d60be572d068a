"""What the learned Green-Kubo tail gains over the method without it.

512 LJ replicas (sizes log-uniform in [500, 4,000] atoms, rho* uniform in
[0.7, 0.9], T* uniform in [0.7, 2.0]) run in one batch: melt, then 2,000
correlated steps (the short run: the network's features and the plain
Green-Kubo integral of the method) and on to 20,000 steps (the long run: the
targets, and the judge).  The network is trained on replicas 0-255 by its
own tensor-core kernels, validated on 256-383 and judged on 384-511: its
eta and kappa must sit closer to the long-run integrals than the short-run
integrals do (root-mean-square relative error, both against the same long
run).  The fallback rule must send a long run (200,000 steps) back to its
own integral, and keep the network for a short run of any size."""
import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_07526_gb300 as pkg

    pkg.lib(build=True)
    return pkg


def rms_rel(a, b):
    return float(np.sqrt(np.mean(((a - b) / b) ** 2)))


def test_learned_tail_beats_the_short_run_integral(pkg):
    from paper_2503_07526_gb300 import learned_tail as lt

    specs = lt.ensemble_specs(512, seed=5, n_range=(500, 4000))
    d = lt.generate(specs, 2000, 20000)
    assert d["X"].shape == (512, 132) and np.all(np.isfinite(d["X"]))
    assert np.all(d["eta_long"] > 0) and np.all(d["kappa_long"] > 0)
    tr, va, te = (lt.split(d, slice(a, b)) for a, b in ((0, 256), (256, 384), (384, 512)))
    m = lt.LearnedTail(lr=1e-3, weight_decay=1e-3, seed=1)
    hist = m.fit(tr, va, epochs=30)
    assert hist[-1] < 0.5 * hist[0]
    eta, kappa, ue, uk = m.predict(te["X"], te["eta_short"], te["kappa_short"], te["steps_short"])
    e_net, e_short = rms_rel(eta, te["eta_long"]), rms_rel(te["eta_short"], te["eta_long"])
    k_net, k_short = rms_rel(kappa, te["kappa_long"]), rms_rel(te["kappa_short"], te["kappa_long"])
    print(f"eta: learned tail {e_net:.3f}, short-run integral {e_short:.3f}; kappa: learned tail {k_net:.3f}, "
          f"short-run integral {k_short:.3f}; network used on {ue.mean():.0%} / {uk.mean():.0%}; validation "
          f"error {m.val_error}, short-run coefficients {m.short_coeff}")
    assert e_net < 0.75 * e_short
    assert k_net < 0.75 * k_short
    # fallback: outside the training box, and for a run long enough that its
    # own integral is the more precise
    X2 = te["X"][:3].copy()
    X2[0, 130] = 5.0
    e2, k2, u2e, u2k = m.predict(X2, te["eta_short"][:3], te["kappa_short"][:3], [2000, 200_000, 5000])
    assert not u2e[0] and not u2k[0] and e2[0] == te["eta_short"][0] and k2[0] == te["kappa_short"][0]
    assert not u2e[1] and not u2k[1] and e2[1] == te["eta_short"][1]
    assert u2e[2] and u2k[2]
