"""Host-side parts of the learned tail (no GPU): the feature builder of the
C ABI against the oracle's definition."""
import numpy as np
import pytest

from paper_2503_07526_gb300 import synth


@pytest.fixture(scope="module")
def pkg():
    from paper_2503_07526_gb300 import build_lib

    build_lib.build()
    import paper_2503_07526_gb300 as pkg

    return pkg


def test_features_match_oracle(pkg):
    from oracle import mlp

    t = np.concatenate([np.arange(16.0)] + [np.arange(8.0, 16.0) * 2 ** (k - 1) for k in range(2, 10)])
    nr = 6
    A = 1e-4 * (1 + synth.uniform01(1, nr))
    tau = 5 + 50 * synth.uniform01(2, nr)
    cs = A[:, None] * np.exp(-t[None, :] / tau[:, None]) + 1e-6 * synth.normal(3, nr * t.size).reshape(nr, -1)
    cq = 2 * A[:, None] * np.cos(t[None, :] / tau[:, None])
    V, T, rho = 1000 + 9000 * synth.uniform01(4, nr), 0.7 + 1.3 * synth.uniform01(5, nr), 0.7 + 0.2 * synth.uniform01(6, nr)
    got = pkg.gk_tail_features(cs, cq, V, T, rho)
    assert got.shape == (nr, 132) and got.dtype == np.float32
    for r in range(nr):
        want = mlp.tail_features(t, cs[r], cq[r], V[r], T[r], rho[r])
        assert np.array_equal(got[r], want.astype(np.float32)), r
    bad = cs.copy()
    bad[2, 0] = -1.0
    with pytest.raises(pkg.MdError):
        pkg.gk_tail_features(bad, cq, V, T, rho)
    with pytest.raises(pkg.MdError):
        pkg.gk_tail_features(cs[:, :63], cq[:, :63], V, T, rho)


def test_tail_rule_calls(pkg):
    """The learned tail's rule behind the C ABI against the rule restated
    here: the training box, the rms relative errors (plain and weighted by
    steps) and the per-run choice between the network and the run's own
    integral."""
    nr = 40
    T = 0.7 + 1.3 * synth.uniform01(31, nr)
    rho = 0.7 + 0.2 * synth.uniform01(32, nr)
    rule = pkg.gk_tail_box(T[:30], rho[:30])
    assert (rule.T_min, rule.T_max, rule.rho_min, rule.rho_max) == (T[:30].min(), T[:30].max(), rho[:30].min(),
                                                                    rho[:30].max())
    a = 1.0 + 0.3 * synth.normal(33, nr)
    b = 1.0 + 0.1 * synth.uniform01(34, nr)
    w = 1000.0 + 4000.0 * synth.uniform01(35, nr)
    assert pkg.gk_tail_rms_rel(a, b) == pytest.approx(np.sqrt(np.mean(((a - b) / b) ** 2)), rel=1e-14)
    assert pkg.gk_tail_rms_rel(a, b, w) == pytest.approx(np.sqrt(np.mean(((a - b) / b) ** 2 * w)), rel=1e-14)
    rule.net_error[0], rule.net_error[1] = 0.1, 0.15
    rule.short_coeff[0], rule.short_coeff[1] = 20.0, 30.0
    steps = 2000.0 + 60000.0 * synth.uniform01(36, nr)
    net = np.stack([2.0 + synth.uniform01(37, nr), 5.0 + synth.uniform01(38, nr)], 1)
    own = np.stack([3.0 + synth.uniform01(39, nr), 7.0 + synth.uniform01(40, nr)], 1)
    out, used = pkg.gk_tail_choose(rule, T, rho, steps, net, own)
    inside = (T >= rule.T_min) & (T <= rule.T_max) & (rho >= rule.rho_min) & (rho <= rule.rho_max)
    for k in range(2):
        want_used = inside & (np.array(rule.short_coeff)[k] / np.sqrt(steps) > np.array(rule.net_error)[k])
        assert np.array_equal(used[:, k], want_used)
        assert np.array_equal(out[:, k], np.where(want_used, net[:, k], own[:, k]))
    assert used.any() and (~used).any()
    with pytest.raises(pkg.MdError):
        pkg.gk_tail_choose(rule, T, rho, np.zeros(nr), net, own)
