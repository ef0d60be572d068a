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
