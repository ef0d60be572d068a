"""Pins of the learned-tail oracle (oracle/mlp.py) against what mathematics
fixes: finite differences of the loss, Adam's closed-form steps, bfloat16
rounding of exactly known values, the features of a closed-form correlation
function.  CPU only."""
import numpy as np
import pytest

from oracle import mlp
from paper_2503_07526_gb300 import synth


def tiny_net(seed=3, dims=(5, 7, 6, 7, 2)):
    return synth.mlp_init(seed, dims, bias_scale=0.3)


def test_bf16_rounding_pins():
    exact = np.array([1.0, -0.5, 3.0, 2.0 ** -20, 1.0 + 2.0 ** -7, 65280.0])
    assert np.array_equal(mlp.bf16(exact), exact)
    # halfway cases go to the even mantissa
    assert mlp.bf16(1.0 + 2.0 ** -8) == 1.0
    assert mlp.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert mlp.bf16(-(1.0 + 3 * 2.0 ** -8)) == -(1.0 + 2.0 ** -6)
    # just above a tie goes up
    assert mlp.bf16(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    torch = pytest.importorskip("torch")
    x = synth.normal(11, 4096) * 10.0 ** synth.uniform01(12, 4096) * 3
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), want)


@pytest.mark.parametrize("emulate", [False])
def test_backward_equals_finite_differences(emulate):
    params = tiny_net()
    X = synth.normal(21, 6 * 5).reshape(6, 5)
    T = synth.normal(22, 6 * 2).reshape(6, 2)
    y, hs = mlp.forward(params, X, emulate)
    grads = mlp.backward(params, hs, y, T, emulate)
    h = 1e-6

    def L(ps):
        return mlp.loss(mlp.forward(ps, X, emulate)[0], T)

    for l, (W, b) in enumerate(params):
        for k, arr in enumerate((W, b)):
            fd = np.zeros_like(arr)
            for idx in np.ndindex(arr.shape):
                ps_p = [(w.copy(), bb.copy()) for w, bb in params]
                ps_m = [(w.copy(), bb.copy()) for w, bb in params]
                ps_p[l][k][idx] += h
                ps_m[l][k][idx] -= h
                fd[idx] = (L(ps_p) - L(ps_m)) / (2 * h)
            g = grads[l][k]
            assert np.abs(g - fd).max() <= 1e-8 * max(1.0, np.abs(fd).max()), (l, k)


def test_emulated_backward_within_bf16_bound():
    """Rounding at the bfloat16 points perturbs each gradient by a few
    bfloat16 units (2^-8 relative) at most, normwise."""
    params = tiny_net(dims=(16, 32, 32, 32, 2))
    X = synth.normal(31, 64 * 16).reshape(64, 16)
    T = synth.normal(32, 64 * 2).reshape(64, 2)
    ye, he = mlp.forward(params, X, True)
    yx, hx = mlp.forward(params, X, False)
    assert np.abs(ye - yx).max() <= 8 * 2.0 ** -8 * np.abs(yx).max()
    ge = mlp.backward(params, he, ye, T, True)
    gx = mlp.backward(params, hx, yx, T, False)
    for (a, b), (c, d) in zip(ge, gx):
        assert np.abs(a - c).max() <= 16 * 2.0 ** -8 * np.abs(c).max()
        assert np.abs(b - d).max() <= 16 * 2.0 ** -8 * np.abs(d).max()


def test_adam_closed_forms():
    w0 = np.array([[0.5, -1.0]]), np.array([0.25])
    g = np.array([[0.2, -3.0]]), np.array([1e-9])
    lr, eps, wd = 0.01, 1e-8, 0.1
    # first step: the bias-corrected moments are g and g^2 exactly
    st = {}
    (w1, b1), = mlp.adam([w0], [g], st, lr=lr, eps=eps, weight_decay=wd)
    assert np.allclose(w1, w0[0] - lr * (g[0] / (np.abs(g[0]) + eps) + wd * w0[0]), rtol=0, atol=1e-15)
    assert np.allclose(b1, w0[1] - lr * g[1] / (np.abs(g[1]) + eps), rtol=0, atol=1e-15)
    # a constant gradient keeps the corrected moments at g and g^2 on every step
    st, ws = {}, [w0]
    for k in range(5):
        ws = mlp.adam(ws, [g], st, lr=lr, eps=eps)
    assert np.allclose(ws[0][0], w0[0] - 5 * lr * g[0] / (np.abs(g[0]) + eps), rtol=0, atol=1e-13)
    # beta1 = beta2 = 0: sign descent with the eps guard, whatever the history
    st, ws = {}, [w0]
    gs = [(np.array([[1.0, -2.0]]), np.array([0.5])), (np.array([[-4.0, 1e-3]]), np.array([-0.5]))]
    for gg in gs:
        ws = mlp.adam(ws, [gg], st, lr=lr, beta1=0.0, beta2=0.0, eps=eps)
    want = w0[0] - lr * sum(gg[0] / (np.abs(gg[0]) + eps) for gg in gs)
    assert np.allclose(ws[0][0], want, rtol=0, atol=1e-15)


def test_features_of_exponential_correlation():
    """C(t) = A exp(-t/tau) on the multiple-tau readout grid (p = 16, m = 2:
    lags 0..15 then 8..15 x 2^(k-1)) gives g = exp(-t/tau) and the log of the
    Green-Kubo scale."""
    t = np.concatenate([np.arange(16.0)] + [np.arange(8.0, 16.0) * 2 ** (k - 1) for k in range(2, 9)])
    A, tau, Aq, tauq, V, T, rho = 3e-4, 40.0, 2e-3, 25.0, 1234.5, 1.3, 0.8
    f = mlp.tail_features(t, A * np.exp(-t / tau), Aq * np.exp(-t / tauq), V, T, rho)
    assert f.shape == (132,)
    assert np.allclose(f[:64], np.exp(-t[:64] / tau), rtol=1e-15, atol=0)
    assert f[64] == pytest.approx(np.log(V * A / T), rel=1e-15)
    assert np.allclose(f[65:129], np.exp(-t[:64] / tauq), rtol=1e-15, atol=0)
    assert f[129] == pytest.approx(np.log(V * Aq / T ** 2), rel=1e-15)
    assert list(f[130:]) == [T, rho]
    with pytest.raises(ValueError):
        mlp.tail_features(t[:63], t[:63], t[:63], V, T, rho)


def test_training_fits_a_teacher():
    """A student of the same shape reaches a small fraction of its initial
    loss on targets written by a fixed random teacher network."""
    dims = (12, 32, 32, 32, 2)
    teacher = synth.mlp_init(41, dims, bias_scale=0.2)
    X = synth.normal(42, 512 * 12).reshape(512, 12)
    T, _ = mlp.forward(teacher, X, emulate=False)
    student = synth.mlp_init(43, dims)
    order = synth.permutations(44, 60, 512)
    y0, _ = mlp.forward(student, X, True)
    _, hist = mlp.train(student, X, T, epochs=60, batch=128, order=order, lr=3e-3)
    assert hist[-1] < 0.1 * mlp.loss(y0, T)
