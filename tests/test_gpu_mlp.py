"""The learned-tail network on the tensor cores against the FP64 oracle
(oracle/mlp.py): initialisation, forward pass, loss and gradients of every
layer, Adam, and a whole training run, through the C ABI of
include/gk_tail.h.

Tolerances.  The oracle rounds to bfloat16 at the same points as the GPU
(emulate=True) and sums in FP64; the GPU sums in FP32 on the tensor cores.
FP32 sums of 132-256 products differ from FP64 by about 1e-6 relative, and
where such a difference straddles a bfloat16 rounding boundary the stored
value moves by one bfloat16 unit (2^-8 = 3.9e-3 relative).  That happens to
about one element in 2,000 (0.2 per row of the three-layer network), and one
such flip moves an output by at most |w| 2^-8.  Measured on GB300: outputs
7e-8 (1 row), 7e-4 (300 rows), 1.1e-3 (4,227 rows) normwise, gradients
1e-4 to 3e-4.  The tests allow one bfloat16 unit, 4e-3, for both.  Against
the oracle without bfloat16 rounding (the FP64 network on the same FP32
weights) the bfloat16 error itself shows: 4e-3 to 6e-3 measured, 3e-2
(outputs) and 6e-2 (gradients) allowed."""
import numpy as np
import pytest

from paper_2503_07526_gb300 import synth

pytestmark = pytest.mark.gpu

DIMS = (132, 128, 128, 128, 2)


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_07526_gb300 as pkg

    pkg.lib(build=True)
    return pkg


@pytest.fixture(scope="module")
def omlp():
    from oracle import mlp

    return mlp


def rel(a, b):
    return float(np.abs(np.asarray(a, dtype=np.float64) - b).max() / np.abs(b).max())


def f32(params):
    return [(W.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)) for W, b in params]


def test_initialisation_is_glorot_uniform(pkg):
    net = pkg.MLP(132, 2, seed=7)
    want = synth.mlp_init(7, DIMS)
    got = net.get_params()
    for (W, b), (Wg, bg) in zip(want, got):
        assert np.array_equal(Wg, W.astype(np.float32).astype(np.float64))
        assert not bg.any()
    assert net.nparams == sum(W.size + b.size for W, b in want)


@pytest.mark.parametrize("rows", [1, 300, 4096 + 131])
def test_forward_matches_oracle(pkg, omlp, rows):
    params = f32(synth.mlp_init(11, DIMS, bias_scale=0.2))
    net = pkg.MLP(132, 2, seed=1)
    net.set_params(params)
    X = (synth.normal(12 + rows, rows * 132).reshape(rows, 132)).astype(np.float32)
    Y = net.forward(X)
    ye, _ = omlp.forward(params, X.astype(np.float64), emulate=True)
    yx, _ = omlp.forward(params, X.astype(np.float64), emulate=False)
    e_emul, e_exact = rel(Y, ye), rel(Y, yx)
    print(f"rows {rows}: vs bf16-emulating oracle {e_emul:.2e}, vs FP64 network {e_exact:.2e}")
    assert e_emul <= 4e-3
    assert e_exact <= 3e-2


def test_forward_layered_path_matches_oracle(pkg, omlp):
    """A five-layer network's weights and activation tiles do not fit one
    CTA's shared memory, so its forward pass runs layer by layer (one
    tensor-core product per layer); same bound as the fused pass."""
    dims = (132, 128, 128, 128, 128, 128, 2)
    params = f32(synth.mlp_init(21, dims, bias_scale=0.2))
    net = pkg.MLP(132, 2, depth=5, seed=1)
    net.set_params(params)
    X = synth.normal(22, 700 * 132).reshape(700, 132).astype(np.float32)
    Y = net.forward(X)
    ye, _ = omlp.forward(params, X.astype(np.float64), emulate=True)
    assert rel(Y, ye) <= 4e-3


def test_forward_many_tiles_device_buffers(pkg, omlp):
    """The fused pass over 1,205 tiles (each CTA loops over several, two at a
    time) from and to device memory: sampled rows against the oracle, and
    every sampled row equal bit for bit to the same row run in a small batch
    on the host path (rows are independent and take the same arithmetic)."""
    import torch

    params = f32(synth.mlp_init(31, DIMS, bias_scale=0.2))
    net = pkg.MLP(132, 2, seed=1)
    net.set_params(params)
    rows = 128 * 1204 + 77
    X = synth.normal(32, rows * 132).reshape(rows, 132).astype(np.float32)
    Yd = net.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    idx = np.unique(np.concatenate([np.arange(130), synth.permutations(33, 1, rows)[0, :1500],
                                    np.arange(rows - 130, rows)]))
    ye, _ = omlp.forward(params, X[idx].astype(np.float64), emulate=True)
    assert rel(Yd[idx], ye) <= 4e-3
    Ys = net.forward(np.ascontiguousarray(X[idx]))
    assert np.array_equal(Ys, Yd[idx])


def test_loss_and_gradients_match_oracle(pkg, omlp):
    B = 256
    params = f32(synth.mlp_init(21, DIMS, bias_scale=0.2))
    net = pkg.MLP(132, 2, batch=B)
    net.set_params(params)
    X = synth.normal(22, B * 132).reshape(B, 132).astype(np.float32)
    T = (2.0 * synth.normal(23, B * 2).reshape(B, 2)).astype(np.float32)
    loss, g = net.loss_grad(X, T)
    ye, hs = omlp.forward(params, X.astype(np.float64), True)
    assert loss == pytest.approx(omlp.loss(ye, T.astype(np.float64)), rel=1e-5)
    ge = omlp.backward(params, hs, ye, T.astype(np.float64), True)
    gx_y, gx_h = omlp.forward(params, X.astype(np.float64), False)
    gx = omlp.backward(params, gx_h, gx_y, T.astype(np.float64), False)
    for l, ((gW, gb), (oW, ob), (xW, xb)) in enumerate(zip(net.unflatten(g), ge, gx)):
        print(f"layer {l}: dW {rel(gW, oW):.2e} db {rel(gb, ob):.2e} (vs FP64 network {rel(gW, xW):.2e})")
        assert rel(gW, oW) <= 4e-3, l
        assert rel(gb, ob) <= 4e-3, l
        assert rel(gW, xW) <= 6e-2, l


def test_adam_steps_match_oracle(pkg, omlp):
    params = f32(synth.mlp_init(31, DIMS, bias_scale=0.2))
    kw = dict(lr=1e-2, beta1=0.9, beta2=0.99, eps=1e-8, weight_decay=0.05)
    net = pkg.MLP(132, 2, **kw)
    net.set_params(params)
    st, po = {}, params
    for k in range(3):
        g = (synth.normal(40 + k, net.nparams) * 1e-2).astype(np.float32)
        net.adam_step(g)
        po = omlp.adam(po, net.unflatten(g), st, **kw)
    got = net.get_params()
    for (W, b), (Wo, bo) in zip(got, po):
        assert np.abs(W - Wo).max() <= 2e-6
        assert np.abs(b - bo).max() <= 2e-6


def test_training_tracks_oracle(pkg, omlp):
    dims = (20, 128, 128, 2)
    teacher = synth.mlp_init(51, dims, bias_scale=0.2)
    n, epochs, B = 512, 30, 128
    X = synth.normal(52, n * 20).reshape(n, 20).astype(np.float32)
    T, _ = omlp.forward(teacher, X.astype(np.float64), emulate=False)
    T = T.astype(np.float32)
    start = f32(synth.mlp_init(53, dims))
    order = synth.permutations(54, epochs, n)
    net = pkg.MLP(20, 2, depth=2, batch=B, lr=3e-3)
    net.set_params(start)
    hist = net.train(X, T, epochs, order=order)
    _, ho = omlp.train(start, X.astype(np.float64), T.astype(np.float64), epochs=epochs, batch=B, order=order,
                       lr=3e-3, emulate=True)
    print("GPU   ", np.array2string(hist[::5], precision=4))
    print("oracle", np.array2string(ho[::5], precision=4))
    assert np.all(np.abs(hist - ho) <= 0.05 * ho)
    assert hist[-1] < 0.2 * hist[0]


def test_scaler_and_bad_arguments(pkg, omlp):
    params = f32(synth.mlp_init(61, DIMS, bias_scale=0.1))
    net = pkg.MLP(132, 2)
    net.set_params(params)
    X = (3.0 + 2.0 * synth.normal(62, 200 * 132).reshape(200, 132)).astype(np.float32)
    T = (np.stack([5 + synth.normal(63, 200), -1 + 0.1 * synth.normal(64, 200)], 1)).astype(np.float32)
    net.fit_scaler(X, T)
    mu, sd = X.astype(np.float64).mean(0), X.astype(np.float64).std(0)
    tmu, tsd = T.astype(np.float64).mean(0), T.astype(np.float64).std(0)
    Y = net.forward(X)
    Xs = ((X - mu.astype(np.float32)) / sd.astype(np.float32)).astype(np.float32)
    ye, _ = omlp.forward(params, Xs.astype(np.float64), emulate=True)
    assert rel(Y, ye * tsd + tmu) <= 4e-3
    with pytest.raises(pkg.MdError):
        pkg.MLP(132, 2, width=96)
    with pytest.raises(pkg.MdError):
        pkg.MLP(132, 2, batch=200)
    with pytest.raises(pkg.MdError):
        net.loss_grad(X[:100], T[:100])


def test_corr_read_rows_equals_corr_read(pkg):
    c = pkg.Corr.create(6, 16, 2, 12)
    x = synth.ar1_series(12, 700, 0.9, 5)
    for row in x:
        c.push(row)
    t, rows = c.read_rows(0, 12, 1)
    for g in range(12):
        tg, vg = c.read(g)
        assert np.array_equal(t, tg) and np.array_equal(rows[g], vg)
    t3, r3 = c.read_rows(3, 3, 3)
    for i in range(3):
        want = np.mean([c.read(3 + 3 * i + a)[1] for a in range(3)], axis=0)
        assert np.allclose(r3[i], want, rtol=1e-14, atol=0)
    with pytest.raises(pkg.MdError):
        c.read_rows(10, 1, 3)


def test_pipeline_wait_timeout_is_an_error_status(pkg, omlp):
    """A tensor-core pipeline wait that runs out ends the call with
    MD_ETIMEOUT and leaves the handle usable.  The wait limit is set to 0,
    so the first wait on a TMA panel or a stage's products that is not
    already complete gives up (the copies and products already issued are
    still waited for before the CTA exits); no wait is left unbounded and
    nothing traps.  With the default limit restored the same call matches
    the oracle again."""
    B = 256
    params = f32(synth.mlp_init(41, DIMS, bias_scale=0.2))
    net = pkg.MLP(132, 2, batch=B)
    net.set_params(params)
    X = synth.normal(42, B * 132).reshape(B, 132).astype(np.float32)
    T = synth.normal(43, B * 2).reshape(B, 2).astype(np.float32)
    net.set_wait_limit(0)
    with pytest.raises(pkg.MdError) as ei:
        net.loss_grad(X, T)
    assert ei.value.code == -5  # MD_ETIMEOUT
    with pytest.raises(pkg.MdError):
        net.set_wait_limit(-1)
    net.set_wait_limit(2_000_000_000)
    net.set_params(params)
    loss, _ = net.loss_grad(X, T)
    ye, _ = omlp.forward(params, X.astype(np.float64), True)
    assert loss == pytest.approx(omlp.loss(ye, T.astype(np.float64)), rel=1e-5)
    net.close()
