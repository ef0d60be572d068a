"""Plain FP64 CPU oracle of the learned Green-Kubo tail (test infrastructure
only: the test suite, the smoke check and the CPU legs of ``bench.py`` use
it; the GPU library never does).

The paper (arXiv 2503.07526) has no learned component.  What it fixes is the
input and the target of this model:
  * the inputs are read out of the multiple-tau correlators of the shear
    stress and the heat flux (Sec. 2.2 Eq. (cor); Appendix D Algorithm 2:
    level 1 gives lags 0..p-1, every higher level k gives lags p/m..p-1 in
    units of m^(k-1) samples), here the first 64 readout points;
  * the targets are the Green-Kubo viscosity and thermal conductivity of
    Sec. 2.3: eta = V/T int <s_ab(t) s_ab(0)> dt (mean over xy, xz, yz) and
    kappa = V/(3 T^2) int <q(t).q(0)> dt.
The network itself is this project's definition, written out here in the
plain order of its steps:
  x (n_in) -> [z = h W^T + b, h = tanh(z)] x depth -> y = h W^T + b (n_out),
loss = mean over the batch and the outputs of (y - t)^2, trained by Adam with
decoupled weight decay on the weight matrices (not the biases).

``emulate=True`` rounds to bfloat16 at exactly the points where the GPU
kernels hold a bfloat16 operand of a tensor-core product: the inputs, the
weight copies, every stored activation (which also feeds tanh' = 1 - h^2),
the output gradient dY and every pre-activation gradient dZ.  Sums are FP64
here (FP32 on the GPU).

Pins (tests/test_oracle_mlp.py): the backward pass against central finite
differences of the loss; Adam's first step and its beta1 = beta2 = 0 limit in
closed form; the features of an exponential correlation function in closed
form; the bfloat16 rounding against exactly representable values and ties.
"""
from __future__ import annotations

import numpy as np

N_POINTS = 64  # readout points per correlation function fed to the network


def bf16(a):
    """Rounds to the nearest bfloat16 value (ties to even), as float64.
    The value is first rounded to float32, as the GPU holds it."""
    a32 = np.ascontiguousarray(a, dtype=np.float32)
    bits = a32.view(np.uint32).astype(np.uint64)
    rounded = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(a))


def _r(a, emulate):
    return bf16(a) if emulate else np.asarray(a, dtype=np.float64)


def forward(params, X, emulate=True):
    """params: list of (W [out, in], b [out]) per layer, the last one linear.
    Returns (y [B, n_out], cache of the stored activations)."""
    h = _r(X, emulate)
    hs = [h]
    for l, (W, b) in enumerate(params):
        z = h @ _r(W, emulate).T + np.asarray(b, dtype=np.float64)
        if l == len(params) - 1:
            return z, hs
        h = _r(np.tanh(z), emulate)
        hs.append(h)
    raise ValueError("no layers")


def loss(y, t):
    """Mean over the batch and the outputs of the squared error."""
    d = y - np.asarray(t, dtype=np.float64)
    return float(np.mean(d * d))


def backward(params, hs, y, t, emulate=True):
    """Gradients [(dW, db)] of ``loss`` by reverse-mode differentiation.
    hs[l] is the input of layer l (hs[0] = x)."""
    B, n_out = y.shape
    dz = _r(2.0 * (y - np.asarray(t, dtype=np.float64)) / (B * n_out), emulate)
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        grads[l] = (dz.T @ hs[l], dz.sum(axis=0))
        if l == 0:
            break
        dh = dz @ _r(W, emulate)
        h = hs[l]
        dz = _r(dh * (1.0 - h * h), emulate)
    return grads


def adam(params, grads, state, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0):
    """One Adam step with bias correction and decoupled weight decay on the
    weight matrices.  state: dict with 't' and per-array moments (created on
    first use).  Returns the new params."""
    t = state.get("t", 0) + 1
    state["t"] = t
    out = []
    for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        new = []
        for k, (w, g) in enumerate(((W, gW), (b, gb))):
            key = (l, k)
            m, v = state.get(key, (np.zeros_like(w, dtype=np.float64), np.zeros_like(w, dtype=np.float64)))
            m = beta1 * m + (1.0 - beta1) * g
            v = beta2 * v + (1.0 - beta2) * g * g
            state[key] = (m, v)
            mh = m / (1.0 - beta1 ** t)
            vh = v / (1.0 - beta2 ** t)
            step = mh / (np.sqrt(vh) + eps)
            if k == 0:
                step = step + weight_decay * w
            new.append(w - lr * step)
        out.append(tuple(new))
    return out


def tail_features(t, c_sigma, c_q, volume, temperature, density):
    """The network's input for one run: the first 64 readout points of the
    shear-stress and heat-flux autocorrelations normalised by their lag-0
    value, the logarithm of the intensive lag-0 scale of each (V C(0)/T for
    the stress, V C(0)/T^2 for the heat flux: the Green-Kubo prefactors of
    Sec. 2.3 times C(0)), then T and the number density.  t is unused beyond
    checking that there are 64 points."""
    if len(t) < N_POINTS or len(c_sigma) < N_POINTS or len(c_q) < N_POINTS:
        raise ValueError("fewer than 64 readout points")
    cs = np.asarray(c_sigma[:N_POINTS], dtype=np.float64)
    cq = np.asarray(c_q[:N_POINTS], dtype=np.float64)
    return np.concatenate([cs / cs[0], [np.log(volume * cs[0] / temperature)],
                           cq / cq[0], [np.log(volume * cq[0] / temperature ** 2)],
                           [temperature, density]])


def train(params, X, T, *, epochs, batch, order, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
          weight_decay=0.0, emulate=True):
    """Mini-batch training: ``order`` [epochs, n] gives the sample order of
    each epoch; the last incomplete batch of an epoch is dropped.  Returns
    (params, mean loss per epoch)."""
    state = {}
    hist = []
    n = X.shape[0]
    for e in range(epochs):
        losses = []
        for b0 in range(0, n - batch + 1, batch):
            idx = order[e][b0:b0 + batch]
            y, hs = forward(params, X[idx], emulate)
            losses.append(loss(y, T[idx]))
            g = backward(params, hs, y, T[idx], emulate)
            params = adam(params, g, state, lr, beta1, beta2, eps, weight_decay)
        hist.append(float(np.mean(losses)))
    return params, np.array(hist)
