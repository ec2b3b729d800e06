"""FP64 reference of the J-interpolation surrogate network. Test infrastructure only.

A fully connected network x (4 inputs) -> 3 hidden layers of width W with GELU ->
1 output, trained on mean-squared error with AdamW. Used to check the library's
hand-written forward, backward and optimiser kernels (gradient parity, one
optimiser step). GELU is the tanh form
  gelu(z) = z/2 (1 + tanh(s (z + 0.044715 z^3))),  s = sqrt(2/pi),
whose derivative is written out below.

parity note: the network itself is not part of the paper (it is one of this
project's extensions); its pins are finite differences and a closed-form AdamW step.
"""
from __future__ import annotations

import numpy as np

S = np.sqrt(2.0 / np.pi)
A = 0.044715


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(S * (z + A * z ** 3)))


def gelu_grad(z):
    u = S * (z + A * z ** 3)
    t = np.tanh(u)
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * S * (1.0 + 3.0 * A * z * z)


def init_params(sizes, seed):
    """He-style normal initialisation, zero biases (seeded)."""
    rng = np.random.default_rng(seed)
    params = []
    for fan_in, fan_out in zip(sizes[:-1], sizes[1:]):
        W = rng.standard_normal((fan_out, fan_in)) * np.sqrt(2.0 / fan_in)
        params.append([W, np.zeros(fan_out)])
    return params


def forward(params, X):
    """Returns the output (N,) and the cache of pre-activations / activations."""
    acts = [X]
    pres = []
    h = X
    for li, (W, b) in enumerate(params):
        z = h @ W.T + b
        pres.append(z)
        h = gelu(z) if li < len(params) - 1 else z
        acts.append(h)
    return h[:, 0], (pres, acts)


def loss_and_grads(params, X, y):
    """Mean-squared error 1/N sum (f(x) - y)^2 and its gradient by backpropagation."""
    out, (pres, acts) = forward(params, X)
    N = X.shape[0]
    r = out - y
    loss = np.mean(r * r)
    grads = [None] * len(params)
    g = (2.0 / N) * r[:, None]                        # dL/d(output pre-activation)
    for li in range(len(params) - 1, -1, -1):
        W, b = params[li]
        gW = g.T @ acts[li]
        gb = g.sum(axis=0)
        grads[li] = [gW, gb]
        if li > 0:
            g = (g @ W) * gelu_grad(pres[li - 1])
    return loss, grads


def adamw_step(params, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
    """One AdamW update (decoupled weight decay on weights, not biases)."""
    new = []
    for li, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        out_l = []
        for pi, (p, gp) in enumerate(((W, gW), (b, gb))):
            key = (li, pi)
            m[key] = beta1 * m.get(key, 0.0) + (1 - beta1) * gp
            v[key] = beta2 * v.get(key, 0.0) + (1 - beta2) * gp * gp
            mh = m[key] / (1 - beta1 ** t)
            vh = v[key] / (1 - beta2 ** t)
            decay = wd * p if pi == 0 else 0.0
            out_l.append(p - lr * (mh / (np.sqrt(vh) + eps) + decay))
        new.append(out_l)
    return new
