"""Reference of the learned cost model's network (test infrastructure).

Plain NumPy, float64: the network the library's hand-written kernels
implement -- inputs normalised as (x - mean) * scale, n_layers hidden ReLU
layers, one linear output -- its mean-squared-error loss, the loss's
gradients by backpropagation, and one Adam step.  Parameters use the
library's flat layout: for each layer W (out x in, row-major) then b (out).
Only tests may import this module.
"""
import numpy as np


def layer_shapes(n_in, n_hidden, n_layers):
    dims = [n_in] + [n_hidden] * n_layers + [1]
    return [(dims[i + 1], dims[i]) for i in range(len(dims) - 1)]


def unpack(params, n_in, n_hidden, n_layers):
    out, o = [], 0
    for (fo, fi) in layer_shapes(n_in, n_hidden, n_layers):
        W = params[o:o + fo * fi].reshape(fo, fi)
        o += fo * fi
        b = params[o:o + fo]
        o += fo
        out.append((W, b))
    assert o == len(params)
    return out


def forward(params, mean, scale, X, n_in, n_hidden, n_layers):
    """Activations of every layer (the first is the normalised input)."""
    acts = [(np.asarray(X, np.float64) - mean) * scale]
    layers = unpack(np.asarray(params, np.float64), n_in, n_hidden, n_layers)
    for li, (W, b) in enumerate(layers):
        z = acts[-1] @ W.T + b
        acts.append(np.maximum(z, 0.0) if li < len(layers) - 1 else z)
    return acts


def loss(params, mean, scale, X, t, n_in, n_hidden, n_layers):
    y = forward(params, mean, scale, X, n_in, n_hidden, n_layers)[-1][:, 0]
    return float(np.mean((y - np.asarray(t, np.float64)) ** 2))


def gradients(params, mean, scale, X, t, n_in, n_hidden, n_layers):
    """d loss / d params by backpropagation, in the flat layout."""
    acts = forward(params, mean, scale, X, n_in, n_hidden, n_layers)
    layers = unpack(np.asarray(params, np.float64), n_in, n_hidden, n_layers)
    n = acts[0].shape[0]
    d = (2.0 / n) * (acts[-1][:, 0] - np.asarray(t, np.float64))[:, None]   # dL/dy
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        grads[li] = (d.T @ acts[li], d.sum(axis=0))
        if li > 0:
            d = (d @ W) * (acts[li] > 0)   # through the ReLU of the layer below
    return np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])


def adam_step(params, grad, m1, m2, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    m1 = b1 * m1 + (1 - b1) * grad
    m2 = b2 * m2 + (1 - b2) * grad * grad
    p = params - lr * (m1 / (1 - b1 ** step)) / (np.sqrt(m2 / (1 - b2 ** step)) + eps)
    return p, m1, m2
