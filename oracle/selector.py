"""Oracle of the learned parameter selector: a plain FP64 multilayer perceptron.

TEST INFRASTRUCTURE ONLY (like everything under oracle/): the product path
never imports this module; tests, smoke() and the bench's CPU baseline may.

The selector is not part of the paper (which fixes one Chebyshev order for all
levels, Sect. 4, and the high-frequency level by the rule of Sect. 2.5): it maps
per-level features to a Chebyshev order and a direction refinement.  This file
is the textbook definition the CUDA kernels are checked against:

  network   4 -> 64 -> 64 -> 64 -> 2, tanh on the hidden layers, linear output;
            the weights enter the products rounded to FP16 (the GPU stores
            them so), everything else is FP64 here;
  loss      L = (1 / B) sum_b 1/2 |y_b - t_b|^2 over a batch of B samples;
  gradient  reverse-mode differentiation of L (backpropagation), w.r.t. the
            unrounded weights (straight-through the FP16 rounding);
  optimiser Adam (Kingma & Ba 2015): m = b1 m + (1 - b1) g,
            v = b2 v + (1 - b2) g^2, w -= lr (m / (1 - b1^k)) /
            (sqrt(v / (1 - b2^k)) + eps), k = step number from 1.

Parameter vector layout (8770 floats): W1 (64 x 4, row-major), b1 (64),
W2 (64 x 64), b2 (64), W3 (64 x 64), b3 (64), W4 (2 x 64), b4 (2).
Pinned by central finite differences of the loss (tests/test_oracle_selector.py)
and by a network whose output has a closed form.
"""
import numpy as np

SIZES = [(64, 4), (64, 64), (64, 64), (2, 64)]
N_PARAMS = sum(o * i + o for o, i in SIZES)


def unpack(theta):
    """List of (W, b) views of a flat parameter vector."""
    theta = np.asarray(theta)
    out, k = [], 0
    for o, i in SIZES:
        W = theta[k:k + o * i].reshape(o, i)
        k += o * i
        b = theta[k:k + o]
        k += o
        out.append((W, b))
    return out


def _round_fp16(theta, fp16):
    t = np.asarray(theta, dtype=np.float64)
    return t.astype(np.float16).astype(np.float64) if fp16 else t


def forward(theta, x, fp16=True):
    """Outputs (B, 2) and the hidden activations [h1, h2, h3] (B, 64) each."""
    layers = unpack(_round_fp16(theta, fp16))
    h = np.asarray(x, dtype=np.float64)
    acts = []
    for li, (W, b) in enumerate(layers):
        z = h @ W.T + b
        if li < len(layers) - 1:
            h = np.tanh(z)
            acts.append(h)
        else:
            h = z
    return h, acts


def loss_and_grad(theta, x, t, fp16=True):
    """(L, dL/dtheta) by backpropagation."""
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    B = x.shape[0]
    y, acts = forward(theta, x, fp16)
    r = y - t
    L = 0.5 * float(np.sum(r * r)) / B
    layers = unpack(_round_fp16(theta, fp16))
    inputs = [x] + acts                     # input of layer li
    grads = [None] * len(layers)
    delta = r / B                           # dL/dz of the output layer
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        grads[li] = (delta.T @ inputs[li], delta.sum(axis=0))
        if li > 0:
            delta = (delta @ W) * (1.0 - acts[li - 1] ** 2)
    g = np.concatenate([np.concatenate([dW.ravel(), db]) for dW, db in grads])
    return L, g


def adam_train(theta, x, t, epochs, lr, b1=0.9, b2=0.999, eps=1e-8, fp16=True):
    """Full-batch Adam for `epochs` steps; returns (theta, losses before each step)."""
    theta = np.array(theta, dtype=np.float64)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    losses = []
    for k in range(1, epochs + 1):
        L, g = loss_and_grad(theta, x, t, fp16)
        losses.append(L)
        m = b1 * m + (1.0 - b1) * g
        v = b2 * v + (1.0 - b2) * g * g
        mh = m / (1.0 - b1 ** k)
        vh = v / (1.0 - b2 ** k)
        theta = theta - lr * mh / (np.sqrt(vh) + eps)
    return theta, np.array(losses)
