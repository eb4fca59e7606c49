"""FP64 numpy oracle of the sweep-proposer network (test infrastructure only).

x -> tanh(W1 x + b1) -> tanh(W2 h1 + b2) -> y = W3 h2 + b3,
L = 1/(2B) sum (y - t)^2, gradients by the chain rule written out layer by
layer, Adam with bias correction.  Parameter layout: flat
[W1 (H x I), b1, W2 (H x H), b2, W3 (O x H), b3].
"""
import numpy as np


def count(I, H, O):
    return H * I + H + H * H + H + O * H + O


def unpack(p, I, H, O):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * I].reshape(H, I); o += H * I
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + O * H].reshape(O, H); o += O * H
    b3 = p[o:o + O]; o += O
    return W1, b1, W2, b2, W3, b3


def forward(p, x, I, H, O):
    W1, b1, W2, b2, W3, b3 = unpack(p, I, H, O)
    h1 = np.tanh(x @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ W3.T + b3, h1, h2


def loss(p, x, t, I, H, O):
    y, _, _ = forward(p, x, I, H, O)
    return 0.5 * np.sum((y - t) ** 2) / x.shape[0]


def grad(p, x, t, I, H, O):
    W1, b1, W2, b2, W3, b3 = unpack(p, I, H, O)
    B = x.shape[0]
    y, h1, h2 = forward(p, x, I, H, O)
    e = (y - t) / B                    # dL/dy
    gW3 = e.T @ h2
    gb3 = e.sum(axis=0)
    d2 = (e @ W3) * (1.0 - h2 ** 2)    # dL/d(pre-activation of layer 2)
    gW2 = d2.T @ h1
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (1.0 - h1 ** 2)
    gW1 = d1.T @ x
    gb1 = d1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])


def adam(p, g, m, v, lr, b1, b2, eps, step):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
