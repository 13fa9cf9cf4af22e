"""Plain FP64 MLP forward pass and backpropagation (numpy).  Oracle only.

The network of the cost model: x (12 features) -> tanh(x W1 + b1) ->
tanh(a1 W2 + b2) -> a2 . w3 + b3, loss = mean over the batch of (out - y)^2.
Parameters in one array: W1[12][64], b1[64], W2[64][64], b2[64], w3[64], b3.
Backpropagation is the chain rule written out layer by layer (Rumelhart,
Hinton, Williams 1986); d tanh(z)/dz = 1 - tanh(z)^2.
"""
import numpy as np

F, H = 12, 64
P = F * H + H + H * H + H + H + 1


def unpack(w):
    w = np.asarray(w, dtype=np.float64)
    o = 0
    W1 = w[o:o + F * H].reshape(F, H); o += F * H
    b1 = w[o:o + H]; o += H
    W2 = w[o:o + H * H].reshape(H, H); o += H * H
    b2 = w[o:o + H]; o += H
    w3 = w[o:o + H]; o += H
    b3 = w[o]
    return W1, b1, W2, b2, w3, b3


def forward(w, X):
    W1, b1, W2, b2, w3, b3 = unpack(w)
    a1 = np.tanh(X @ W1 + b1)
    a2 = np.tanh(a1 @ W2 + b2)
    return a2 @ w3 + b3, (a1, a2)


def loss(w, X, Y):
    out, _ = forward(w, X)
    return float(np.mean((out - Y) ** 2))


def gradient(w, X, Y):
    W1, b1, W2, b2, w3, b3 = unpack(w)
    out, (a1, a2) = forward(w, X)
    B = X.shape[0]
    dy = 2.0 * (out - Y) / B
    gw3 = a2.T @ dy
    gb3 = dy.sum()
    d2 = np.outer(dy, w3) * (1.0 - a2 ** 2)
    gW2 = a1.T @ d2
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2.T) * (1.0 - a1 ** 2)
    gW1 = X.T @ d1
    gb1 = d1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])
