"""Pins of the FP64 proposal-network oracle: the backward pass equals central
finite differences of the loss, and conv3 equals a brute-force sum."""
import numpy as np

from oracle import net_oracle as nn


def make(cin=5, hidden=7, nout=2, L=6, B=3, seed=0):
    rng = np.random.default_rng(seed)
    p = {"W1": rng.normal(size=(hidden, 3 * cin)) * 0.4, "b1": rng.normal(size=hidden) * 0.1,
         "W2": rng.normal(size=(hidden, 3 * hidden)) * 0.3, "b2": rng.normal(size=hidden) * 0.1,
         "W3": rng.normal(size=(cin, 3 * hidden)) * 0.3, "b3": rng.normal(size=cin) * 0.1,
         "Wh": rng.normal(size=(nout, hidden)) * 0.3, "bh": rng.normal(size=nout) * 0.1}
    x = rng.normal(size=(B, L, cin))
    ty = rng.normal(size=(B, L, cin))
    tz = rng.normal(size=(B, nout))
    return p, x, ty, tz


def test_conv3_brute_force():
    p, x, _, _ = make()
    B, L, C = x.shape
    W, b = p["W1"], p["b1"]
    out = nn.im2col(x) @ W.T + b
    for bb in range(B):
        for l in range(L):
            for o in range(W.shape[0]):
                s = b[o]
                for j in range(3):
                    if 0 <= l + j - 1 < L:
                        s += sum(W[o, j * C + c] * x[bb, l + j - 1, c] for c in range(C))
                assert abs(out[bb, l, o] - s) < 1e-12


def test_gradients_match_finite_differences():
    p, x, ty, tz = make()
    lam = 0.7
    _, g, _, _ = nn.loss_and_grads(p, x, ty, tz, lam)
    flat = nn.flatten(p)
    gflat = nn.flatten(g)
    rng = np.random.default_rng(1)
    for i in rng.choice(flat.size, 40, replace=False):
        h = 1e-6
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        lp = nn.loss_and_grads(nn.split(fp, 5, 7, 2), x, ty, tz, lam)[0]
        lm = nn.loss_and_grads(nn.split(fm, 5, 7, 2), x, ty, tz, lam)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gflat[i]) <= 1e-7 * max(1.0, abs(fd))
