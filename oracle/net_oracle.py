"""Plain FP64 CPU oracle of the proposal network (test infrastructure only:
imported by tests/ and bench.py's baseline leg).

    h1 = gelu(conv3(x; W1, b1)), h2 = gelu(conv3(h1; W2, b2)),
    y = conv3(h2; W3, b3), z = Wh mean_l(h2) + bh,
    loss = mean((y - ty)^2) + lambda mean((z - tz)^2)

conv3 is a width-3 convolution along l with zero padding: output channel o
at l sums W[o][j*C + c] x[l + j - 1][c] over j = 0, 1, 2 and channels c.
gelu(x) = x Phi(x) with Phi the standard normal CDF.  Backward pass written
out by the chain rule; pinned against central finite differences."""
import numpy as np
from scipy.special import erf

NAMES = ("W1", "b1", "W2", "b2", "W3", "b3", "Wh", "bh")


def split(flat, cin, hidden, nout):
    sizes = [hidden * 3 * cin, hidden, hidden * 3 * hidden, hidden, cin * 3 * hidden, cin, nout * hidden, nout]
    shapes = [(hidden, 3 * cin), (hidden,), (hidden, 3 * hidden), (hidden,), (cin, 3 * hidden), (cin,),
              (nout, hidden), (nout,)]
    out, o = {}, 0
    for nm, sz, sh in zip(NAMES, sizes, shapes):
        out[nm] = np.asarray(flat[o:o + sz], dtype=np.float64).reshape(sh)
        o += sz
    return out


def flatten(d):
    return np.concatenate([d[nm].ravel() for nm in NAMES])


def im2col(x):
    B, L, C = x.shape
    xp = np.zeros((B, L + 2, C))
    xp[:, 1:-1] = x
    return np.concatenate([xp[:, j:j + L, :] for j in range(3)], axis=2)  # [B][L][3C]


def col2im(dcols, C):
    """adjoint of im2col"""
    B, L, _ = dcols.shape
    dxp = np.zeros((B, L + 2, C))
    for j in range(3):
        dxp[:, j:j + L, :] += dcols[:, :, j * C:(j + 1) * C]
    return dxp[:, 1:-1]


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2 * np.pi)


def forward(p, x):
    c1 = im2col(x)
    a1 = c1 @ p["W1"].T + p["b1"]
    h1 = gelu(a1)
    c2 = im2col(h1)
    a2 = c2 @ p["W2"].T + p["b2"]
    h2 = gelu(a2)
    c3 = im2col(h2)
    y = c3 @ p["W3"].T + p["b3"]
    pooled = h2.mean(axis=1)
    z = pooled @ p["Wh"].T + p["bh"]
    return y, z, dict(c1=c1, a1=a1, c2=c2, a2=a2, c3=c3, pooled=pooled, h2=h2)


def loss_and_grads(p, x, ty, tz, lam):
    y, z, s = forward(p, x)
    B, L, C = x.shape
    ry, rz = y - ty, z - tz
    loss = (ry ** 2).mean() + lam * (rz ** 2).mean()
    dy = 2.0 * ry / ry.size
    dz = 2.0 * lam * rz / rz.size
    g = {}
    g["W3"] = np.einsum("blo,blk->ok", dy, s["c3"])
    g["b3"] = dy.sum(axis=(0, 1))
    dh2 = col2im(dy @ p["W3"], p["W2"].shape[0])
    g["Wh"] = dz.T @ s["pooled"]
    g["bh"] = dz.sum(axis=0)
    dh2 += (dz @ p["Wh"])[:, None, :] / L
    da2 = dh2 * gelu_grad(s["a2"])
    g["W2"] = np.einsum("blo,blk->ok", da2, s["c2"])
    g["b2"] = da2.sum(axis=(0, 1))
    dh1 = col2im(da2 @ p["W2"], p["W1"].shape[0])
    da1 = dh1 * gelu_grad(s["a1"])
    g["W1"] = np.einsum("blo,blk->ok", da1, s["c1"])
    g["b1"] = da1.sum(axis=(0, 1))
    return loss, g, y, z
