"""Proposal network on the GPU (BF16 tensor-core GEMMs, FP32 accumulation)
against the FP64 oracle network on identical parameters and inputs.

Tolerance: BF16 keeps 8 significand bits, so rounding of inputs, weights
and activations gives ~4e-3 relative error per factor; over the three
layers the relative L2 error of outputs and gradients is held to 3e-2."""
import numpy as np
import pytest

from oracle import net_oracle as nn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    from paper_1705_03838_gb300 import build, opf

    build.build()
    opf.lib()
    return torch, opf


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


@pytest.mark.parametrize("cin,hidden,L,B", [(40, 48, 32, 8), (70, 100, 17, 5), (720, 384, 32, 16)])
def test_forward_and_gradients_match_oracle(env, cin, hidden, L, B):
    torch, opf = env
    net = opf.opf_net_create(cin, hidden, L, 2, seed=7)
    flat = opf.opf_net_get_params(net)
    p = nn.split(flat.astype(np.float64), cin, hidden, 2)
    # non-zero biases so their gradients and the bias path are exercised
    rng = np.random.default_rng(3)
    for k in ("b1", "b2", "b3", "bh"):
        p[k] = rng.normal(size=p[k].shape) * 0.1
    flat = nn.flatten(p).astype(np.float32)
    opf.opf_net_set_params(net, flat)
    p = nn.split(flat.astype(np.float64), cin, hidden, 2)
    x = rng.normal(size=(B, L, cin)).astype(np.float32)
    ty = rng.normal(size=(B, L, cin)).astype(np.float32) * 0.5
    tz = rng.normal(size=(B, 2)).astype(np.float32)
    dx, dty, dtz = (torch.from_numpy(a).cuda() for a in (x, ty, tz))
    dy = torch.empty_like(dx)
    dz = torch.empty((B, 2), dtype=torch.float32, device="cuda")
    opf.opf_net_forward(net, dx.data_ptr(), B, dy.data_ptr(), dz.data_ptr())
    lam = 0.5
    loss_ref, g_ref, y_ref, z_ref = nn.loss_and_grads(p, x.astype(np.float64), ty, tz, lam)
    assert rel(dy.cpu().numpy(), y_ref) < 3e-2
    assert rel(dz.cpu().numpy(), z_ref) < 3e-2
    loss = opf.opf_net_gradients(net, dx.data_ptr(), dty.data_ptr(), dtz.data_ptr(), B, lam)
    assert abs(loss - loss_ref) / loss_ref < 3e-2
    g = nn.split(opf.opf_net_get_params(net, grads=True).astype(np.float64), cin, hidden, 2)
    for k in nn.NAMES:
        assert rel(g[k], g_ref[k]) < 3e-2, k


def test_training_reduces_loss(env):
    torch, opf = env
    cin, hidden, L, B = 64, 96, 32, 32
    net = opf.opf_net_create(cin, hidden, L, 2, seed=11)
    rng = np.random.default_rng(5)
    x = rng.normal(size=(B, L, cin)).astype(np.float32)
    ty = (0.3 * np.tanh(x) + 0.1 * np.roll(x, 1, axis=1)).astype(np.float32)
    tz = np.stack([x.mean(axis=(1, 2)), x.std(axis=(1, 2))], axis=1).astype(np.float32)
    dx, dty, dtz = (torch.from_numpy(a).cuda() for a in (x, ty, tz))
    losses = [opf.opf_net_train_step(net, dx.data_ptr(), dty.data_ptr(), dtz.data_ptr(), B, 1.0, 1e-3)
              for _ in range(60)]
    assert losses[-1] < 0.2 * losses[0]
