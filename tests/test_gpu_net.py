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


def test_device_minibatch_augmentation_matches_the_host_rotation(env):
    """opf_net_gather_augment (the training minibatch, gathered and turned by
    the flow's symmetries on the device) against learned.rotate_features
    (the host form): an axial shift a and azimuthal rotation phi per sample
    multiply mode (k, m) by e^{i(alpha k a + m_p m phi)}; the head targets are
    gathered unchanged."""
    torch, opf = env
    from paper_1705_03838_gb300 import learned as lp

    rng = np.random.default_rng(3)
    rows, L, nz, B, alpha, m_p = 40, 12, 3, 16, 1.25, 2
    x = rng.standard_normal((rows, L, lp.NCH)).astype(np.float32)
    y = rng.standard_normal((rows, L, lp.NCH)).astype(np.float32)
    z = rng.standard_normal((rows, nz)).astype(np.float32)
    idx = rng.integers(0, rows, B)
    a = rng.uniform(0, 2 * np.pi / alpha, B)
    phi = rng.uniform(0, 2 * np.pi / m_p, B)
    net = opf.opf_net_create(lp.NCH, 16, L, nz, seed=1)
    dx, dy, dz = (torch.from_numpy(v).cuda() for v in (x, y, z))
    bx = torch.empty((B, L, lp.NCH), device="cuda")
    by = torch.empty_like(bx)
    bz = torch.empty((B, nz), device="cuda")
    torch.cuda.synchronize()
    ang = np.stack([alpha * a, m_p * phi], axis=1)
    opf.opf_net_gather_augment(net, dx.data_ptr(), dy.data_ptr(), dz.data_ptr(), rows, idx, ang, L, 3, lp.NKF,
                               lp.MF, nz, bx.data_ptr(), by.data_ptr(), bz.data_ptr())
    torch.cuda.synchronize()
    want_x = lp.rotate_features(x[idx], a, phi, alpha, m_p)
    want_y = lp.rotate_features(y[idx], a, phi, alpha, m_p)
    assert np.abs(bx.cpu().numpy() - want_x).max() < 2e-5 * np.abs(want_x).max()
    assert np.abs(by.cpu().numpy() - want_y).max() < 2e-5 * np.abs(want_y).max()
    assert np.array_equal(bz.cpu().numpy(), z[idx])
    with pytest.raises(opf.OpfError):
        opf.opf_net_gather_augment(net, dx.data_ptr(), dy.data_ptr(), dz.data_ptr(), rows, [rows], [[0.0, 0.0]],
                                   L, 3, lp.NKF, lp.MF, nz, bx.data_ptr(), by.data_ptr(), bz.data_ptr())
