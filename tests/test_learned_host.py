"""Host logic of the learned-proposal pipeline: feature packing, the axial
shift on features, and the recurrence scan against brute force and against a
synthetic relative-periodic signal whose period and shift are known."""
import math

import numpy as np

from paper_1705_03838_gb300 import inputs
from paper_1705_03838_gb300 import learned as lp

N, K, M, m_p, alpha = 10, 9, 9, 2, 1.25


def state(seed, amp=0.05):
    return inputs.seeded_state(N, K, M, m_p, alpha, amp, seed, envelope=inputs.envelope_exp)


def test_feature_round_trip_keeps_only_low_modes():
    U = state(3)
    f = lp.features(U, K, M, N)
    assert f.shape == (N, lp.NCH) and f.dtype == np.float32
    lam = inputs.laminar_state(N, K, M)
    V = lp.apply_features(lam, f, K, M, N)
    np.testing.assert_allclose(lp.features(V, K, M, N), f, rtol=0, atol=1e-7)
    P = lp.perturbation(U, K, N)
    Q = lp.perturbation(V, K, N)
    ks = np.abs(np.arange(2 * K - 1) - (K - 1)) < lp.KF
    mask = np.zeros((M, 2 * K - 1), dtype=bool)
    mask[:lp.MF] = ks[None, :]
    assert np.abs(Q[:, ~mask]).max() == 0.0
    np.testing.assert_allclose(Q[:, mask], P[:, mask], rtol=0, atol=2e-8 * np.abs(P).max())


def test_feature_channel_order():
    """channel ((c*15 + k)*8 + m)*2 + (re, im) at radial point n"""
    U = inputs.laminar_state(N, K, M)
    c, k, m, n = 1, -3, 5, 4
    U[c, m, k + K - 1, n] += 0.25 - 0.5j
    f = lp.features(U, K, M, N)
    ch = ((c * lp.NKF + (k + lp.KF - 1)) * lp.MF + m) * 2
    assert f[n, ch] == np.float32(0.25) and f[n, ch + 1] == np.float32(-0.5)
    assert np.count_nonzero(f) == 2


def test_shift_on_features_equals_shift_on_state():
    U = state(5)
    s = 1.7
    a = lp.features(lp.shifted(U, s, alpha, K), K, M, N)
    b = lp.shift_features(lp.features(U, K, M, N).astype(np.float64), s, alpha)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-6 * np.abs(a).max())


def _random_feats(S, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(S, 4, lp.NCH)).astype(np.float32)


def test_recurrence_matrix_equals_brute_force():
    f = _random_feats(9, 1)
    nshift = 16
    D, Sh = lp.recurrence_matrix(f, alpha, 2, 5, nshift)
    L = 2 * np.pi / alpha
    for i in range(9):
        for t, tau in enumerate(range(2, 6)):
            if i + tau >= 9:
                assert np.isinf(D[i, t])
                continue
            best, arg = np.inf, None
            for q in range(nshift):
                s = q * L / nshift
                fi = f[i].astype(np.float64)
                d = np.linalg.norm(lp.shift_features(f[i + tau], s, alpha) - fi) / np.linalg.norm(fi)
                if d < best:
                    best, arg = d, s
            assert abs(D[i, t] - best) < 1e-9 * max(1.0, best)
            assert abs(Sh[i, t] - arg) < 1e-12


def test_scan_finds_known_period_and_shift():
    """f(t) = sigma_{c t} h(t) with h of period P: the scan must return T = P
    and the shift s = -c P (mod L) that closes it, with D ~ 0."""
    rng = np.random.default_rng(7)
    L = 2 * np.pi / alpha
    P, dt_s, nshift = 24, 0.5, 128
    c = (-5 * L / nshift) / (P * dt_s)  # closing shift = 5 grid points
    base = rng.normal(size=(3, 4, lp.NCH))
    S = 80
    f = np.empty((S, 4, lp.NCH), dtype=np.float32)
    for i in range(S):
        ph = 2 * math.pi * i / P
        h = base[0] + math.cos(ph) * base[1] + math.sin(2 * ph) * base[2]
        f[i] = lp.shift_features(h, c * i * dt_s, alpha)
    recs = lp.best_recurrences(f, alpha, dt_s, 6.0, 20.0, thresh=0.3, nshift=nshift)
    recs = [r for r in recs if r[0] < S - P]  # later starts cannot see a full period
    assert len(recs) == S - P
    for (i, tau, T, s, d) in recs:
        assert tau == P and abs(T - P * dt_s) < 1e-12
        assert abs(s - 5 * L / nshift) < 1e-9
        assert d < 1e-5
    x, ty, tz = lp.labels(f, recs, alpha, T_scale=20.0)
    assert np.abs(ty).max() < 1e-5 * np.abs(x).max()  # exact recurrences need no correction
    T, s = lp.decode_z(tz, alpha, 20.0)
    np.testing.assert_allclose(T, P * dt_s, rtol=1e-6)
    np.testing.assert_allclose(s, 5 * L / nshift, atol=1e-5)


def test_local_minima():
    recs = [(0, 5, 2.5, 0.0, 0.2), (1, 5, 2.5, 0.0, 0.1), (2, 5, 2.5, 0.0, 0.15), (4, 5, 2.5, 0.0, 0.25)]
    assert [r[0] for r in lp.local_minima(recs)] == [1, 4]


def test_interior_dips_only():
    """A slowly drifting signal (D grows with tau) has no interior dip."""
    rng = np.random.default_rng(3)
    base = rng.normal(size=(2, 4, lp.NCH))
    f = np.stack([base[0] + 0.002 * i * base[1] for i in range(40)]).astype(np.float32)
    assert len(lp.best_recurrences(f, alpha, 0.5, 2.0, 8.0, thresh=0.3, interior=False)) > 0
    assert lp.best_recurrences(f, alpha, 0.5, 2.0, 8.0, thresh=0.3, interior=True) == []


def test_constant_predictor_loss():
    ty = np.full((2, 3, 4), 2.0)
    tz = np.array([[1.0, 0.0], [3.0, 0.0]])
    assert lp.constant_predictor_loss(ty, tz, 0.5, tz.mean(0), scale=2.0) == 1.0 + 0.5 * 0.5


def test_rotation_of_features_equals_rotation_of_state():
    """Axial shift + azimuthal rotation on features equals the same symmetry
    applied to the full state (mode (k, m) times e^{i(alpha k a + m_p m phi)})."""
    U = state(9)
    a, phi = 0.9, 0.4
    k = np.arange(-(K - 1), K)
    m = np.arange(M)
    V = U * np.exp(1j * (alpha * k[None, :] * a + m_p * m[:, None] * phi))[None, :, :, None]
    f = lp.features(U, K, M, N)[None]
    g = lp.rotate_features(f, np.array([a]), np.array([phi]), alpha, m_p)[0]
    np.testing.assert_allclose(g, lp.features(V, K, M, N), rtol=0, atol=1e-6 * np.abs(g).max())
