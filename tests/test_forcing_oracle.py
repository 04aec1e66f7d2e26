"""Pins of the oracle's forcing hook and Coriolis term: the Coriolis force does
no work (energy budget dE/dt = I - D unchanged), an axial rotation leaves an
axisymmetric swirl's velocity unchanged (its Coriolis force is radial and the
pressure takes it), and a uniform axial body force c at fixed flux changes
nothing but the driving: beta -> beta - c Re / 4."""
import numpy as np

from oracle.opf_oracle import Oracle, Params
from paper_1705_03838_gb300 import inputs


def coriolis_part(U, rot, N, K, M, m_p=1):
    o = Oracle(Params(N, K, M, m_p, 1.25, 500.0, 0.01, rotation=rot))
    o0 = Oracle(Params(N, K, M, m_p, 1.25, 500.0, 0.01))
    return o, o.nonlinear(U) - o0.nonlinear(U)


def test_coriolis_does_no_work():
    """<u, -2 Omega x u> = 0 pointwise, so its quadrature inner product with u
    vanishes to round-off; the term is linear in Omega."""
    N, K, M = 24, 4, 4
    U = inputs.seeded_state(N, K, M, 1, 1.25, 0.1, 13)
    rot = (0.3, -0.2, 0.5)
    o, C = coriolis_part(U, rot, N, K, M)
    wm = np.where(np.arange(M) == 0, 1.0, 2.0)
    work = np.sum(wm[None, :, None, None] * np.real(np.conj(U) * C) * o.w[None, None, None, :])
    scale = np.sum(wm[None, :, None, None] * np.abs(U) * np.abs(C) * o.w[None, None, None, :])
    assert abs(work) < 1e-13 * scale
    _, C2 = coriolis_part(U, tuple(2 * x for x in rot), N, K, M)
    np.testing.assert_allclose(C2, 2 * C, rtol=0, atol=1e-13)


def test_coriolis_of_the_laminar_profile_closed_form():
    """-2 Omega x (U(r) z) with U = 1 - r^2 is a transverse (m = 1, k = 0)
    force: in +- components N+ = 0, N- = -2 U (Omega_y + i Omega_x)."""
    N, K, M = 24, 3, 3
    U = inputs.laminar_state(N, K, M)
    ox, oy = 0.3, -0.2
    o, C = coriolis_part(U, (ox, oy, 0.0), N, K, M)
    Ub = 1 - o.r ** 2
    Np = C[0, 1, K - 1] + 1j * C[1, 1, K - 1]
    Nm = C[0, 1, K - 1] - 1j * C[1, 1, K - 1]
    np.testing.assert_allclose(Np, 0.0, atol=1e-14)
    np.testing.assert_allclose(Nm, -2 * Ub * (oy + 1j * ox), rtol=0, atol=1e-14)
    C[:, 1, K - 1] = 0.0
    assert np.abs(C).max() < 1e-14  # nothing in any other mode


def test_axial_rotation_leaves_swirl_unchanged():
    """The swirl's Coriolis force under axial rotation is radial: the pressure
    takes it, up to the finite-difference divergence error, which shrinks at
    high order under radial refinement."""
    diffs = []
    for N in (24, 48):
        K, M, Re, dt = 3, 3, 200.0, 0.01
        U = inputs.laminar_state(N, K, M)
        r = np.cos(np.pi * (N - np.arange(1, N + 1)) / (2 * N - 1))
        U[1, 0, K - 1] = 0.05 * r * (1 - r * r)
        a = Oracle(Params(N, K, M, 1, 1.25, Re, dt, rotation=(0.0, 0.0, 0.7))).step(U, 10)
        b = Oracle(Params(N, K, M, 1, 1.25, Re, dt)).step(U, 10)
        diffs.append(np.abs(a - b).max())
    assert diffs[0] < 1e-7 and diffs[1] < diffs[0] / 50, diffs


def test_uniform_axial_force_shifts_driving_only():
    N, K, M, Re, dt, c = 24, 3, 3, 800.0, 0.01, 0.003
    U = inputs.seeded_state(N, K, M, 1, 1.25, 0.05, 17)
    f = np.zeros_like(U)
    f[2, 0, K - 1] = c
    of = Oracle(Params(N, K, M, 1, 1.25, Re, dt, forcing=f))
    o0 = Oracle(Params(N, K, M, 1, 1.25, Re, dt))
    a, b = of.step(U, 5), o0.step(U, 5)
    assert np.abs(a - b).max() < 1e-11
    assert abs((of.beta - o0.beta) + c * Re / 4) < 1e-9
