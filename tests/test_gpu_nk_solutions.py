"""Newton-Krylov-hookstep (paper section 2) on non-trivial invariant
solutions, each certified by the oracle's own time stepper.

* A forced equilibrium: a steady body force on the (k, m) = (1, 1) axial
  velocity at Re = 150 drives a steady 3-D flow whose mean-flow distortion and
  m = 2 content come only from the nonlinear term.  The force breaks the
  axial translation symmetry, so the shift stays fixed at 0: with s free,
  sigma_s Phi_T(u) = u is n equations in n + 1 unknowns whose solutions form
  a one-parameter family (fixed points of 'evolve, then shift by s'), of
  which only s = 0 is invariant under the flow -- a free shift is meaningful
  only where sigma_s is a symmetry, as in the rotating pipe below.
* A travelling wave of rotating pipe flow (the frame rotation of section
  3.1's Coriolis example, about the pipe axis): at Omega = 1 U_cl/R,
  alpha = 1, m_p = 2 Hagen-Poiseuille flow loses stability near Re = 108 to
  a helical mode (m~ = 2, k = -1); at Re = 140 it saturates into a wave that
  rotates and travels, i.e. (being helical) translates along the axis at a
  constant speed: sigma_s Phi_T(u) = u with s = c T.  It is solved with T
  fixed and s free (the axial phase condition), with s fixed and T free (the
  time phase condition), and by multiple shooting with two sections.
"""
import functools

import numpy as np
import pytest
from scipy.optimize import minimize_scalar

from oracle.opf_oracle import Oracle, Params, mesh
from paper_1705_03838_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def opf():
    from paper_1705_03838_gb300 import build, opf as _opf

    build.build()
    _opf.lib()
    return _opf


def shift(U, s, alpha):
    K = (U.shape[2] + 1) // 2
    return U * np.exp(1j * alpha * np.arange(-(K - 1), K) * s)[None, None, :, None]


def best_shift(U1, U2, alpha):
    """s minimising |sigma_s U2 - U1| (grid search, then a bounded refinement)."""
    L = 2 * np.pi / alpha
    grid = np.linspace(0.0, L, 1441)
    r = [np.linalg.norm(shift(U2, s, alpha) - U1) for s in grid]
    s0 = grid[int(np.argmin(r))]
    res = minimize_scalar(lambda s: np.linalg.norm(shift(U2, s, alpha) - U1), bounds=(s0 - L / 700, s0 + L / 700),
                          method="bounded", options={"xatol": 1e-13})
    return res.x


def oracle_residual(o, u, T, s, nsteps, alpha):
    """|sigma_s Phi_T(u) - u| / |u| with the oracle's own time stepper."""
    v = o.step(u, nsteps)
    return np.linalg.norm(shift(v, s, alpha) - u) / np.linalg.norm(u)


# ------------------------------------------------------------- forced equilibrium
FORCED = dict(N=16, K=3, M=3, m_p=1, alpha=1.25, Re=150.0)


def forcing_field(amp=0.08):
    N, K, M = FORCED["N"], FORCED["K"], FORCED["M"]
    r = mesh(N)
    F = np.zeros((3, M, 2 * K - 1, N), complex)
    F[2, 1, K] = amp * (1 - r ** 2) * r  # f_z ~ (1 - r^2) r cos(alpha z + theta)
    return F


def test_newton_krylov_certifies_a_forced_equilibrium(opf):
    p = FORCED
    args = (p["N"], p["K"], p["M"], p["m_p"], p["alpha"], p["Re"])
    F = forcing_field()
    lam = inputs.laminar_state(p["N"], p["K"], p["M"])
    # near the equilibrium by time stepping, then a perturbed copy as the guess
    h = opf.opf_create(*args, 0.02)
    opf.opf_set_forcing(h, F)
    opf.opf_set_state(h, lam)
    opf.opf_step(h, 2000)
    ue = opf.opf_get_state(h)
    guess = ue + inputs.seeded_state(p["N"], p["K"], p["M"], p["m_p"], p["alpha"], 1e-2, 91, laminar=False)
    T, dt = 2.0, 0.02
    states, Tn, sn, res, it = opf.opf_nk_solve(*args, [guess], [T], [0.0], fix_T=1, fix_s=1, dt=dt, tol=1e-11,
                                               max_krylov=60, gmres_tol=1e-6, max_newton=20, forcing=F)
    u = states[0]
    assert res[0] < 1e-11, res
    assert it[0] >= 1
    dev = u - lam
    assert np.linalg.norm(dev) > 0.05  # a finite-amplitude response ...
    nonlinear = np.linalg.norm(dev[:, 0, p["K"] - 1]) + np.linalg.norm(dev[:, 2])
    assert nonlinear > 1e-2 * np.linalg.norm(dev)  # ... with nonlinearly driven modes
    o = Oracle(Params(*args, T / round(T / dt), forcing=F))
    assert oracle_residual(o, u, T, sn[0], round(T / dt), p["alpha"]) < 1e-10


# ------------------------------------------------------------- rotating-pipe travelling wave
ROT = dict(N=20, K=4, M=5, m_p=2, alpha=1.0, Re=140.0)
ROT_OMEGA = (0.0, 0.0, 1.0)
TW_T, TW_DT = 5.0, 0.01


@functools.lru_cache(maxsize=None)
def travelling_wave(opf_mod):
    """Time-step to the saturated wave, then converge it (T fixed, s free)."""
    p = ROT
    args = (p["N"], p["K"], p["M"], p["m_p"], p["alpha"], p["Re"])
    h = opf_mod.opf_create(*args, TW_DT)
    opf_mod.opf_set_option(h, "rot_z", ROT_OMEGA[2])
    opf_mod.opf_set_state(h, inputs.seeded_state(p["N"], p["K"], p["M"], p["m_p"], p["alpha"], 0.05, 140))
    opf_mod.opf_step(h, 30000)
    u1 = opf_mod.opf_get_state(h)
    opf_mod.opf_step(h, round(TW_T / TW_DT))
    u2 = opf_mod.opf_get_state(h)
    s0 = best_shift(u1, u2, p["alpha"])
    states, T, s, res, it = opf_mod.opf_nk_solve(*args, [u2], [TW_T], [s0], fix_T=1, fix_s=0, dt=TW_DT,
                                                 tol=1e-11, max_krylov=60, gmres_tol=1e-6, max_newton=20,
                                                 rot=ROT_OMEGA)
    return states[0], s[0], res[0], it[0], np.linalg.norm(shift(u2, s0, p["alpha"]) - u1) / np.linalg.norm(u1)


def rot_oracle():
    p = ROT
    return Oracle(Params(p["N"], p["K"], p["M"], p["m_p"], p["alpha"], p["Re"], TW_DT, rotation=ROT_OMEGA))


def test_travelling_wave_of_rotating_pipe_flow_T_fixed_s_free(opf):
    p = ROT
    u, s, res, it, start_res = travelling_wave(opf)
    assert res < 1e-11, (res, start_res)
    lam = inputs.laminar_state(p["N"], p["K"], p["M"])
    assert np.linalg.norm(u - lam) / np.linalg.norm(lam) > 0.05  # a finite-amplitude wave
    c = s / TW_T
    assert 0.05 < abs(c) < 1.5  # it travels (phase speed of order the flow speed)
    assert oracle_residual(rot_oracle(), u, TW_T, s, round(TW_T / TW_DT), p["alpha"]) < 1e-10


def test_travelling_wave_with_s_fixed_and_T_free(opf):
    """With the shift fixed 2 % above the wave's s* = c T*, the period must
    come out 2 % above T* (T = s / c) through the time phase condition; the
    state is the same wave up to an axial shift (and the time-step change)."""
    p = ROT
    args = (p["N"], p["K"], p["M"], p["m_p"], p["alpha"], p["Re"])
    u, s, _, _, _ = travelling_wave(opf)
    guess = u + inputs.seeded_state(p["N"], p["K"], p["M"], p["m_p"], p["alpha"], 1e-3, 141, laminar=False)
    s_fix = 1.02 * s
    states, T, sn, res, it = opf.opf_nk_solve(*args, [guess], [TW_T], [s_fix], fix_T=0, fix_s=1, dt=TW_DT,
                                              tol=1e-11, max_krylov=60, gmres_tol=1e-6, max_newton=20,
                                              rot=ROT_OMEGA)
    assert res[0] < 1e-11, res
    assert sn[0] == s_fix
    # the wave is now integrated at dt = T / 500 instead of 0.01: its shape and
    # speed move by the O(dt^2) time-discretisation error (~1e-5)
    assert abs(T[0] / (1.02 * TW_T) - 1.0) < 1e-4, T
    v = states[0]
    a = best_shift(u, v, p["alpha"])
    assert np.linalg.norm(shift(v, a, p["alpha"]) - u) / np.linalg.norm(u) < 1e-4
    nsteps = round(TW_T / TW_DT)  # the solver keeps its step count; dt = T / nsteps
    o = Oracle(Params(*args, T[0] / nsteps, rotation=ROT_OMEGA))
    assert oracle_residual(o, v, T[0], sn[0], nsteps, p["alpha"]) < 1e-10


def test_multiple_shooting_converges_to_the_same_travelling_wave(opf):
    """Two sections of T/2 (section 2's multiple-shooting option): from
    perturbed copies of the wave and of its state half a period later."""
    p = ROT
    args = (p["N"], p["K"], p["M"], p["m_p"], p["alpha"], p["Re"])
    u, s, _, _, _ = travelling_wave(opf)
    h = opf.opf_create(*args, TW_DT)
    opf.opf_set_option(h, "rot_z", ROT_OMEGA[2])
    opf.opf_set_state(h, u)
    opf.opf_step(h, round(TW_T / TW_DT / 2))
    half = opf.opf_get_state(h)
    pert = [inputs.seeded_state(p["N"], p["K"], p["M"], p["m_p"], p["alpha"], 1e-3, 150 + q, laminar=False)
            for q in range(2)]
    secs, T, sn, res, it = opf.opf_nk_solve_ms(*args, [[u + pert[0], half + pert[1]]], [TW_T], [s], fix_T=1,
                                               fix_s=0, dt=TW_DT, tol=1e-11, max_krylov=80, gmres_tol=1e-6,
                                               max_newton=20, rot=ROT_OMEGA)
    assert res[0] < 1e-11, res
    assert abs(sn[0] - s) < 1e-7
    u0 = secs[0][0]
    a = best_shift(u, u0, p["alpha"])
    assert np.linalg.norm(shift(u0, a, p["alpha"]) - u) / np.linalg.norm(u) < 1e-7
    o = rot_oracle()
    # each section is carried onto the next by the oracle's stepper
    n2 = round(TW_T / TW_DT / 2)
    v = o.step(secs[0][0], n2)
    assert np.linalg.norm(v - secs[0][1]) / np.linalg.norm(secs[0][1]) < 1e-10
    w = o.step(secs[0][1], n2)
    assert np.linalg.norm(shift(w, sn[0], p["alpha"]) - secs[0][0]) / np.linalg.norm(secs[0][0]) < 1e-10
