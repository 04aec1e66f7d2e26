"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

FP64 tolerance: the target is relative L2 <= 1e-10 on all spectral
coefficients after 100 steps of the small workload; single evaluations are
held to ~1e-12 (differences are round-off only: banded pivot-free LU with
influence matrices vs dense pivoted LU of the coupled system, FFT ordering).
"""
import functools
import re

import numpy as np
import pytest

from oracle.opf_oracle import Oracle, Params
from paper_1705_03838_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def opf():
    from paper_1705_03838_gb300 import build, opf as _opf

    build.build()
    _opf.lib()
    return _opf


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@functools.lru_cache(maxsize=None)
def oracle_run(N, K, M, m_p, alpha, Re, dt, amp, seed, nsteps):
    o = Oracle(Params(N, K, M, m_p, alpha, Re, dt))
    U0 = inputs.seeded_state(N, K, M, m_p, alpha, amp, seed)
    U = o.step(U0, nsteps)
    return U0, U, o.energy(U), o.beta


def gpu_run(opf, N, K, M, m_p, alpha, Re, dt, U0, nsteps, **opts):
    h = opf.opf_create(N, K, M, m_p, alpha, Re, dt)
    for k, v in opts.items():
        opf.opf_set_option(h, k, v)
    opf.opf_set_state(h, U0)
    opf.opf_step(h, nsteps)
    return h, opf.opf_get_state(h)


# ---------------------------------------------------------------- stages
# the last five hit the compiled FFT plans: 3K or 3M in 48, 72, 96, 192, 384
@pytest.mark.parametrize("N,K,M,m_p", [(16, 4, 6, 1), (12, 3, 4, 2), (9, 1, 1, 1), (20, 5, 3, 3),
                                       (32, 16, 16, 1), (10, 24, 32, 1), (10, 64, 2, 1), (10, 2, 64, 2),
                                       (9, 128, 2, 1), (9, 2, 128, 1)])
def test_nonlinear_term_matches_oracle(opf, N, K, M, m_p):
    alpha, Re = 1.25, 1000.0
    U0 = inputs.seeded_state(N, K, M, m_p, alpha, 0.1, 77)
    h = opf.opf_create(N, K, M, m_p, alpha, Re, 0.01)
    got = opf.opf_nonlinear(h, U0)
    want = Oracle(Params(N, K, M, m_p, alpha, Re, 0.01)).nonlinear(U0)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("N,K,M,m_p", [(10, 24, 32, 1), (10, 64, 2, 1), (9, 2, 128, 1)])
def test_mixed_nonlinear_term_on_compiled_plans(opf, N, K, M, m_p):
    """FP32 transforms with compiled plans (72, 96, 192, 384 points) against
    the FP64 oracle: FP32 round-off only."""
    alpha, Re = 1.25, 1000.0
    U0 = inputs.seeded_state(N, K, M, m_p, alpha, 0.1, 78)
    h = opf.opf_create(N, K, M, m_p, alpha, Re, 0.01)
    opf.opf_set_option(h, "precision", 1)
    got = opf.opf_nonlinear(h, U0)
    want = Oracle(Params(N, K, M, m_p, alpha, Re, 0.01)).nonlinear(U0)
    assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()


def test_fp64_steps_with_interleaved_calls_equal_plain_steps(opf):
    """FP64 steps take the curl of each solved state inside the solve; every
    call that writes the state or the work buffers in between (energy, the
    nonlinear term of another state, an option, set_state) must leave the
    next step starting from the curl of the current state.  A stale curl
    would change the result at the size of the perturbation; the only
    difference allowed is the round-off of the set_state(get_state) round
    trip (u+- <-> u_r, u_theta)."""
    N, K, M, m_p, alpha, Re, dt = 16, 4, 4, 1, 1.25, 800.0, 0.01
    U0 = inputs.seeded_state(N, K, M, m_p, alpha, 0.05, 321)
    other = inputs.seeded_state(N, K, M, m_p, alpha, 0.05, 322)
    h, plain = gpu_run(opf, N, K, M, m_p, alpha, Re, dt, U0, 6)
    h2 = opf.opf_create(N, K, M, m_p, alpha, Re, dt)
    opf.opf_set_state(h2, U0)
    opf.opf_step(h2, 2)
    opf.opf_energy(h2)
    opf.opf_step(h2, 1)
    opf.opf_nonlinear(h2, other)
    opf.opf_step(h2, 1)
    opf.opf_set_option(h2, "n_corr", 1)
    opf.opf_step(h2, 1)
    opf.opf_set_state(h2, opf.opf_get_state(h2))
    opf.opf_step(h2, 1)
    assert rel(opf.opf_get_state(h2), plain) < 1e-13
    # a mixed-precision step, then FP64 steps: as if started from that state
    h3 = opf.opf_create(N, K, M, m_p, alpha, Re, dt)
    opf.opf_set_state(h3, U0)
    opf.opf_set_option(h3, "precision", 1)
    opf.opf_step(h3, 1)
    mid = opf.opf_get_state(h3)
    opf.opf_set_option(h3, "precision", 0)
    opf.opf_step(h3, 2)
    _, ref = gpu_run(opf, N, K, M, m_p, alpha, Re, dt, mid, 2)
    # set_state also projects the m = 0 modes of the mixed-precision state
    # onto Hermitian symmetry (FP32 round-off breaks it slightly): ~1e-12
    assert rel(opf.opf_get_state(h3), ref) < 1e-10


def test_state_round_trip_and_hermitian_projection(opf):
    N, K, M = 16, 4, 4
    h = opf.opf_create(N, K, M, 1, 1.25, 100.0, 0.01)
    U0 = inputs.seeded_state(N, K, M, 1, 1.25, 0.1, 3)
    opf.opf_set_state(h, U0)
    assert opf.lib().opf_last_error() == b""  # the seeded m = 0 part is Hermitian
    # u+- = u_r +- i u_theta and back: exact up to one rounding
    assert np.abs(opf.opf_get_state(h) - U0).max() <= 4e-16 * np.abs(U0).max()
    V = U0.copy()
    V[:, 0, K] += 1e-3 * (1 + 1j)  # break symmetry
    opf.opf_set_state(h, V)
    note = opf.lib().opf_last_error().decode()
    assert "not Hermitian" in note
    # the reported asymmetry: max |A(k,0) - conj A(-k,0)| over parts, relative
    # to the largest m = 0 part, to the 2^-20 of its reduction
    d = V[:, 0] - np.conj(V[:, 0, ::-1])
    want = max(np.abs(d.real).max(), np.abs(d.imag).max()) / max(
        np.abs(V[:, 0].real).max(), np.abs(V[:, 0].imag).max())
    got = float(re.search(r"\| = ([0-9.eE+-]+) of the largest", note).group(1))
    assert abs(got - want) <= 1e-2 * want
    W = opf.opf_get_state(h)
    assert np.abs(W[:, 0] - Oracle.hermitian_project(V)[:, 0]).max() <= 4e-16 * np.abs(V).max()
    opf.opf_set_state(h, W)  # the projected state is Hermitian: no note
    assert opf.lib().opf_last_error() == b""


def test_nan_state_is_rejected_and_previous_kept(opf):
    N, K, M = 12, 3, 3
    h = opf.opf_create(N, K, M, 1, 1.25, 100.0, 0.01)
    U0 = inputs.seeded_state(N, K, M, 1, 1.25, 0.1, 4)
    opf.opf_set_state(h, U0)
    bad = U0.copy()
    bad[1, 2, 1, 3] = np.nan
    with pytest.raises(opf.OpfError) as e:
        opf.opf_set_state(h, bad)
    assert e.value.code == opf.OPF_ENAN
    assert np.abs(opf.opf_get_state(h) - U0).max() <= 4e-16 * np.abs(U0).max()


def test_invalid_arguments(opf):
    with pytest.raises(opf.OpfError):
        opf.opf_create(8, 4, 4, 1, 1.25, 100.0, 0.01)
    with pytest.raises(opf.OpfError):
        opf.opf_create(16, 7, 4, 1, 1.25, 100.0, 0.01)  # 3K = 21 has factor 7
    h = opf.opf_create(16, 4, 4, 1, 1.25, 100.0, 0.01)
    with pytest.raises(opf.OpfError):
        opf.opf_step(h, -1)
    with pytest.raises(opf.OpfError):
        opf.opf_set_option(h, "no_such_option", 1)


# ---------------------------------------------------------------- whole steps
@pytest.mark.parametrize("N,K,M,m_p,graph", [(16, 4, 4, 1, 1), (16, 4, 4, 1, 0), (12, 3, 5, 2, 1),
                                             (9, 1, 1, 1, 1), (10, 2, 1, 1, 1), (9, 1, 3, 3, 1),
                                             (40, 5, 6, 1, 1)])
def test_steps_match_oracle(opf, N, K, M, m_p, graph):
    alpha, Re, dt = 1.25, 800.0, 0.01
    U0, ref, e_ref, beta_ref = oracle_run(N, K, M, m_p, alpha, Re, dt, 0.05, 123, 3)
    h, U = gpu_run(opf, N, K, M, m_p, alpha, Re, dt, U0, 3, graph=graph)
    assert rel(U, ref) < 1e-12
    e = opf.opf_energy(h)
    # E and D are plain quadratures; I carries beta = beta' Re / 4, which
    # scales beta's round-off by Re / 4
    assert abs(e[0] - e_ref[0]) < 1e-12 and abs(e[2] - e_ref[2]) < 1e-12
    assert abs(e[1] - e_ref[1]) < 1e-14 * Re
    assert abs(opf.opf_get_beta(h) - beta_ref) < 1e-14 * Re
    g = opf.opf_wall_residual(h)
    assert g[0] < 1e-14 and g[1] < 1e-10


def test_small_workload_100_steps(opf):
    """The plain-method small workload: N=32, |k|<16, m<16, Re=2000,
    alpha=1.25, dt=0.01, amplitude 1e-2, 100 steps; rel L2 <= 1e-10."""
    w = inputs.WORKLOADS["small"]
    args = (w["N"], w["K"], w["M"], w["m_p"], w["alpha"], w["Re"], w["dt"])
    o = Oracle(Params(*args))
    U0 = inputs.workload_state("small")
    ref = o.step(U0, 100)
    h, U = gpu_run(opf, *args, U0, 100)
    assert rel(U, ref) < 1e-10
    e, e_ref = opf.opf_energy(h), o.energy(ref)
    assert abs(e[0] - e_ref[0]) < 1e-12 and abs(e[2] - e_ref[2]) < 1e-12
    assert abs(e[1] - e_ref[1]) < 1e-13 * w["Re"]


def test_medium_workload_100_steps(opf):
    """Full medium size (N=48, |k|<32, m<24, m_p=2, Re=2400, amplitude 0.1):
    all coefficients after 100 FP64 steps against the oracle, the same
    bound as the small workload (relative L2 <= 1e-10)."""
    w = inputs.WORKLOADS["medium"]
    args = (w["N"], w["K"], w["M"], w["m_p"], w["alpha"], w["Re"], w["dt"])
    o = Oracle(Params(*args))
    U0 = inputs.workload_state("medium")
    ref = o.step(U0, 100)
    h, U = gpu_run(opf, *args, U0, 100)
    assert rel(U, ref) < 1e-10
    e, e_ref = opf.opf_energy(h), o.energy(ref)
    assert abs(e[0] - e_ref[0]) < 1e-12 and abs(e[2] - e_ref[2]) < 1e-12


def test_hagen_poiseuille_steady_on_gpu(opf):
    N, K, M = 24, 4, 4
    U0 = inputs.laminar_state(N, K, M)
    h, U = gpu_run(opf, N, K, M, 1, 1.25, 2000.0, 0.01, U0, 200)
    # steady to round-off: 200 steps of accumulated FP64 rounding stay ~1e-13
    assert np.abs(U - U0).max() < 1e-12
    assert np.allclose(opf.opf_energy(h), 1.0, atol=1e-13)


def test_time_and_options(opf):
    h = opf.opf_create(12, 2, 2, 1, 1.0, 100.0, 0.02)
    opf.opf_set_state(h, inputs.laminar_state(12, 2, 2))
    opf.opf_step(h, 5)
    assert abs(opf.opf_get_time(h) - 0.1) < 1e-15
    assert opf.opf_get_dt(h) == 0.02
    opf.opf_set_option(h, "n_corr", 2)
    assert opf.opf_get_option(h, "n_corr") == 2


def test_two_correctors_match_oracle(opf):
    N, K, M, alpha, Re, dt = 12, 3, 3, 1.25, 300.0, 0.01
    U0 = inputs.seeded_state(N, K, M, 1, alpha, 0.1, 8)
    o = Oracle(Params(N, K, M, 1, alpha, Re, dt, n_corr=2))
    ref = o.step(U0, 2)
    h, U = gpu_run(opf, N, K, M, 1, alpha, Re, dt, U0, 2, n_corr=2)
    assert rel(U, ref) < 1e-12


@pytest.mark.parametrize("precision", [0, 1])
def test_predictor_only_steps_match_oracle(opf, precision):
    """n_corr = 0: each step is the predictor alone (one nonlinear term, one
    solve), in FP64 and with the mixed-precision step (FP32 round-off)."""
    N, K, M, alpha, Re, dt = 16, 3, 4, 1.25, 600.0, 0.01
    U0 = inputs.seeded_state(N, K, M, 1, alpha, 0.1, 18)
    ref = Oracle(Params(N, K, M, 1, alpha, Re, dt, n_corr=0)).step(U0, 3)
    h, U = gpu_run(opf, N, K, M, 1, alpha, Re, dt, U0, 3, n_corr=0, precision=precision)
    assert rel(U, ref) < (1e-12 if precision == 0 else 1e-7)
    assert opf.opf_get_option(h, "n_corr") == 0


def test_handles_of_different_sizes_coexist(opf):
    """A large handle keeps working after a smaller one is created (kernel
    shared-memory limits are process-wide)."""
    w = inputs.WORKLOADS["medium"]
    args = (w["N"], w["K"], w["M"], w["m_p"], w["alpha"], w["Re"], w["dt"])
    big = opf.opf_create(*args)
    opf.opf_set_state(big, inputs.workload_state("medium"))
    small = opf.opf_create(12, 2, 2, 1, 1.0, 100.0, 0.01)
    opf.opf_set_state(small, inputs.laminar_state(12, 2, 2))
    opf.opf_step(small, 1)
    opf.opf_step(big, 2)
    assert np.isfinite(opf.opf_energy(big)).all()
