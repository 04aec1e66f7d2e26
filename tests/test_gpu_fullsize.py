"""GPU parity against the oracle on the launch shapes of the full workloads.

The solve kernel changes shape with N and with the number of modes per
launch: tiles of 4, 8 or 16 modes per block, u_j and the influence responses
staged in shared memory or not, u_j near the wall kept in a scratch array or
read from global memory.  The medium workload (N = 48) runs tile 4 staged;
the ensemble's N = 48 and N = 64 groups run tile 16 unstaged; the large
workload (N = 128) runs tile 8 unstaged.  Each of these is compared here with
the oracle: on a few axial/azimuthal modes at N = 64 and N = 128, on members
of ensemble groups of the ensemble's own resolutions, and, at the large
workload's full resolution, through the nonlinear term (FFT work the oracle
affords) and the predictor solve on sampled modes (the oracle's dense solve of
all 32,640 modes of order 513 is out of its reach).

FP64 throughout; tolerances as in the other parity tests: ~1e-12 for a few
steps (round-off of pivot-free banded LU with influence matrices against a
dense pivoted LU of the coupled system).
"""
import functools

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
def oracle_steps(N, K, M, m_p, alpha, Re, dt, amp, seed, nsteps):
    o = Oracle(Params(N, K, M, m_p, alpha, Re, dt))
    U0 = inputs.seeded_state(N, K, M, m_p, alpha, amp, seed)
    return U0, o.step(U0, nsteps), o.beta


# ------------------------------------------------- N = 64 and N = 128 solves
@pytest.mark.parametrize("N,K,M,tile,spike", [(64, 4, 4, 0, 0), (64, 4, 4, 0, 1), (64, 4, 4, 16, 0),
                                              (128, 2, 3, 0, 0), (128, 2, 3, 0, 1), (128, 2, 3, 8, 0)])
def test_solve_paths_at_n64_and_n128(opf, N, K, M, tile, spike):
    """5 steps at N = 64 (staged tile 4, single-chain and split; unstaged tile
    16 as in the ensemble) and N = 128 (unstaged tile 4, single-chain and
    split; tile 8 as in the large workload)."""
    alpha, Re, dt = 1.25, 2000.0, 0.005
    U0, ref, beta = oracle_steps(N, K, M, 1, alpha, Re, dt, 0.05, 640 + N, 5)
    h = opf.opf_create(N, K, M, 1, alpha, Re, dt)
    opf.opf_set_option(h, "tile", tile)
    opf.opf_set_option(h, "spike", spike)
    assert opf.opf_get_option(h, "spike") == spike
    opf.opf_set_state(h, U0)
    opf.opf_step(h, 5)
    assert rel(opf.opf_get_state(h), ref) < 1e-12
    # beta' divides the flux defect's round-off (~1e-16) by sum(w G) ~ dt / 2,
    # and beta is Re / 4 times beta' (as in the large-resolution test below)
    assert abs(opf.opf_get_beta(h) - beta) < 10 * 2.2e-16 / (dt / 2) * Re / 4
    g = opf.opf_wall_residual(h)
    assert g[0] < 1e-14 and g[1] < 1e-9


# ------------------------------------------------- ensemble groups
def test_ensemble_members_of_the_workload_resolutions_match_oracle(opf):
    """Two members each of N=48 |k|<24 m<24 and N=64 |k|<32 m<32 (the
    ensemble's second and third resolutions) at different Re, stepped
    together in one batched group per shape with the ensemble's tile of 16
    modes, FP64, 2 steps: one member of each shape against the oracle."""
    shapes = [(48, 24, 24), (48, 24, 24), (64, 32, 32), (64, 32, 32)]
    Re = [1900.0, 2300.0, 2100.0, 2500.0]
    amp = [1e-2, 1e-1, 1e-1, 1e-2]
    alpha, dt = 1.25, 0.005
    n = len(shapes)
    N, K, M = zip(*shapes)
    e = opf.opf_ens_create(N, K, M, [1] * n, [alpha] * n, Re, [dt] * n)
    opf.opf_ens_set_option(e, "tile", 16)
    U0s = []
    for i, (Ni, Ki, Mi) in enumerate(shapes):
        U0s.append(inputs.seeded_state(Ni, Ki, Mi, 1, alpha, amp[i], 1705038383 + i))
        opf.opf_ens_set_state(e, i, U0s[i])
    opf.opf_ens_step(e, 2)
    for i in (1, 2):
        Ni, Ki, Mi = shapes[i]
        ref = Oracle(Params(Ni, Ki, Mi, 1, alpha, Re[i], dt)).step(U0s[i], 2)
        assert rel(opf.opf_ens_get_state(e, i), ref) < 1e-11, i


# ------------------------------------------------- the large workload's grid
@functools.lru_cache(maxsize=None)
def large_oracle():
    w = inputs.WORKLOADS["large"]
    o = Oracle(Params(w["N"], w["K"], w["M"], w["m_p"], w["alpha"], w["Re"], 2e-5))
    U0 = inputs.workload_state("large")
    return o, U0, o.nonlinear(U0)


def large_handle(opf, dt):
    w = inputs.WORKLOADS["large"]
    return opf.opf_create(w["N"], w["K"], w["M"], w["m_p"], w["alpha"], w["Re"], dt)


def test_nonlinear_term_at_the_large_resolution(opf):
    """N=128, |k|<128, m<128 (3/2 grid 384 x 384 per radial point): the
    nonlinear term of the large workload's start against the oracle."""
    o, U0, want = large_oracle()
    h = large_handle(opf, 2e-5)
    got = opf.opf_nonlinear(h, U0)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    assert rel(got, want) < 1e-13


def test_predictor_solve_at_the_large_resolution_on_sampled_modes(opf):
    """One predictor-only step (n_corr = 0: u = solve(u_j, N_j)) of the large
    workload's start, FP64, against the oracle's dense solve of sampled modes:
    the mean flow (fixed flux, beta'), low and high axial and azimuthal
    wavenumbers, both signs of k, and the corner |k| = 127, m = 127."""
    w = inputs.WORKLOADS["large"]
    K, Re = w["K"], w["Re"]
    o, U0, Nj = large_oracle()
    h = large_handle(opf, 2e-5)
    opf.opf_set_option(h, "n_corr", 0)
    opf.opf_set_state(h, U0)
    opf.opf_step(h, 1)
    U1 = opf.opf_get_state(h)
    modes = [(0, K - 1), (0, K), (0, K - 1 + 40), (1, K - 1), (1, K - 2), (2, K + 5), (17, K - 1 - 33),
             (64, K - 1), (64, K + 90), (100, K - 1 - 120), (127, 0), (127, 2 * K - 2)]
    ref = o.solve_modes(U0, Nj, modes)
    got = np.stack([U1[:, m, kk] for m, kk in modes])
    want = np.stack([ref[mk][0] for mk in modes])
    assert rel(got, want) < 1e-12
    for i, mk in enumerate(modes):  # each mode against its own size
        assert np.linalg.norm(got[i] - want[i]) <= 1e-11 * np.linalg.norm(want[i]) + 1e-18, mk
    # beta' = (1/4 - q) / sum(w G) divides a flux defect q - 1/4 of ~1e-10 by
    # sum(w G) ~ dt / 2 (G = (1/dt - c L)^-1 1 ~ dt): the ~1e-16 round-off of
    # q becomes ~1e-16 / (dt / 2) in beta', i.e. Re / 4 times that in beta
    dt = 2e-5
    assert abs(opf.opf_get_beta(h) - ref[(0, K - 1)][1] * Re / 4.0) < 10 * 2.2e-16 / (dt / 2) * Re / 4


# ------------------------------------------------- the split (two-partition) solve
@pytest.mark.parametrize("N,K,M,m_p,prec", [(48, 32, 24, 2, 1), (32, 16, 16, 1, 0), (26, 4, 5, 1, 0), (40, 6, 6, 3, 1)])
def test_split_solve_matches_the_plain_solve_and_the_oracle(opf, N, K, M, m_p, prec):
    """Where one wave of 4-mode blocks covers the grid and N is even, the
    solve substitutes the two halves of each banded system at once and joins
    them through an 8 x 8 interface system and rank-4 spikes: the same
    solution to round-off as the single-chain substitution, and the oracle's
    (FP64) after 5 steps."""
    alpha, Re, dt = 1.25, 2000.0, 0.005
    U0 = inputs.seeded_state(N, K, M, m_p, alpha, 0.05, 330 + N)
    out = []
    for spike in (0, 1):
        h = opf.opf_create(N, K, M, m_p, alpha, Re, dt)
        opf.opf_set_option(h, "precision", prec)
        opf.opf_set_option(h, "spike", spike)
        assert opf.opf_get_option(h, "spike") == spike
        opf.opf_set_state(h, U0)
        opf.opf_step(h, 5)
        out.append(opf.opf_get_state(h))
        if spike:
            g = opf.opf_wall_residual(h)
            assert g[0] < 1e-14 and g[1] < 1e-9
    assert rel(out[1], out[0]) < 1e-13
    if prec == 0:
        ref = Oracle(Params(N, K, M, m_p, alpha, Re, dt)).step(U0, 5)
        assert rel(out[1], ref) < 1e-12


def test_split_solve_defaults(opf):
    """On by default where the grid is at most one 4-mode block per SM (the
    small workload); available but off up to three (the medium workload);
    absent for odd N, N < 26 or larger grids, where setting it is a no-op."""
    w = inputs.WORKLOADS
    for name, default, avail in (("small", 1, 1), ("medium", 0, 1)):
        a = w[name]
        h = opf.opf_create(a["N"], a["K"], a["M"], a["m_p"], a["alpha"], a["Re"], a["dt"])
        assert opf.opf_get_option(h, "spike") == default, name
        opf.opf_set_option(h, "spike", 1)
        assert opf.opf_get_option(h, "spike") == avail, name
    for args in ((27, 4, 4, 1), (24, 4, 4, 1), (64, 32, 32, 1)):
        h = opf.opf_create(*args, 1.25, 2000.0, 0.005)
        assert opf.opf_get_option(h, "spike") == 0
        opf.opf_set_option(h, "spike", 1)
        assert opf.opf_get_option(h, "spike") == 0
