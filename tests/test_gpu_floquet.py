"""Floquet multipliers of pipe-flow states on the GPU (batched Arnoldi over
the library's time integrations): the axisymmetric swirl multipliers
exp(-j_{1,n}^2 T / Re) of Hagen-Poiseuille flow, agreement with the oracle's
Arnoldi on the same starting vector, and batched problems equal to single
ones."""
import numpy as np
import pytest
from scipy.special import jn_zeros

from oracle import floquet_oracle as fo
from oracle.opf_oracle import Oracle, Params
from paper_1705_03838_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def opf():
    from paper_1705_03838_gb300 import build, opf as _opf

    build.build()
    _opf.lib()
    return _opf


def test_swirl_multipliers(opf):
    N, K, M, Re, T, dt = 32, 4, 4, 100.0, 1.0, 0.01
    U = inputs.laminar_state(N, K, M)
    start = np.zeros_like(U)
    start[1, 0, K - 1] = np.random.default_rng(7).normal(size=N)
    start[1, 0, K - 1, -1] = 0.0
    ev, res = opf.opf_floquet(N, K, M, 1, 1.25, Re, [U], [T], [0.0], 12, 12, dt, start=[start])
    for mu in np.exp(-jn_zeros(1, 3) ** 2 * T / Re):
        assert np.min(np.abs(ev[0] - mu)) < 2e-5 * mu, (mu, ev[0])


def test_matches_oracle_arnoldi_on_the_same_start(opf):
    N, K, M, Re, T, dt = 12, 3, 3, 100.0, 2.0, 0.05
    lam = inputs.laminar_state(N, K, M)
    U = lam + inputs.seeded_state(N, K, M, 1, 1.25, 1e-3, 21, laminar=False)
    start = inputs.seeded_state(N, K, M, 1, 1.25, 1.0, 22, laminar=False)
    k = 20
    ev, res = opf.opf_floquet(N, K, M, 1, 1.25, Re, [U], [T], [0.0], k, 4, dt, start=[start])
    o = Oracle(Params(N, K, M, 1, 1.25, Re, dt))
    ref = fo.floquet(o, U, T, 0.0, fo.pack(start, K, M), k)
    for e in ev[0][:3]:
        assert np.min(np.abs(ref - e)) < 1e-6 * abs(e), (ev[0], ref[:6])


def test_batched_equals_single(opf):
    N, K, M, Re, dt = 12, 3, 3, 150.0, 0.05
    lam = inputs.laminar_state(N, K, M)
    U1 = lam + inputs.seeded_state(N, K, M, 1, 1.25, 1e-3, 31, laminar=False)
    U2 = lam + inputs.seeded_state(N, K, M, 1, 1.25, 2e-3, 32, laminar=False)
    both, r2 = opf.opf_floquet(N, K, M, 1, 1.25, Re, [U1, U2], [1.0, 1.0], [0.0, 0.3], 10, 3, dt, seed=5)
    one, r1 = opf.opf_floquet(N, K, M, 1, 1.25, Re, [U1], [1.0], [0.0], 10, 3, dt, seed=5)
    np.testing.assert_array_equal(both[0], one[0])
    assert np.isfinite(both).all() and np.isfinite(r2).all()
    assert (np.abs(both) < 1.0).all()  # laminar flow at Re = 150 is stable
