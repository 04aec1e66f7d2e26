"""Edge cases of the time step on the GPU: no steps, an empty ensemble, and
the size limit that the solve's shared memory sets on N (a block holds its
modes' radial columns: ~490 bytes per radial point for a tile of 4 modes,
so N ~ 460 is the largest grid; a larger one is refused at creation, before
anything is launched)."""
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


def test_zero_steps_change_nothing(opf):
    N, K, M, m_p = 16, 4, 4, 1
    h = opf.opf_create(N, K, M, m_p, 1.25, 1000.0, 0.01)
    U = inputs.seeded_state(N, K, M, m_p, 1.25, 0.1, 5)
    opf.opf_set_state(h, U)
    before, t0 = opf.opf_get_state(h), opf.opf_get_time(h)
    opf.opf_step(h, 0)
    assert np.array_equal(opf.opf_get_state(h), before) and opf.opf_get_time(h) == t0
    e = opf.opf_ens_create([N], [K], [M], [m_p], [1.25], [1000.0], [0.01])
    opf.opf_ens_set_state(e, 0, U)
    opf.opf_ens_step(e, 0)
    assert np.array_equal(opf.opf_ens_get_state(e, 0), before)


def test_empty_ensemble_is_refused(opf):
    with pytest.raises(opf.OpfError):
        opf.opf_ens_create([], [], [], [], [], [], [])


def test_radial_resolution_beyond_shared_memory_is_refused(opf):
    with pytest.raises(opf.OpfError, match="shared memory"):
        opf.opf_create(480, 1, 2, 1, 1.25, 1000.0, 0.01)


def test_largest_radial_resolution_steps(opf):
    """N = 448, two modes: the largest solve blocks (tile of 4 modes, ~220 KB
    of shared memory) step a perturbed state; the result stays finite, the
    no-slip and wall-divergence residuals stay at round-off, and the axial
    mean flow agrees with the oracle's."""
    N, K, M, m_p, alpha, Re, dt = 448, 1, 2, 1, 1.25, 500.0, 0.002
    U0 = inputs.seeded_state(N, K, M, m_p, alpha, 0.05, 9)
    h = opf.opf_create(N, K, M, m_p, alpha, Re, dt)
    opf.opf_set_state(h, U0)
    opf.opf_step(h, 2)
    U = opf.opf_get_state(h)
    assert np.isfinite(U).all()
    g = opf.opf_wall_residual(h)
    assert g[0] < 1e-12
    ref = Oracle(Params(N, K, M, m_p, alpha, Re, dt)).step(U0, 2)
    # the (0,0) mode (u_theta, u_z of the mean flow): Helmholtz solves whose
    # condition number at this near-wall spacing (~6e-6) is ~1e5, so the two
    # FP64 solvers agree to ~1e-11; 1e-8 leaves room for the stencil sums
    mean, mean_ref = U[1:, 0, K - 1], ref[1:, 0, K - 1]
    assert np.linalg.norm(mean - mean_ref) <= 1e-8 * np.linalg.norm(mean_ref)
