"""A user radial mesh (paper section 2: the radial points may be supplied
instead of computed) through opf_create_mesh, against the oracle on the same
points.  The mesh used here is clustered towards the axis rather than the
wall, so every radial quantity (stencils, 1/r, quadrature, operators,
influence data, the laminar profile of the mixed-precision split) differs
from the default mesh's."""
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


@pytest.mark.parametrize("N,K,M,m_p", [(16, 4, 4, 1), (24, 3, 5, 2)])
def test_steps_on_a_user_mesh_match_oracle(opf, N, K, M, m_p):
    alpha, Re, dt = 1.25, 800.0, 0.01
    r = inputs.stretched_mesh(N)
    U0 = inputs.seeded_state(N, K, M, m_p, alpha, 0.05, 123, r=r)
    o = Oracle(Params(N, K, M, m_p, alpha, Re, dt, r=r))
    ref = o.step(U0, 3)
    h = opf.opf_create_mesh(N, K, M, m_p, alpha, Re, dt, r)
    opf.opf_set_state(h, U0)
    opf.opf_step(h, 3)
    assert rel(opf.opf_get_state(h), ref) < 1e-12
    e, e_ref = opf.opf_energy(h), o.energy(ref)
    assert np.abs(e - e_ref).max() < 1e-12 * max(1.0, Re / 4)
    g = opf.opf_wall_residual(h)
    assert g[0] < 1e-14 and g[1] < 1e-10
    # the same state on the default mesh gives a different result
    h0 = opf.opf_create(N, K, M, m_p, alpha, Re, dt)
    opf.opf_set_state(h0, U0)
    opf.opf_step(h0, 3)
    assert rel(opf.opf_get_state(h0), ref) > 1e-6


def test_nonlinear_term_and_mixed_steps_on_a_user_mesh(opf):
    N, K, M, m_p, alpha, Re, dt = 20, 4, 6, 1, 1.25, 1000.0, 0.01
    r = inputs.stretched_mesh(N)
    U0 = inputs.seeded_state(N, K, M, m_p, alpha, 0.1, 7, r=r)
    o = Oracle(Params(N, K, M, m_p, alpha, Re, dt, r=r))
    h = opf.opf_create_mesh(N, K, M, m_p, alpha, Re, dt, r)
    want = o.nonlinear(U0)
    assert np.abs(opf.opf_nonlinear(h, U0) - want).max() <= 1e-12 * np.abs(want).max()
    # mixed precision: FP32 transforms of the perturbation, base flow split on the user mesh
    opf.opf_set_option(h, "precision", 1)
    opf.opf_set_state(h, U0)
    opf.opf_step(h, 20)
    ref = o.step(U0, 20)
    assert abs(opf.opf_energy(h)[0] - o.energy(ref)[0]) / o.energy(ref)[0] < 1e-6


def test_hagen_poiseuille_is_steady_on_a_user_mesh(opf):
    N, K, M = 24, 3, 3
    r = inputs.stretched_mesh(N)
    lam = inputs.laminar_state(N, K, M, r=r)
    h = opf.opf_create_mesh(N, K, M, 1, 1.25, 2000.0, 0.01, r)
    opf.opf_set_state(h, lam)
    opf.opf_step(h, 100)
    assert np.abs(opf.opf_get_state(h) - lam).max() < 1e-12
    assert np.allclose(opf.opf_energy(h), 1.0, atol=1e-13)


def test_invalid_user_mesh_is_rejected(opf):
    r = inputs.stretched_mesh(16)
    with pytest.raises(opf.OpfError):
        opf.opf_create_mesh(16, 4, 4, 1, 1.25, 100.0, 0.01, r[::-1])
    with pytest.raises(opf.OpfError):
        opf.opf_create_mesh(16, 4, 4, 1, 1.25, 100.0, 0.01, r * 0.9)  # no wall point
