"""Forcing hook and frame rotation on the GPU against the oracle (FP64), the
mixed-precision path against FP64, and the argument checks."""
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


@pytest.mark.parametrize("m_p,rot", [(1, (0.3, -0.2, 0.5)), (2, (0.0, 0.0, 0.8))])
def test_rotation_matches_oracle(opf, m_p, rot):
    N, K, M, alpha, Re, dt = 16, 4, 4, 1.25, 800.0, 0.01
    U0 = inputs.seeded_state(N, K, M, m_p, alpha, 0.05, 41)
    h = opf.opf_create(N, K, M, m_p, alpha, Re, dt)
    for key, v in zip(("rot_x", "rot_y", "rot_z"), rot):
        opf.opf_set_option(h, key, v)
    opf.opf_set_state(h, U0)
    opf.opf_step(h, 20)
    ref = Oracle(Params(N, K, M, m_p, alpha, Re, dt, rotation=rot)).step(U0, 20)
    assert rel(opf.opf_get_state(h), ref) < 1e-10
    assert opf.opf_get_option(h, "rot_z") == rot[2]


def test_forcing_matches_oracle(opf):
    N, K, M, m_p, alpha, Re, dt = 16, 4, 4, 1, 1.25, 800.0, 0.01
    U0 = inputs.seeded_state(N, K, M, m_p, alpha, 0.05, 42)
    f = inputs.seeded_state(N, K, M, m_p, alpha, 0.02, 43, laminar=False)
    h = opf.opf_create(N, K, M, m_p, alpha, Re, dt)
    opf.opf_set_forcing(h, f)
    opf.opf_set_state(h, U0)
    opf.opf_step(h, 20)
    ref = Oracle(Params(N, K, M, m_p, alpha, Re, dt, forcing=f)).step(U0, 20)
    assert rel(opf.opf_get_state(h), ref) < 1e-10
    # removing the forcing restores the plain step
    opf.opf_set_forcing(h, None)
    opf.opf_set_state(h, U0)
    opf.opf_step(h, 5)
    assert rel(opf.opf_get_state(h), Oracle(Params(N, K, M, m_p, alpha, Re, dt)).step(U0, 5)) < 1e-10


def test_mixed_precision_rotation_and_forcing(opf):
    N, K, M, m_p, alpha, Re, dt = 24, 8, 8, 1, 1.25, 1500.0, 0.01
    U0 = inputs.seeded_state(N, K, M, m_p, alpha, 0.05, 44)
    f = inputs.seeded_state(N, K, M, m_p, alpha, 0.01, 45, laminar=False)
    out = []
    for prec in (0, 1):
        h = opf.opf_create(N, K, M, m_p, alpha, Re, dt)
        opf.opf_set_option(h, "precision", prec)
        opf.opf_set_option(h, "rot_x", 0.4)
        opf.opf_set_option(h, "rot_z", -0.3)
        opf.opf_set_forcing(h, f)
        opf.opf_set_state(h, U0)
        opf.opf_step(h, 30)
        out.append((opf.opf_get_state(h), opf.opf_energy(h)))
    assert abs(out[1][1][0] - out[0][1][0]) / out[0][1][0] < 1e-8
    lam = inputs.laminar_state(N, K, M)
    assert np.linalg.norm(out[1][0] - out[0][0]) / np.linalg.norm(out[0][0] - lam) < 1e-5


def test_transverse_rotation_needs_mp1(opf):
    h = opf.opf_create(16, 4, 4, 2, 1.25, 800.0, 0.01)
    with pytest.raises(opf.OpfError):
        opf.opf_set_option(h, "rot_x", 0.1)
    opf.opf_set_option(h, "rot_z", 0.1)  # axial rotation keeps the m_p symmetry
