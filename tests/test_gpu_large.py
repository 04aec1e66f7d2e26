"""The large workload's grid (N=128, |k|<128, m<128, m_p=1, alpha=0.4,
Re=5300, broadband start of amplitude 0.3) is beyond what the oracle steps in
seconds, so it is checked by properties that hold at any size: no-slip and
wall divergence at round-off, the energy budget dE/dt = I - D (laminar
normalisation: dE^/dt = (12/Re)(I^ - D^)), and mixed precision against FP64
on the same steps."""
import numpy as np
import pytest

from paper_1705_03838_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def opf():
    from paper_1705_03838_gb300 import build, opf as _opf

    build.build()
    _opf.lib()
    return _opf


def run(opf, precision, dt, steps):
    w = inputs.WORKLOADS["large"]
    h = opf.opf_create(w["N"], w["K"], w["M"], w["m_p"], w["alpha"], w["Re"], dt)
    opf.opf_set_option(h, "precision", precision)
    opf.opf_set_state(h, inputs.workload_state("large"))
    E = []
    for _ in range(steps):
        opf.opf_step(h, 1)
        E.append(opf.opf_energy(h))
    return h, np.array(E)


def test_large_grid_properties(opf):
    w = inputs.WORKLOADS["large"]
    dt = 2e-5  # below the CFL limit of this start (~7.7e-5 at C = 0.5)
    h64, E64 = run(opf, 0, dt, 5)
    wall = opf.opf_wall_residual(h64)
    assert max(wall) < 1e-10, wall
    # centred energy budget at the middle steps
    for j in (1, 2, 3):
        lhs = (E64[j + 1][0] - E64[j - 1][0]) / (2 * dt)
        rhs = (12.0 / w["Re"]) * (E64[j][1] - E64[j][2])
        assert abs(lhs - rhs) < 2e-3 * (12.0 / w["Re"]) * abs(E64[j][2]), (j, lhs, rhs)
    h32, E32 = run(opf, 1, dt, 5)
    rel = np.abs(E32[:, 0] - E64[:, 0]) / E64[:, 0]
    assert rel.max() < 1e-8, rel
    U64, U32 = opf.opf_get_state(h64), opf.opf_get_state(h32)
    pert = U64.copy()
    r = inputs.radial_points(w["N"])
    pert[2, 0, w["K"] - 1] -= 1.0 - r * r
    assert np.linalg.norm(U32 - U64) / np.linalg.norm(pert) < 1e-5
